// swr_mlp.cu -- small BF16 multilayer perceptron with its own training kernels.
//
// Predicts the initial interface traces of the SWR iteration from subdomain
// descriptors (learned initial guess; not part of the paper's method, which
// starts from g^(0) = 0).  Architecture: n_in -> width -> ... -> width -> n_out,
// tanh after every hidden layer, identity output.  Weights are kept in FP32
// (master copy, Adam moments) and rounded to BF16 for the products; every
// product runs on the tensor cores with mma.sync m16n8k16 (BF16 inputs, FP32
// accumulation).  Training minimises the mean squared error with Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "swr_internal.cuh"

namespace swr {

// C[M x N] (FP32) = op(A) op(B), A, B in BF16 row-major.
//   TA = 0: A is M x K (lda);  TA = 1: A is stored K x M (lda), op(A) = A^T
//   TB = 0: B is K x N (ldb);  TB = 1: B is stored N x K (ldb), op(B) = B^T
// 64 x 64 tile per CTA, 4 warps of 32 x 32, K step 16.
template <int TA, int TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                                                   int K, int lda, int ldb, int ldc, int accumulate) {
    __shared__ __nv_bfloat16 As[64][16 + 8];   // [m][k]
    __shared__ __nv_bfloat16 Bs[64][16 + 8];   // [n][k]
    const int tm = blockIdx.y * 64, tn = blockIdx.x * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 128) {
            const int m = e / 16, k = e % 16;
            const int gm = tm + m, gk = k0 + k;
            __nv_bfloat16 a = zero;
            if (gm < M && gk < K) a = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[m][k] = a;
            const int gn = tn + m;
            __nv_bfloat16 b = zero;
            if (gn < N && gk < K) b = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[m][k] = b;
        }
        __syncthreads();
        unsigned af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r0 = wm + 16 * i + g;
            af[i][0] = *(const unsigned*)&As[r0][2 * tg];
            af[i][1] = *(const unsigned*)&As[r0 + 8][2 * tg];
            af[i][2] = *(const unsigned*)&As[r0][2 * tg + 8];
            af[i][3] = *(const unsigned*)&As[r0 + 8][2 * tg + 8];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n0 = wn + 8 * j + g;
            bfr[j][0] = *(const unsigned*)&Bs[n0][2 * tg];
            bfr[j][1] = *(const unsigned*)&Bs[n0][2 * tg + 8];
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = tm + wm + 16 * i + g + (r >= 2 ? 8 : 0);
                const int col = tn + wn + 8 * j + 2 * tg + (r & 1);
                if (row < M && col < N) {
                    float* p = C + (long long)row * ldc + col;
                    *p = accumulate ? *p + acc[i][j][r] : acc[i][j][r];
                }
            }
}

__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(x[e]);
}

// z = y + bias (row broadcast); act: h = tanh(z) (hidden) or z (output)
__global__ void k_bias_act(float* y, const float* bias, int rows, int cols, int act, __nv_bfloat16* hb, float* hf) {
    const long long n = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % cols);
        float z = y[e] + bias[c];
        float h = act ? tanhf(z) : z;
        y[e] = z;
        if (hf) hf[e] = h;
        if (hb) hb[e] = __float2bfloat16(h);
    }
}

// dZ = dH * (1 - h^2) for tanh layers; also writes the BF16 copy.
__global__ void k_tanh_back(const float* dh, const float* h, float* dz, __nv_bfloat16* dzb, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float d = dh[e] * (1.f - h[e] * h[e]);
        dz[e] = d;
        dzb[e] = __float2bfloat16(d);
    }
}

// Mean squared error: dY = 2 (y - t) / (rows*cols), loss partials per block.
__global__ void k_mse(const float* y, const float* t, float* dy, __nv_bfloat16* dyb, long long n, float* part) {
    __shared__ float red[256];
    float acc = 0.f;
    const float sc = 2.f / (float)n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float d = y[e] - t[e];
        acc += d * d;
        dy[e] = sc * d;
        dyb[e] = __float2bfloat16(sc * d);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// db[c] = sum_rows dz[r][c]
__global__ void k_colsum(const float* dz, float* db, int rows, int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += dz[(long long)r * cols + c];
    db[c] = acc;
}

// Adam on FP32 master parameters; refreshes the BF16 copies of the weights.
__global__ void k_adam(float* p, const float* gr, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float g = gr[e];
        float mm = b1 * m[e] + (1.f - b1) * g;
        float vv = b2 * v[e] + (1.f - b2) * g * g;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

}  // namespace swr

using namespace swr;

struct swr_mlp {
    std::string err;
    int n_in, width, n_hidden, n_out, n_layers;
    std::vector<int> dims;             // n_layers + 1
    std::vector<long long> w_off, b_off;  // into the parameter vector
    long long n_params = 0;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // params, grads, Adam moments
    __nv_bfloat16* wb = nullptr;       // BF16 copy of the parameter vector
    int cap_batch = 0;
    std::vector<float*> act_f;         // per layer output (FP32), layer 0 = input copy
    std::vector<__nv_bfloat16*> act_b; // BF16 copies
    float *dz = nullptr, *dh = nullptr, *part = nullptr;
    __nv_bfloat16* dzb = nullptr;
    long long adam_t = 0;
};

static swr_status mlp_fail(swr_mlp* m, swr_status s, const char* msg) {
    if (m) m->err = msg;
    return s;
}

#define MCU(call)                                                         \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return mlp_fail(m, SWR_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

static unsigned gsz(long long n) { return (unsigned)(n < 256LL * 4096 ? (n + 255) / 256 : 4096); }

static swr_status ensure_batch(swr_mlp* m, int batch) {
    if (batch <= m->cap_batch) return SWR_OK;
    for (float* f : m->act_f) cudaFree(f);
    for (__nv_bfloat16* b : m->act_b) cudaFree(b);
    cudaFree(m->dz);
    cudaFree(m->dh);
    cudaFree(m->dzb);
    m->act_f.assign(m->n_layers + 1, nullptr);
    m->act_b.assign(m->n_layers + 1, nullptr);
    int wmax = 0;
    for (int d : m->dims) wmax = d > wmax ? d : wmax;
    for (int l = 0; l <= m->n_layers; ++l) {
        MCU(cudaMalloc(&m->act_f[l], sizeof(float) * (size_t)batch * m->dims[l]));
        MCU(cudaMalloc(&m->act_b[l], sizeof(__nv_bfloat16) * (size_t)batch * m->dims[l]));
    }
    MCU(cudaMalloc(&m->dz, sizeof(float) * (size_t)batch * wmax));
    MCU(cudaMalloc(&m->dh, sizeof(float) * (size_t)batch * wmax));
    MCU(cudaMalloc(&m->dzb, sizeof(__nv_bfloat16) * (size_t)batch * wmax));
    m->cap_batch = batch;
    return SWR_OK;
}

template <int TA, int TB>
static void gemm(cudaStream_t st, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N, int K, int lda,
                 int ldb, int ldc, int accumulate) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm_bf16<TA, TB><<<grid, 128, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, accumulate);
}

extern "C" swr_status swr_mlp_create(int n_in, int width, int n_hidden, int n_out, void* stream, swr_mlp** out) {
    if (!out || n_in < 1 || width < 1 || n_hidden < 1 || n_out < 1 || n_in > 65536 || width > 65536 || n_out > 65536)
        return SWR_EINVAL;
    swr_mlp* m = new swr_mlp();
    m->n_in = n_in;
    m->width = width;
    m->n_hidden = n_hidden;
    m->n_out = n_out;
    m->n_layers = n_hidden + 1;
    m->stream = (cudaStream_t)stream;
    m->dims.push_back(n_in);
    for (int i = 0; i < n_hidden; ++i) m->dims.push_back(width);
    m->dims.push_back(n_out);
    long long off = 0;
    for (int l = 0; l < m->n_layers; ++l) {
        m->w_off.push_back(off);
        off += (long long)m->dims[l] * m->dims[l + 1];
        m->b_off.push_back(off);
        off += m->dims[l + 1];
    }
    m->n_params = off;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->p, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(float) * 4096);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * off, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * off, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->p, 0, sizeof(float) * off, m->stream);
    if (e != cudaSuccess) {
        delete m;
        return SWR_ENOMEM;
    }
    *out = m;
    return SWR_OK;
}

extern "C" swr_status swr_mlp_param_count(swr_mlp* m, size_t* n) {
    if (!m || !n) return SWR_EINVAL;
    *n = (size_t)m->n_params;
    return SWR_OK;
}

extern "C" swr_status swr_mlp_set_params(swr_mlp* m, const float* host, size_t n) {
    if (!m || !host || n != (size_t)m->n_params) return mlp_fail(m, SWR_EINVAL, "parameter count mismatch");
    MCU(cudaMemcpyAsync(m->p, host, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaMemsetAsync(m->m, 0, sizeof(float) * n, m->stream));
    MCU(cudaMemsetAsync(m->v, 0, sizeof(float) * n, m->stream));
    m->adam_t = 0;
    MCU(cudaStreamSynchronize(m->stream));
    return SWR_OK;
}

extern "C" swr_status swr_mlp_get_params(swr_mlp* m, float* host, size_t n) {
    if (!m || !host || n != (size_t)m->n_params) return mlp_fail(m, SWR_EINVAL, "parameter count mismatch");
    MCU(cudaMemcpyAsync(host, m->p, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    return SWR_OK;
}

// Forward pass on device arrays: x [batch x n_in] FP32 -> y [batch x n_out] FP32.
static swr_status forward(swr_mlp* m, const float* x, int batch) {
    swr_status st = ensure_batch(m, batch);
    if (st != SWR_OK) return st;
    cudaStream_t s = m->stream;
    k_to_bf16<<<gsz(m->n_params), 256, 0, s>>>(m->p, m->wb, m->n_params);
    MCU(cudaMemcpyAsync(m->act_f[0], x, sizeof(float) * (size_t)batch * m->n_in, cudaMemcpyDeviceToDevice, s));
    k_to_bf16<<<gsz((long long)batch * m->n_in), 256, 0, s>>>(x, m->act_b[0], (long long)batch * m->n_in);
    for (int l = 0; l < m->n_layers; ++l) {
        const int din = m->dims[l], dout = m->dims[l + 1];
        const bool last = (l == m->n_layers - 1);
        gemm<0, 0>(s, m->act_b[l], m->wb + m->w_off[l], m->act_f[l + 1], batch, dout, din, din, dout, dout, 0);
        // act_f[l+1] holds z; hidden layers keep h = tanh(z) in act_f and BF16 in act_b
        k_bias_act<<<gsz((long long)batch * dout), 256, 0, s>>>(m->act_f[l + 1], m->p + m->b_off[l], batch, dout,
                                                                last ? 0 : 1, m->act_b[l + 1], m->act_f[l + 1]);
    }
    return SWR_OK;
}

extern "C" swr_status swr_mlp_forward(swr_mlp* m, const float* x_dev, int batch, float* y_dev) {
    if (!m || !x_dev || !y_dev || batch < 1) return mlp_fail(m, SWR_EINVAL, "bad argument");
    swr_status st = forward(m, x_dev, batch);
    if (st != SWR_OK) return st;
    MCU(cudaMemcpyAsync(y_dev, m->act_f[m->n_layers], sizeof(float) * (size_t)batch * m->n_out,
                        cudaMemcpyDeviceToDevice, m->stream));
    MCU(cudaGetLastError());
    return SWR_OK;
}

// One Adam step on the mean squared error; loss_host (nullable) receives the
// loss before the update, grad_host (nullable) the gradient (n_params floats).
extern "C" swr_status swr_mlp_train_step(swr_mlp* m, const float* x_dev, const float* t_dev, int batch, float lr,
                                         float* loss_host, float* grad_host) {
    if (!m || !x_dev || !t_dev || batch < 1) return mlp_fail(m, SWR_EINVAL, "bad argument");
    swr_status st = forward(m, x_dev, batch);
    if (st != SWR_OK) return st;
    cudaStream_t s = m->stream;
    const int L = m->n_layers;
    const long long nout = (long long)batch * m->n_out;
    const unsigned nb = gsz(nout) < 1024 ? gsz(nout) : 1024;
    // output layer: dZ = dY
    k_mse<<<nb, 256, 0, s>>>(m->act_f[L], t_dev, m->dz, m->dzb, nout, m->part);
    for (int l = L - 1; l >= 0; --l) {
        const int din = m->dims[l], dout = m->dims[l + 1];
        // dW = X^T dZ  (din x dout), db = colsum dZ
        gemm<1, 0>(s, m->act_b[l], m->dzb, m->g + m->w_off[l], din, dout, batch, din, dout, dout, 0);
        k_colsum<<<(dout + 255) / 256, 256, 0, s>>>(m->dz, m->g + m->b_off[l], batch, dout);
        if (l > 0) {
            // dH = dZ W^T  (batch x din), then through tanh of layer l
            gemm<0, 1>(s, m->dzb, m->wb + m->w_off[l], m->dh, batch, din, dout, dout, dout, din, 0);
            k_tanh_back<<<gsz((long long)batch * din), 256, 0, s>>>(m->dh, m->act_f[l], m->dz, m->dzb,
                                                                    (long long)batch * din);
        }
    }
    if (loss_host) {
        std::vector<float> part(nb);
        MCU(cudaMemcpyAsync(part.data(), m->part, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
        MCU(cudaStreamSynchronize(s));
        double acc = 0;
        for (float x : part) acc += x;
        *loss_host = (float)(acc / (double)nout);
    }
    if (grad_host) {
        MCU(cudaMemcpyAsync(grad_host, m->g, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, s));
        MCU(cudaStreamSynchronize(s));
    }
    if (lr > 0.f) {
        m->adam_t += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        k_adam<<<gsz(m->n_params), 256, 0, s>>>(m->p, m->g, m->m, m->v, m->n_params, lr, b1, b2, 1e-8f, c1, c2);
    }
    MCU(cudaGetLastError());
    return SWR_OK;
}

extern "C" void swr_mlp_destroy(swr_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (float* f : m->act_f) cudaFree(f);
    for (__nv_bfloat16* b : m->act_b) cudaFree(b);
    cudaFree(m->dz);
    cudaFree(m->dh);
    cudaFree(m->dzb);
    cudaFree(m->p);
    cudaFree(m->g);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->wb);
    cudaFree(m->part);
    delete m;
}

extern "C" const char* swr_mlp_last_error(const swr_mlp* m) { return m ? m->err.c_str() : ""; }
