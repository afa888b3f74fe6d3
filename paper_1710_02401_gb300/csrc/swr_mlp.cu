// swr_mlp.cu -- small BF16 multilayer perceptron with its own training kernels.
//
// Predicts the initial interface traces of the SWR iteration from subdomain
// descriptors (learned initial guess; not part of the paper's method, which
// starts from g^(0) = 0).  Architecture: n_in -> width -> ... -> width -> n_out,
// tanh after every hidden layer, identity output.  Weights are kept in FP32
// (master copy, Adam moments) and rounded to BF16 for the products; every
// product runs on the 5th-generation tensor cores (tcgen05.mma kind::f16, BF16
// inputs, FP32 accumulation in tensor memory).  Training minimises the mean
// squared error with Adam.
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
// ------------------------------------------------- tcgen05 (5th-gen tensor cores)
//
// The same product on the Blackwell tensor cores: a CTA computes a 128 x 64 tile
// of C with tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor
// memory).  K advances 64 at a time: the CTA stages the A (128 x 64) and B
// (64 x 64) blocks into shared memory as K-major core matrices (8 rows x 16
// bytes each, no swizzle, zero outside the matrices), one thread issues four
// K = 16 MMAs and commits them to an mbarrier, every thread waits for it
// (bounded: on timeout the flag records it and the CTA frees its tensor memory
// and returns), and the next block is staged.  The accumulator is read back
// with tcgen05.ld (warp w reads rows 32w..32w+31).
#define TC_M 128
#define TC_N 64
#define TC_K 64
#define TC_THREADS 128
#define TC_SPIN (1LL << 22)

__device__ inline unsigned tc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// lbo = bytes between core matrices adjacent in K, sbo = bytes between core
// matrices adjacent in M (N), descriptor version 1.
__device__ inline unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    unsigned long long d = (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ULL << 46;
    return d;
}

// Byte offset of element (row, k) of a block stored as K-major core matrices:
// core (row/8, k/8) at ((row/8) * TC_K/8 + k/8) * 128, rows 16 bytes apart inside.
__device__ inline int tc_off(int row, int k) {
    return ((row >> 3) * (TC_K / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ inline bool tc_wait(unsigned mbar, int parity) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int TA, int TB>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M,
                                                        int N, int K, int lda, int ldb, int ldc, int accumulate,
                                                        int* err) {
    __shared__ __align__(1024) unsigned char As[TC_M * TC_K * 2];
    __shared__ __align__(1024) unsigned char Bs[TC_N * TC_K * 2];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_slot;
    __shared__ int s_fail;
    const int tm = blockIdx.y * TC_M, tn = blockIdx.x * TC_N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_slot)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, N, M
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_N >> 3) << 17) |
                           ((unsigned)(TC_M >> 4) << 24);
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    __nv_bfloat16* as = reinterpret_cast<__nv_bfloat16*>(As);
    __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(Bs);
    int parity = 0;
    for (int k0 = 0; k0 < K; k0 += TC_K) {
        for (int e = threadIdx.x; e < TC_M * TC_K; e += TC_THREADS) {
            // coalesced along the contiguous global index
            const int m = TA ? e % TC_M : e / TC_K, k = TA ? e / TC_M : e % TC_K;
            const int gm = tm + m, gk = k0 + k;
            __nv_bfloat16 a = zero;
            if (gm < M && gk < K) a = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            as[tc_off(m, k) >> 1] = a;
        }
        for (int e = threadIdx.x; e < TC_N * TC_K; e += TC_THREADS) {
            const int n = TB ? e / TC_K : e % TC_N, k = TB ? e % TC_K : e / TC_N;
            const int gn = tn + n, gk = k0 + k;
            __nv_bfloat16 b = zero;
            if (gn < N && gk < K) b = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            bs[tc_off(n, k) >> 1] = b;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
                const unsigned long long ad = tc_desc(tc_smem(As) + kk * 256, 128, 1024);
                const unsigned long long bd = tc_desc(tc_smem(Bs) + kk * 256, 128, 1024);
                const unsigned acc = (k0 > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(&mbar))
                         : "memory");
        }
        if (!tc_wait(tc_smem(&mbar), parity)) s_fail = 1;
        parity ^= 1;
        __syncthreads();
        if (s_fail) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            tc_wait(tc_smem(&mbar), parity ^ 1);  // bounded: the products in flight, before the memory is freed
        }
    } else {
        const int row = tm + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            unsigned r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = tn + c0 + j;
                    if (col < N) {
                        float* p = C + (long long)row * ldc + col;
                        const float x = __uint_as_float(r[j]);
                        *p = accumulate ? *p + x : x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
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
    int* flag = nullptr;               // set by a tensor-core product whose completion wait timed out
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
                 int ldb, int ldc, int accumulate, int* flag) {
    dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M);
    k_gemm_tc<TA, TB><<<grid, TC_THREADS, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, accumulate, flag);
}

// Reads the tensor-core timeout flag (synchronises the stream).
static swr_status check_flag(swr_mlp* m) {
    int f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, m->flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_fail(m, SWR_ECUDA, cudaGetErrorString(e));
    if (f) return mlp_fail(m, SWR_ETIMEOUT, "a tensor-core product did not complete (bounded wait)");
    return SWR_OK;
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
    if (e == cudaSuccess) e = cudaMalloc(&m->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->flag, 0, sizeof(int), m->stream);
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
        gemm<0, 0>(s, m->act_b[l], m->wb + m->w_off[l], m->act_f[l + 1], batch, dout, din, din, dout, dout, 0, m->flag);
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
    return check_flag(m);
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
        gemm<1, 0>(s, m->act_b[l], m->dzb, m->g + m->w_off[l], din, dout, batch, din, dout, dout, 0, m->flag);
        k_colsum<<<(dout + 255) / 256, 256, 0, s>>>(m->dz, m->g + m->b_off[l], batch, dout);
        if (l > 0) {
            // dH = dZ W^T  (batch x din), then through tanh of layer l
            gemm<0, 1>(s, m->dzb, m->wb + m->w_off[l], m->dh, batch, din, dout, dout, dout, din, 0, m->flag);
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
    return check_flag(m);
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
    cudaFree(m->flag);
    delete m;
}

extern "C" const char* swr_mlp_last_error(const swr_mlp* m) { return m ? m->err.c_str() : ""; }
