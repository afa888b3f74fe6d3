// swr_robin.cu -- the response of the step matrix to the Robin source,
// w^n = kappa dt G b'^n, for every step of a window before the window runs.
//
// In imaginary time a step is (Sec. 5.2, system SIT; Sec. 5.4 steps 2 and 4)
//     y^{n+1} = G (y^n / s_n + kappa dt b'^{n+1}) = (G y^n) / s_n + w^{n+1},
// and the Robin source of the previous iteration's traces is known for every
// step before the window starts.  With w^{n+1} at hand, the product G y^n no
// longer waits for the global normalisation s_n: the window forms it while
// the partials of s_n travel, and scales it afterwards.
//
// b' lies in a small subspace.  It is the Galerkin load of the Robin data on
// the interior edges (Sec. 5.1, Eq. RTC): in the orthonormal tensor basis
// (index e = a + kd b) an edge slot of coordinate 0 contributes
// Lv0[a] h[b] and one of coordinate 1 contributes h[a] Lv1[b], with Lv the
// basis values on that edge and h the tangential Galerkin sums of the Robin
// data.  As a kd x kd matrix, b' = U X^T + Y V^T with U (V) the edge-value
// vectors of the present slots of coordinate 0 (1).  So
//     G b' = GE h,   GE = G [E_1 ... E_J],
// where GE has one column per (slot, tangential index) pair: J = 4 kd at
// most, against K = kd^2 columns of G.  GE is formed once at assembly.
//
// h is recovered from the stored b' of every step by the gauge-fixed
// decomposition (X^T V = 0):
//     Y = B V (V^T V)^{-1},   X^T = (U^T U)^{-1} U^T (B - Y V^T),
// exact (to rounding) for every b' of that form; the same kernel serves a
// fresh iteration and a restored trace window, so a run resumed from a
// checkpoint repeats the uninterrupted run bit for bit.  One electron:
// b' = sum_s g_s Lv_s and h = (U^T U)^{-1} U^T b'.
//
// Then W[n] = kappa dt GE H[n] for n = 0..n_prev (the previous window; later
// steps hold its last value) is a batched product on the FP32 pipes in
// double-single, tiles of 64 rows x 64 steps.
#include <math.h>

#include "swr_internal.cuh"

namespace swr {

#define RB_THREADS 256

// Present edge slots of a subdomain in slot order (coordinate 0 first):
// their number and, per slot, its column block (-1 when absent).
__host__ __device__ inline int robin_slots(const SubDev& s, int (&blk)[4]) {
    int n = 0;
    for (int sl = 0; sl < 4; ++sl) blk[sl] = (s.gam_off[sl] >= 0 && sl / 2 < s.N) ? n++ : -1;
    return n;
}

// Columns of GE (and entries of h per step).
__host__ __device__ inline int robin_cols(const SubDev& s) {
    int blk[4];
    const int n = robin_slots(s, blk);
    return s.N == 2 ? n * s.kd : n;
}

// Edge values of slot sl (coordinate sl / 2, lo edge for even sl, hi for odd).
__device__ inline const double* robin_edge(const SwrDeviceView& v, const SubDev& s, int sl) {
    const T1Layout lay(s.q, s.kd);
    return v.arena + s.t1[sl / 2] + lay.Lv() + (long long)((sl & 1) ? 3 : 0) * s.kd;
}

// GE[r][j] (pairs) from the FP64 step-matrix inverse: for the slot of column
// block j / kd and tangential index m = j % kd,
//   coordinate 0: sum_a G[r][a + kd m] Lv0[a];  coordinate 1: sum_b G[r][m + kd b] Lv1[b].
__global__ void k_robin_ge(SwrDeviceView v) {
    const SubDev& s = v.sub[blockIdx.y];
    const int K = s.K, kd = s.kd, J = robin_cols(s);
    if (J == 0) return;
    int blk[4];
    robin_slots(s, blk);
    const double* G = v.arena + s.Gm;
    float2* GE = reinterpret_cast<float2*>(v.arena + s.GE);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)K * J;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / J), j = (int)(e - (long long)r * J);
        const int b = s.N == 2 ? j / kd : j, m = s.N == 2 ? j - b * kd : 0;
        int sl = 0;
        while (blk[sl] != b) ++sl;
        const double* Lv = robin_edge(v, s, sl);
        const double* g = G + (long long)r * K;
        double acc = 0;
        if (s.N == 1) {
            for (int a = 0; a < kd; ++a) acc = fma(g[a], Lv[a], acc);
        } else if (sl < 2) {
            for (int a = 0; a < kd; ++a) acc = fma(g[a + kd * m], Lv[a], acc);
        } else {
            for (int bb = 0; bb < kd; ++bb) acc = fma(g[m + kd * bb], Lv[bb], acc);
        }
        GE[e] = dsp_split_int(acc);
    }
}

// Inverse of the Gram matrix of n <= 2 vectors of length kd (row-major n x n).
__device__ inline void gram_inverse(const double* const* vec, int n, int kd, double* inv) {
    double g[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0;
            for (int a = 0; a < kd; ++a) acc = fma(vec[i][a], vec[j][a], acc);
            g[i * n + j] = acc;
        }
    if (n == 1) {
        inv[0] = 1.0 / g[0];
    } else if (n == 2) {
        const double det = g[0] * g[3] - g[1] * g[2];
        inv[0] = g[3] / det;
        inv[1] = -g[1] / det;
        inv[2] = -g[2] / det;
        inv[3] = g[0] / det;
    }
}

// H[n] (pairs, J per step) from the stored b'^n, n = 0..n_prev, by the
// gauge-fixed decomposition above.  Steps strided over blockIdx.x.
__global__ void __launch_bounds__(RB_THREADS) k_robin_h(SwrDeviceView v, const int* win_prev) {
    const SubDev& s = v.sub[blockIdx.y];
    const int wp = win_prev[s.inst];
    const int K = s.K, kd = s.kd, J = robin_cols(s);
    if (wp <= 0 || J == 0 || (int)blockIdx.x > wp) return;
    int blk[4];
    robin_slots(s, blk);
    __shared__ const double* U[2];
    __shared__ const double* V[2];
    __shared__ int slU[2], slV[2], p, q;
    __shared__ double GUi[4], GVi[4];
    __shared__ double Ys[64][2], UY[2][2];
    __shared__ double Qs[2][64];
    extern __shared__ double Bm[];  // K
    if (threadIdx.x == 0) {
        p = q = 0;
        for (int sl = 0; sl < 4; ++sl) {
            if (blk[sl] < 0) continue;
            if (sl < 2) {
                slU[p] = sl;
                U[p++] = robin_edge(v, s, sl);
            } else {
                slV[q] = sl;
                V[q++] = robin_edge(v, s, sl);
            }
        }
        gram_inverse(U, p, kd, GUi);
        gram_inverse(V, q, kd, GVi);
    }
    __syncthreads();
    float2* H = reinterpret_cast<float2*>(v.arena + s.Hr);
    for (int n = blockIdx.x; n <= wp; n += gridDim.x) {
        const double* b = v.arena + s.bvec + (long long)n * K;
        float2* h = H + (long long)n * J;
        if (s.N == 1) {
            // h = (U^T U)^{-1} U^T b'
            if (threadIdx.x < 32) {
                double t[2] = {0, 0};
                for (int i = 0; i < p; ++i) {
                    double acc = 0;
                    for (int a = threadIdx.x; a < kd; a += 32) acc = fma(U[i][a], b[a], acc);
                    t[i] = warp_sum(acc);
                }
                if (threadIdx.x < p) {
                    const int i = threadIdx.x;
                    double x = 0;
                    for (int k = 0; k < p; ++k) x = fma(GUi[i * p + k], t[k], x);
                    h[blk[slU[i]]] = dsp_split_int(x);
                }
            }
            continue;
        }
        for (int e = threadIdx.x; e < K; e += RB_THREADS) Bm[e] = b[e];
        __syncthreads();
        // Y = B V (V^T V)^{-1}: B[a][bb] = b'[a + kd bb]
        for (int it = threadIdx.x; it < kd * q; it += RB_THREADS) {
            const int a = it / q, t = it - a * q;
            double acc = 0;
            for (int bb = 0; bb < kd; ++bb) acc = fma(Bm[a + kd * bb], V[t][bb], acc);
            Ys[a][t] = acc;  // (B V)[a][t], scaled below
        }
        // Q = U^T B
        for (int it = threadIdx.x; it < kd * p; it += RB_THREADS) {
            const int t = it / kd, bb = it - t * kd;
            double acc = 0;
            for (int a = 0; a < kd; ++a) acc = fma(U[t][a], Bm[a + kd * bb], acc);
            Qs[t][bb] = acc;
        }
        __syncthreads();
        if (threadIdx.x < kd) {
            const int a = threadIdx.x;
            double y[2] = {0, 0};
            for (int sidx = 0; sidx < q; ++sidx)
                for (int t = 0; t < q; ++t) y[sidx] = fma(Ys[a][t], GVi[t * q + sidx], y[sidx]);
            for (int sidx = 0; sidx < q; ++sidx) Ys[a][sidx] = y[sidx];  // row a is this thread's alone
        }
        __syncthreads();
        // U^T Y (p x q)
        if (threadIdx.x < p * q) {
            const int t = threadIdx.x / q, u = threadIdx.x - t * q;
            double acc = 0;
            for (int a = 0; a < kd; ++a) acc = fma(U[t][a], Ys[a][u], acc);
            UY[t][u] = acc;
        }
        __syncthreads();
        // h: X^T = (U^T U)^{-1} (U^T B - (U^T Y) V^T) for coordinate-0 slots, Y for coordinate 1
        for (int it = threadIdx.x; it < kd * (p + q); it += RB_THREADS) {
            const int sidx = it / kd, m = it - sidx * kd;
            double x;
            int sl;
            if (sidx < p) {
                x = 0;
                for (int t = 0; t < p; ++t) {
                    double r = Qs[t][m];
                    for (int u = 0; u < q; ++u) r = fma(-UY[t][u], V[u][m], r);
                    x = fma(GUi[sidx * p + t], r, x);
                }
                sl = slU[sidx];
            } else {
                x = Ys[m][sidx - p];
                sl = slV[sidx - p];
            }
            h[blk[sl] * kd + m] = dsp_split_int(x);
        }
        __syncthreads();
    }
}

// W[n][r] = kappa dt sum_j GE[r][j] H[n][j] (pairs, rows of ldw = df32_ld(K)),
// n = 0..n_prev, tiles of 64 rows x 64 steps of all subdomains numbered in
// one sequence and strided over the grid (balanced whatever the subdomain
// count); each thread 4 rows x 4 steps, inner chunks of 16 columns staged in
// shared memory (rows padded by two pairs), 32-byte stores of 4 consecutive rows.
#define RW_T 64
#define RW_C 16
#define RW_P (RW_T + 2)
#define RW_MAXSUB 160
__global__ void __launch_bounds__(RB_THREADS) k_robin_w(SwrDeviceView v, const int* win_prev) {
    __shared__ __align__(16) float2 As[RW_C][RW_P];
    __shared__ __align__(16) float2 Bs[RW_C][RW_P];
    __shared__ int first[RW_MAXSUB + 1];  // first global tile of each subdomain
    if (threadIdx.x == 0) {
        int t = 0;
        for (int sid = 0; sid < v.n_sub && sid < RW_MAXSUB; ++sid) {
            first[sid] = t;
            const SubDev& s = v.sub[sid];
            const int wp = win_prev[s.inst];
            if (wp > 0 && robin_cols(s) > 0) t += ((s.K + RW_T - 1) / RW_T) * ((wp + RW_T) / RW_T);
        }
        first[v.n_sub < RW_MAXSUB ? v.n_sub : RW_MAXSUB] = t;
    }
    __syncthreads();
    const int nsub = v.n_sub < RW_MAXSUB ? v.n_sub : RW_MAXSUB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // rows tx*4.., steps ty*4..
    for (int g = blockIdx.x; g < first[nsub]; g += gridDim.x) {
        int sid = 0;
        while (first[sid + 1] <= g) ++sid;
        const SubDev& s = v.sub[sid];
        const InstDev& in = v.inst[s.inst];
        const int wp = win_prev[s.inst];
        const int K = s.K, J = robin_cols(s), ldw = df32_ld(K);
        const float2* GE = reinterpret_cast<const float2*>(v.arena + s.GE);
        const float2* H = reinterpret_cast<const float2*>(v.arena + s.Hr);
        float2* W = reinterpret_cast<float2*>(v.arena + s.Wr);
        const float2 kdt = dsp_split_int(in.kappa * in.dt);
        const int tr = (K + RW_T - 1) / RW_T, tile = g - first[sid];
        const int r0 = (tile % tr) * RW_T, n0 = (tile / tr) * RW_T;
        float ah[4][4], al[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) ah[k][i] = al[k][i] = 0.f;
        for (int j0 = 0; j0 < J; j0 += RW_C) {
            __syncthreads();
            for (int e = threadIdx.x; e < RW_C * RW_T; e += RB_THREADS) {
                const int jj = e & (RW_C - 1), x = e >> 4, j = j0 + jj;  // 16 consecutive columns per row
                const int r = r0 + x, n = n0 + x;
                As[jj][x] = (j < J && r < K) ? GE[(long long)r * J + j] : make_float2(0.f, 0.f);
                Bs[jj][x] = (j < J && n <= wp) ? H[(long long)n * J + j] : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < RW_C; ++jj) {
                const float4 a01 = *reinterpret_cast<const float4*>(&As[jj][tx * 4]);
                const float4 a23 = *reinterpret_cast<const float4*>(&As[jj][tx * 4 + 2]);
                const float4 b01 = *reinterpret_cast<const float4*>(&Bs[jj][ty * 4]);
                const float4 b23 = *reinterpret_cast<const float4*>(&Bs[jj][ty * 4 + 2]);
                const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                                     make_float2(a23.z, a23.w)};
                const float2 bq[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                                      make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int i = 0; i < 4; ++i) ds_fma(ah[k][i], al[k][i], a[k], bq[i]);
            }
        }
        const int rb = r0 + tx * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = n0 + ty * 4 + i;
            if (n > wp || rb >= K) continue;
            float2 o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = dsp_mul(dsp_norm(ah[k][i], al[k][i]), kdt);
            float2* dst = W + (long long)n * ldw + rb;  // 32-byte aligned: ldw and rb are multiples of 4
            if (rb + 4 <= ldw) {
                // rows past K are padding (never read)
                *reinterpret_cast<float4*>(dst) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                *reinterpret_cast<float4*>(dst + 2) = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
            }
        }
    }
}

static inline unsigned rb_div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// GE of every subdomain (assembly, after the step-matrix inverse).
cudaError_t launch_robin_ge(const SwrDeviceView& v, cudaStream_t st, int max_K, int max_J) {
    k_robin_ge<<<dim3(rb_div_up((long long)max_K * max_J, RB_THREADS), v.n_sub), RB_THREADS, 0, st>>>(v);
    return cudaGetLastError();
}

// H and W of every subdomain for the coming window (before it is launched);
// the grids do not depend on the window lengths, which the kernels read on
// the device (a captured iteration replays them unchanged).
cudaError_t launch_robin_w(const SwrDeviceView& v, cudaStream_t st, const int* d_win_prev, int max_K, int nsm) {
    const size_t sm = (size_t)max_K * sizeof(double);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_robin_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int per = (2 * nsm + v.n_sub - 1) / v.n_sub;
    k_robin_h<<<dim3(per > 0 ? per : 1, v.n_sub), RB_THREADS, sm, st>>>(v, d_win_prev);
    k_robin_w<<<4 * nsm, RB_THREADS, 0, st>>>(v, d_win_prev);
    return cudaGetLastError();
}

// Columns of GE for the arena layout.
int robin_columns(const SubDev& s) { return robin_cols(s); }

}  // namespace swr
