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
// gauge-fixed decomposition above, in double-single on the FP32 pipes (this
// part's FP64 unit would make it as long as the product that follows).  One
// warp per step, steps strided over the warps of the grid; the per-subdomain
// constants (edge vectors, inverse Gram matrices) are staged once per CTA.
// Dynamic shared memory: per warp the step's b' as a kd x kd matrix with
// column stride kd + 1 (conflict-free column walks).
#define RH_MAXKD 64
__global__ void k_robin_h(SwrDeviceView v, const int* win_prev) {
    const SubDev& s = v.sub[blockIdx.y];
    const int wp = win_prev[s.inst];
    const int K = s.K, kd = s.kd, J = robin_cols(s);
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wp <= 0 || J == 0 || (int)blockIdx.x * nw > wp) return;
    int blk[4];
    robin_slots(s, blk);
    __shared__ float2 U2[2][RH_MAXKD], V2[2][RH_MAXKD];
    __shared__ float2 GUi2[4], GVi2[4];
    __shared__ int slU[2], slV[2], p, q;
    __shared__ float2 Ysw[8][RH_MAXKD][2], Qsw[8][2][RH_MAXKD], UYw[8][4];
    extern __shared__ float2 Bw[];  // [nw][kd (kd + 1)] (two electrons)
    if (threadIdx.x == 0) {
        const double* U[2] = {nullptr, nullptr};
        const double* V[2] = {nullptr, nullptr};
        int pp = 0, qq = 0;
        for (int sl = 0; sl < 4; ++sl) {
            if (blk[sl] < 0) continue;
            if (sl < 2) {
                slU[pp] = sl;
                U[pp++] = robin_edge(v, s, sl);
            } else {
                slV[qq] = sl;
                V[qq++] = robin_edge(v, s, sl);
            }
        }
        double gu[4] = {0, 0, 0, 0}, gv[4] = {0, 0, 0, 0};
        gram_inverse(U, pp, kd, gu);
        gram_inverse(V, qq, kd, gv);
        for (int i = 0; i < 4; ++i) {
            GUi2[i] = dsp_split_int(gu[i]);
            GVi2[i] = dsp_split_int(gv[i]);
        }
        p = pp;
        q = qq;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * kd; e += blockDim.x) {
        const int i = e / kd, a = e - i * kd;
        if (i < p) U2[i][a] = dsp_split_int(robin_edge(v, s, slU[i])[a]);
        if (i < q) V2[i][a] = dsp_split_int(robin_edge(v, s, slV[i])[a]);
    }
    __syncthreads();
    const int ldb = kd + 1;
    float2* Bm = Bw + (size_t)warp * kd * ldb;
    float2 (*Ys)[2] = Ysw[warp];
    float2 (*Qs)[RH_MAXKD] = Qsw[warp];
    float2* UY = UYw[warp];
    float2* H = reinterpret_cast<float2*>(v.arena + s.Hr);
    for (int n = blockIdx.x * nw + warp; n <= wp; n += gridDim.x * nw) {
        const double* b = v.arena + s.bvec + (long long)n * K;
        float2* h = H + (long long)n * J;
        if (s.N == 1) {
            // h = (U^T U)^{-1} U^T b'
            float2 t[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            for (int i = 0; i < p; ++i) {
                float th = 0.f, tl = 0.f;
                for (int a = lane; a < kd; a += 32) ds_fma(th, tl, U2[i][a], dsp_split_int(b[a]));
                float2 acc = dsp_norm(th, tl);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc = dsp_shfl_add(acc, o);
                t[i] = acc;
            }
            if (lane < p) {
                float2 x = make_float2(0.f, 0.f);
                for (int k = 0; k < p; ++k) x = dsp_add(x, dsp_mul(GUi2[lane * p + k], t[k]));
                h[blk[slU[lane]]] = x;
            }
            continue;
        }
        for (int e = lane; e < K; e += 32) {
            const int bb = e / kd, a = e - bb * kd;
            Bm[a + ldb * bb] = dsp_split_int(b[e]);
        }
        __syncwarp();
        // (B V)[a][t] and Q = U^T B
        for (int it = lane; it < kd * q; it += 32) {
            const int a = it / q, t = it - a * q;
            float hh = 0.f, ll = 0.f;
            for (int bb = 0; bb < kd; ++bb) ds_fma(hh, ll, Bm[a + ldb * bb], V2[t][bb]);
            Ys[a][t] = dsp_norm(hh, ll);
        }
        for (int it = lane; it < kd * p; it += 32) {
            const int t = it / kd, bb = it - t * kd;
            float hh = 0.f, ll = 0.f;
            for (int a = 0; a < kd; ++a) ds_fma(hh, ll, U2[t][a], Bm[a + ldb * bb]);
            Qs[t][bb] = dsp_norm(hh, ll);
        }
        __syncwarp();
        // Y = (B V) (V^T V)^{-1}: every lane its own rows a
        for (int a = lane; a < kd; a += 32) {
            float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            for (int si = 0; si < q; ++si)
                for (int t = 0; t < q; ++t) y[si] = dsp_add(y[si], dsp_mul(Ys[a][t], GVi2[t * q + si]));
            for (int si = 0; si < q; ++si) Ys[a][si] = y[si];
        }
        __syncwarp();
        // U^T Y (p x q)
        if (lane < p * q) {
            const int t = lane / q, u = lane - t * q;
            float hh = 0.f, ll = 0.f;
            for (int a = 0; a < kd; ++a) ds_fma(hh, ll, U2[t][a], Ys[a][u]);
            UY[t * 2 + u] = dsp_norm(hh, ll);
        }
        __syncwarp();
        // h: X^T = (U^T U)^{-1} (U^T B - (U^T Y) V^T) for coordinate-0 slots, Y for coordinate 1
        for (int it = lane; it < kd * (p + q); it += 32) {
            const int si = it / kd, m = it - si * kd;
            float2 x;
            int sl;
            if (si < p) {
                x = make_float2(0.f, 0.f);
                for (int t = 0; t < p; ++t) {
                    float rh = Qs[t][m].x, rl = Qs[t][m].y;
                    for (int u = 0; u < q; ++u) ds_fma(rh, rl, dsp_neg(UY[t * 2 + u]), V2[u][m]);
                    x = dsp_add(x, dsp_mul(GUi2[si * p + t], dsp_norm(rh, rl)));
                }
                sl = slU[si];
            } else {
                x = Ys[m][si - p];
                sl = slV[si - p];
            }
            h[blk[sl] * kd + m] = x;
        }
        __syncwarp();
    }
}

// W[n][r] = kappa dt sum_j GE[r][j] H[n][j] (pairs, rows of ldw = df32_ld(K)),
// n = 0..n_prev, tiles of 64 rows x 64 steps of all subdomains numbered in
// one sequence (tiles[sid] the first tile of subdomain sid, tiles[n_sub] the
// total, from k_robin_tiles) and strided over the grid, balanced whatever the
// subdomain count; each thread 4 rows x 4 steps, inner chunks of 16 columns
// staged in shared memory (rows padded by two pairs), 32-byte stores of 4
// consecutive rows.
#define RW_T 64
#define RW_C 16
#define RW_P (RW_T + 2)
__global__ void __launch_bounds__(RB_THREADS) k_robin_w(SwrDeviceView v, const int* win_prev, const int* tiles) {
    __shared__ __align__(16) float2 As[RW_C][RW_P];
    __shared__ __align__(16) float2 Bs[RW_C][RW_P];
    const int total = tiles[v.n_sub];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // rows tx*4.., steps ty*4..
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        int lo = 0, hi = v.n_sub;  // the subdomain: tiles[sid] <= g < tiles[sid + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tiles[mid] <= g) lo = mid;
            else hi = mid;
        }
        const int sid = lo;
        const SubDev& s = v.sub[sid];
        const InstDev& in = v.inst[s.inst];
        const int wp = win_prev[s.inst];
        const int K = s.K, J = robin_cols(s), ldw = df32_ld(K);
        const float2* GE = reinterpret_cast<const float2*>(v.arena + s.GE);
        const float2* H = reinterpret_cast<const float2*>(v.arena + s.Hr);
        float2* W = reinterpret_cast<float2*>(v.arena + s.Wr);
        const float2 kdt = dsp_split_int(in.kappa * in.dt);
        const int tr = (K + RW_T - 1) / RW_T, tile = g - tiles[sid];
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

// tiles[sid] = the first tile of subdomain sid in the product's sequence
// (64 x 64 tiles of K rows by n_prev + 1 steps; subdomains without an
// interior edge get their zeros the same way), tiles[n_sub] = the total: an
// exclusive scan by one CTA over contiguous runs of subdomains.
__global__ void k_robin_tiles(SwrDeviceView v, const int* win_prev, int* tiles) {
    __shared__ int part[1024];
    const int ns = v.n_sub, per = (ns + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(ns, s0 + per);
    int sum = 0;
    for (int sid = s0; sid < s1; ++sid) {
        const SubDev& s = v.sub[sid];
        const int wp = win_prev[s.inst];
        if (wp > 0) sum += ((s.K + RW_T - 1) / RW_T) * ((wp + RW_T) / RW_T);
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int x = part[t];
            part[t] = acc;
            acc += x;
        }
        tiles[ns] = acc;
    }
    __syncthreads();
    int acc = part[threadIdx.x];
    for (int sid = s0; sid < s1; ++sid) {
        tiles[sid] = acc;
        const SubDev& s = v.sub[sid];
        const int wp = win_prev[s.inst];
        if (wp > 0) acc += ((s.K + RW_T - 1) / RW_T) * ((wp + RW_T) / RW_T);
    }
}

static inline unsigned rb_div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// GE of every subdomain (assembly, after the step-matrix inverse).
// Also raises the dynamic shared-memory cap of k_robin_h to the most its
// launches ask for (160 KB beside its static arrays), here at assembly and not
// inside a captured iteration.
cudaError_t launch_robin_ge(const SwrDeviceView& v, cudaStream_t st, int max_K, int max_J) {
    cudaError_t e = cudaFuncSetAttribute(k_robin_h, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    if (max_J > 0) k_robin_ge<<<dim3(rb_div_up((long long)max_K * max_J, RB_THREADS), v.n_sub), RB_THREADS, 0, st>>>(v);
    return cudaGetLastError();
}

// H and W of every subdomain for the coming window (before it is launched);
// the grids do not depend on the window lengths, which the kernels read on
// the device (a captured iteration replays them unchanged).  kd2: the largest
// kd of the two-electron subdomains (0 when there are none).
cudaError_t launch_robin_w(const SwrDeviceView& v, cudaStream_t st, const int* d_win_prev, int kd2, int nsm,
                           int* d_tiles) {
    int nw = 8;
    size_t sm = 0;
    if (kd2 > 0) {
        const size_t per_warp = (size_t)kd2 * (kd2 + 1) * sizeof(float2);
        while (nw > 1 && nw * per_warp > 160 * 1024) --nw;
        sm = nw * per_warp;
    }
    const int per = (2 * nsm + v.n_sub - 1) / v.n_sub;
    k_robin_h<<<dim3(per > 0 ? per : 1, v.n_sub), 32 * nw, sm, st>>>(v, d_win_prev);
    k_robin_tiles<<<1, 1024, 0, st>>>(v, d_win_prev, d_tiles);
    k_robin_w<<<4 * nsm, RB_THREADS, 0, st>>>(v, d_win_prev, d_tiles);
    return cudaGetLastError();
}

// Columns of GE for the arena layout.
int robin_columns(const SubDev& s) { return robin_cols(s); }

}  // namespace swr
