// swr_window.cu -- the time window of one Schwarz iteration (imaginary time).
//
// Sec. 5.2 (system SIT) and Sec. 5.4 steps 2 and 4 of the paper: on every
// subdomain, implicit Euler in the orthonormal local basis,
//     y^{n+1} = G (y^n / s_n + kappa dt b'^{n+1}),   G = (I + dt H')^{-1},
// where y^n is the iterate before the normalisation of t_n and
//     s_n^2 = sum_i y_i^n . (Pp (x) Pp) y_i^n      (partition-of-unity norm)
// is the global normalisation; the inner stop is ||c^{n+1} - c^n|| <= tol with
// c^n = y^n / s_n (Sec. 5.2).
//
// One persistent cooperative launch runs the whole window.  A task is a block
// of rows of one subdomain's G, sized so that every SM gets the same number of
// rows; a CTA keeps its tasks' constants, their own rows of y^n, y^{n-1}, z^n,
// z^{n-1}, the Kronecker factors Pp and (mixed precision) its rows of G_hi in
// shared memory for the whole window.  Per step:
//   phase A(n+1): y^{n+1} rows = G v, v = y^n/s_n + kappa dt b'^{n+1}, and the
//                 partial of delta_n^2 from the CTA's own rows;
//   reduce-barrier: the last CTA to arrive sums the delta partials per
//                 instance (fixed order) and releases the grid;
//   phase B(n+1): stop decisions, z^{n+1} rows = (Pp (x) Pp) y^{n+1}, partial
//                 of s_{n+1}^2;
//   reduce-barrier: the same for the s^2 partials.
// Every wait is bounded; on timeout the kernel raises SWR_ERR_TIMEOUT and
// returns.
//
// Precision: FP64 (DFMA), or double-single (SWR_PREC_MIXED): G = G_hi + G_lo
// in FP32 pairs, v = v_hi + v_lo; products run on the FP32 pipes with
// error-free TwoProduct/TwoSum accumulation into a (hi, lo) pair, which keeps
// the FP64 accuracy of the step (~1e-14) on units with 64x the FP64 rate.
#include <limits.h>
#include <math.h>

#include "swr_internal.cuh"

namespace swr {

#define WIN_THREADS 256
#define WIN_TPC 4    // tasks per CTA kept in shared memory
#define WIN_RB 64    // rows per task

__device__ inline unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ inline double wblock_sum(double x, double* red) {
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < WIN_THREADS / 32; ++i) t += red[i];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Grid barrier fused with a per-instance reduction.  Every CTA has written its
// partials to part[]; the CTA whose arrival completes the count sums them per
// instance in task order into sums[], then publishes 2*gen + go on the release
// word, go = 0 when `nact` (if given) shows that no instance is still stepping.
// With scal_out it also stores s = sqrt(sum) (1 without normalisation) and 1/s
// per instance: scal_out[i], scal_out[n_inst + i].
// Bounded waits; returns false on error, *go_out receives go.
__device__ bool reduce_barrier(unsigned* count, unsigned* release, unsigned target, unsigned gen, bool reduce,
                               const double* part, const int* inst_task0, int n_inst, double* sums, int* err,
                               long long limit, double* red, const int* nact, int* go_out,
                               const InstDev* inst = nullptr, double* scal_out = nullptr) {
    __shared__ int s_last, s_ok, s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned old = atomicAdd(count, 1u);
        s_last = (old == target - 1);
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (reduce) {
            if (n_inst < 8) {
                for (int i = 0; i < n_inst; ++i) {
                    double x = 0;
                    for (int u = inst_task0[i] + threadIdx.x; u < inst_task0[i + 1]; u += WIN_THREADS)
                        x += __ldcg(part + u);
                    x = wblock_sum(x, red);
                    if (threadIdx.x == 0) sums[i] = x;
                }
            } else {
                // one warp per instance: lanes stride over its tasks, fixed-order shuffle sum
                const int lane = threadIdx.x & 31;
                for (int i = threadIdx.x >> 5; i < n_inst; i += WIN_THREADS / 32) {
                    double x = 0;
#pragma unroll 4
                    for (int u = inst_task0[i] + lane; u < inst_task0[i + 1]; u += 32) x += __ldcg(part + u);
                    x = warp_sum(x);
                    if (lane == 0) sums[i] = x;
                }
            }
        }
        if (scal_out) {
            // s_n = sqrt(s_n^2) and 1/s_n once per instance (FP64 square root and
            // division are slow sequences: here instead of in every task)
            __syncthreads();
            for (int i = threadIdx.x; i < n_inst; i += WIN_THREADS) {
                const double sn = inst[i].normalize ? sqrt(sums[i]) : 1.0;
                scal_out[i] = sn;
                scal_out[n_inst + i] = 1.0 / sn;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int go = nact ? (__ldcg(nact) > 0) : 1;
            s_go = go;
            __threadfence();
            st_release_u32(release, 2u * gen + (unsigned)go);
        }
    } else if (threadIdx.x == 0) {
        long long it = 0;
        unsigned w = 0;
        while ((w = ld_acquire_u32(release)) < 2u * gen) {
            if (++it > limit) { atomicOr(err, SWR_ERR_TIMEOUT); s_ok = 0; break; }
            if ((it & 255) == 0 && *(volatile int*)err) { s_ok = 0; break; }
            __nanosleep(20);
        }
        s_go = (int)(w & 1u);
        __threadfence();
    }
    __syncthreads();
    *go_out = s_go;
    return s_ok != 0 && *(volatile int*)err == 0;
}

// Grid barrier without reduction: the CTA whose arrival completes the count
// publishes 2*gen + go at once (go = 0 when `nact` shows no instance still
// stepping); every CTA then sums the partials it needs itself (block_sums2).
// Bounded waits; returns false on error.
__device__ bool release_barrier(unsigned* count, unsigned* release, unsigned target, unsigned gen, int* err,
                                long long limit, const int* nact, int* go_out) {
    __shared__ int s_ok, s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        __threadfence();
        const unsigned old = atomicAdd(count, 1u);
        if (old == target - 1) {
            const int go = nact ? (__ldcg(nact) > 0) : 1;
            s_go = go;
            __threadfence();
            st_release_u32(release, 2u * gen + (unsigned)go);
        } else {
            long long it = 0;
            unsigned w = 0;
            while ((w = ld_acquire_u32(release)) < 2u * gen) {
                if (++it > limit) { atomicOr(err, SWR_ERR_TIMEOUT); s_ok = 0; break; }
                if ((it & 255) == 0 && *(volatile int*)err) { s_ok = 0; break; }
                __nanosleep(20);
            }
            s_go = (int)(w & 1u);
        }
        __threadfence();
    }
    __syncthreads();
    *go_out = s_go;
    return s_ok != 0 && *(volatile int*)err == 0;
}

// sa = sum of part_a[t0, t1), sb = sum of part_b[t0, t1): strided per thread,
// warp tree, warps in order -- the same order in every CTA, so every CTA gets
// the same bits.
__device__ void block_sums2(const double* part_a, const double* part_b, int t0, int t1, double* red, double* sa,
                            double* sb) {
    double xa = 0, xb = 0;
    for (int u = t0 + threadIdx.x; u < t1; u += WIN_THREADS) {
        xa += __ldcg(part_a + u);
        xb += __ldcg(part_b + u);
    }
    xa = warp_sum(xa);
    xb = warp_sum(xb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[w] = xa;
        red[16 + w] = xb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0;
        for (int i = 0; i < WIN_THREADS / 32; ++i) {
            ta += red[i];
            tb += red[16 + i];
        }
        *sa = ta;
        *sb = tb;
    }
    __syncthreads();
}

__device__ inline void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Antisymmetric states (Appendix A): the mirror subdomain (i2, i1) of the
// task's subdomain (i1, i2), and the index of coefficient (a, b) -> (b, a)
// (index a + kd b: the orthonormal per-coordinate functions of an interval
// are the same in both coordinates, dropped directions kept as zero columns).
__device__ inline int mirror_sid(const SwrDeviceView& v, const TaskCache& tc) {
    const InstDev& in = v.inst[tc.inst];
    const int s = tc.sid - in.sub_base;
    return in.sub_base + s / in.L + in.L * (s % in.L);
}
__device__ inline int swap_index(int c, int kd) { return c / kd + kd * (c % kd); }
// The lower subdomain of a mirror pair has no tasks (its iterates are the
// mirror images of the upper one's): the partials of an off-diagonal task of
// an antisymmetric instance count twice in the instance's sums; the
// projection onto the antisymmetric part is then needed on the diagonal only.
__device__ inline double mirror_weight(const SwrDeviceView& v, const TaskCache& tc) {
    return (v.inst[tc.inst].anti && mirror_sid(v, tc) != tc.sid) ? 2.0 : 1.0;
}
__device__ inline bool diagonal_anti(const SwrDeviceView& v, const TaskCache& tc) {
    return v.inst[tc.inst].anti && mirror_sid(v, tc) == tc.sid;
}

// rows [r0, r0+nr) of z = (P1 (x) P2) y (N = 2) or P1 y (N = 1); y in shared
// memory, P in shared or global memory.  Warp-parallel dot products (lanes over
// the contraction, shuffle reduction) keep the FP64 dependency chains short.
__device__ void z_rows_sm(const TaskCache& tc, const double* P1, const double* P2, const double* ys, double* z,
                          double* tmp) {
    const int kd = tc.kd, r0 = tc.r0, r1 = tc.r0 + tc.nr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = WIN_THREADS / 32;
    if (tc.N == 1) {
        for (int r = r0 + warp; r < r1; r += nw) {
            double acc = 0;
            for (int c = lane; c < kd; c += 32) acc += P1[r * kd + c] * ys[c];
            acc = warp_sum(acc);
            if (lane == 0) z[r - r0] = acc;
        }
        __syncthreads();
        return;
    }
    const int b0 = r0 / kd, b1 = (r1 - 1) / kd, nb = b1 - b0 + 1;
    // tmp[bb][c] = sum_e Y[c][e] P2[b0+bb][e]   (kd <= 32: one lane per e)
    for (int item = warp; item < nb * kd; item += nw) {
        const int bb = item / kd, c = item % kd;
        double x = (lane < kd) ? ys[c + kd * lane] * P2[(b0 + bb) * kd + lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) tmp[bb * kd + c] = x;
    }
    __syncthreads();
    for (int r = r0 + warp; r < r1; r += nw) {
        const int b = r / kd, a = r - b * kd;
        double x = (lane < kd) ? P1[a * kd + lane] * tmp[(b - b0) * kd + lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) z[r - r0] = x;
    }
    __syncthreads();
}

// Rows [r0, r0+nr) of z = (P1 (x) P2) y (N = 2) or P1 y (N = 1), y in shared
// memory, for a task whose factors are in global memory: the factors are
// first staged in shared memory (Ps: 2 kd^2 doubles, one coalesced pass), then
// every thread computes whole outputs of the two small products
//   tmp[bb][c] = sum_e Y[c][e] P2[b0+bb][e],   z[(a,b)] = sum_c P1[a][c] tmp[b-b0][c]
// (no per-output warp reductions waiting on separate loads).
__device__ void z_rows_staged(const TaskCache& tc, const double* P1g, const double* P2g, const double* ys, double* z,
                              double* tmp, double* Ps) {
    const int kd = tc.kd, r0 = tc.r0, r1 = tc.r0 + tc.nr, kk = kd * kd;
    double* P1 = Ps;
    double* P2 = Ps + kk;
    for (int e = threadIdx.x; e < kk; e += WIN_THREADS) {
        P1[e] = P1g[e];
        if (tc.N == 2) P2[e] = P2g[e];
    }
    __syncthreads();
    if (tc.N == 1) {
        for (int r = r0 + threadIdx.x; r < r1; r += WIN_THREADS) {
            double acc = 0;
            for (int c = 0; c < kd; ++c) acc = fma(P1[r * kd + c], ys[c], acc);
            z[r - r0] = acc;
        }
        __syncthreads();
        return;
    }
    const int b0 = r0 / kd, b1 = (r1 - 1) / kd, nb = b1 - b0 + 1;
    for (int item = threadIdx.x; item < nb * kd; item += WIN_THREADS) {
        const int bb = item / kd, c = item - bb * kd;
        const double* p2 = P2 + (b0 + bb) * kd;
        double acc = 0;
        for (int e = 0; e < kd; ++e) acc = fma(ys[c + kd * e], p2[e], acc);
        tmp[item] = acc;
    }
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < r1; r += WIN_THREADS) {
        const int b = r / kd, a = r - b * kd;
        const double* p1 = P1 + a * kd;
        const double* tb = tmp + (b - b0) * kd;
        double acc = 0;
        for (int c = 0; c < kd; ++c) acc = fma(p1[c], tb[c], acc);
        z[r - r0] = acc;
    }
    __syncthreads();
}

// Bulk prefetch of [p, p + bytes) into L2 by the copy engine (no registers, no
// shared memory): the range is widened to 16-byte boundaries (it stays inside
// the workspace, whose matrices are followed by other arena data) and issued
// in pieces of at most 64 KB.
__device__ inline void prefetch_l2(const void* p, size_t bytes) {
    const unsigned long long g = (unsigned long long)__cvta_generic_to_global(p);
    unsigned long long a = g & ~15ULL;
    const unsigned long long e = (g + bytes + 15ULL) & ~15ULL;
    while (a < e) {
        const unsigned n = (unsigned)((e - a) < 65536ULL ? (e - a) : 65536ULL);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
        a += n;
    }
}

// Lane 0 prefetches rows [rb, rb + nrow) of the task's step matrix (both FP32
// planes, or the FP64 rows).
template <bool DF32>
__device__ inline void prefetch_rows(const SwrDeviceView& v, const TaskCache& tc, int rb, int nrow) {
    if (nrow <= 0) return;
    if (DF32) {
        const long long ld = df32_ld(tc.K);
        const float* Gh = (const float*)(v.arena + tc.Gf);
        prefetch_l2(Gh + rb * ld, (size_t)nrow * ld * sizeof(float));
        prefetch_l2(Gh + (long long)tc.K * ld + rb * ld, (size_t)nrow * ld * sizeof(float));
    } else {
        prefetch_l2(v.arena + tc.Gm + (long long)rb * tc.K, (size_t)nrow * tc.K * sizeof(double));
    }
}

// One double-single multiply-add: (yh, yl) += (g0 + g1)(x0 + x1), TwoProduct of
// the leading terms, TwoSum into (yh, yl), the cross terms into yl.
__device__ inline void df32_acc(float& yh, float& yl, float g0, float g1, float x0, float x1) {
    const float p = g0 * x0, e = fmaf(g0, x0, -p);
    float sh, q;
    two_sum(yh, p, sh, q);
    yh = sh;
    yl += (q + e) + fmaf(g0, x1, g1 * x0);
}

// Rows [rb, rb + nrow), nrow <= 4, of G v in double-single: one warp, lanes
// over groups of 4 columns (16-byte loads from each FP32 plane, rows of ld
// columns zero-padded), independent (hi, lo) accumulators per row so that the
// loads of four rows are in flight together; y[i] to lane 0.
__device__ inline void df32_rows4(const float* Gh, const float* Gl, int ld, const float2* vf, int rb, int nrow,
                                  int lane, double* y) {
    float yh[4] = {0.f, 0.f, 0.f, 0.f}, yl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = lane * 4; c < ld; c += 128) {
        const float4 xa = *reinterpret_cast<const float4*>(vf + c);      // h0 l0 h1 l1
        const float4 xb = *reinterpret_cast<const float4*>(vf + c + 2);  // h2 l2 h3 l3
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < nrow) {
                const long long o = (long long)(rb + i) * ld + c;
                const float4 gh = *reinterpret_cast<const float4*>(Gh + o);
                const float4 gl = *reinterpret_cast<const float4*>(Gl + o);
                df32_acc(yh[i], yl[i], gh.x, gl.x, xa.x, xa.y);
                df32_acc(yh[i], yl[i], gh.y, gl.y, xa.z, xa.w);
                df32_acc(yh[i], yl[i], gh.z, gl.z, xb.x, xb.y);
                df32_acc(yh[i], yl[i], gh.w, gl.w, xb.z, xb.w);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float sh, eh;
            const float oh = __shfl_xor_sync(0xffffffffu, yh[i], o), ol = __shfl_xor_sync(0xffffffffu, yl[i], o);
            two_sum(yh[i], oh, sh, eh);
            yh[i] = sh;
            yl[i] = yl[i] + ol + eh;
        }
        y[i] = (double)yh[i] + (double)yl[i];
    }
}

// Rows [rb, rb + nrow), nrow <= 4, of G v in FP64: per row two accumulators
// over columns c = lane + 64 m and c = lane + 32 + 64 m, then a shuffle sum
// (the same order for every row whatever warp computes it); y[i] to all lanes.
__device__ inline void fp64_rows4(const double* G, int K, const double* vs, int rb, int nrow, int lane, double* y) {
    double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
    int c = lane;
    for (; c + 32 < K; c += 64) {
        const double x0 = vs[c], x1 = vs[c + 32];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < nrow) {
                const double* g = G + (long long)(rb + i) * K;
                a[i] = fma(g[c], x0, a[i]);
                b[i] = fma(g[c + 32], x1, b[i]);
            }
        }
    }
    if (c < K) {
        const double x0 = vs[c];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < nrow) a[i] = fma(G[(long long)(rb + i) * K + c], x0, a[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] = warp_sum(a[i] + b[i]);
}

// Two-phase window: two reduce-barriers per step (see the top of the file).
// DF32 = false: G in FP64 (DFMA).  DF32 = true: G as FP32 hi/lo planes
// (8 bytes per element like FP64, on the FP32 pipes).  Per-task state sits in
// shared memory when the CTA has at most WIN_TPC tasks, else (A.many) in
// global memory.  Dynamic shared memory (doubles):
//   vs[kmax] | vf[kmax] (float2) | tmp[rows_max + 2 kdmax] | P[tasks_per_cta][2][kdmax^2]
// (many: P[1][2][kdmax^2], the factors of the task at hand)
template <bool DF32>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window_2ph(SweepArgs A) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ TaskCache s_tcs[WIN_TPC];
    __shared__ double s_own[WIN_TPC][4][WIN_RB];
    __shared__ int s_alive[WIN_TPC];
    int go = 1;
    const SwrDeviceView& v = A.v;
    const int t_begin = A.cta_task0[blockIdx.x];
    const int ntk = A.cta_task0[blockIdx.x + 1] - t_begin;
    const bool many = A.many != 0;
    TaskCache* tcs = many ? A.g_tc + t_begin : s_tcs;
    int* alive = many ? A.g_alive + t_begin : s_alive;
    const int cap = A.cap;
    const int kmax = df32_ld(A.kmax), kdmax = A.kdmax;
    double* vs = sm;
    float2* vf = (float2*)(sm + kmax);
    double* tmp = sm + 2 * kmax;
    double* Psm = tmp + A.rows_max + 2 * kdmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = WIN_THREADS / 32;
    unsigned target = 0, gen = 0;
    // own rows: slots 0,1 = y^n ring, 2,3 = z^n ring
    auto own = [&](int j, int slot) -> double* {
        return many ? A.g_own + tcs[j].own + (long long)slot * tcs[j].nr : &s_own[j][slot][0];
    };
    auto pmat = [&](int j, int which) -> const double* {
        return many ? v.arena + (which ? tcs[j].p2 : tcs[j].p1)
                    : Psm + (long long)j * 2 * kdmax * kdmax + (which ? (long long)kdmax * kdmax : 0);
    };
    // z rows: factors resident in shared memory (few tasks), else staged per task into Psm
    auto z_rows = [&](int j, const TaskCache& tc, double* z) {
        if (many) z_rows_staged(tc, v.arena + tc.p1, v.arena + tc.p2, vs, z, tmp, Psm);
        else z_rows_sm(tc, pmat(j, 0), pmat(j, 1), vs, z, tmp);
    };

    // ------------------------------------------------------- set-up + step 0
    for (int j = 0; j < ntk; ++j) {
        const int t = A.cta_list[t_begin + j];
        if (tid == 0) {
            tcs[j] = make_task_cache(A, t);
            alive[j] = 1;
        }
        __syncthreads();
        const TaskCache tc = tcs[j];
        const int kd = tc.kd, K = tc.K, nr = tc.nr;
        if (!many) {
            double* P1 = Psm + (long long)j * 2 * kdmax * kdmax;
            double* P2 = P1 + (long long)kdmax * kdmax;
            const double* P1g = v.arena + tc.p1;
            const double* P2g = v.arena + tc.p2;
            for (int e = tid; e < kd * kd; e += WIN_THREADS) {
                P1[e] = P1g[e];
                P2[e] = P2g[e];
            }
        }
        const double* c0 = v.arena + tc.c0;
        for (int c = tid; c < K; c += WIN_THREADS) vs[c] = c0[c];
        __syncthreads();
        double* h0 = v.arena + tc.hist;
        double* y0 = own(j, 0);
        for (int r = tid; r < nr; r += WIN_THREADS) {
            h0[tc.r0 + r] = vs[tc.r0 + r];
            y0[r] = vs[tc.r0 + r];  // y^0 in slot 0
        }
        z_rows(j, tc, own(j, 2));  // z^0 in slot 2
        double acc = 0;
        const double* z0 = own(j, 2);
        for (int r = tid; r < nr; r += WIN_THREADS) acc += y0[r] * z0[r];
        acc = wblock_sum(acc, red);
        if (tid == 0) A.part_s[t] = acc * mirror_weight(v, tc);
    }
    target += gridDim.x;
    ++gen;
    if (!reduce_barrier(&A.bar->count, &A.bar->gen, target, gen, true, A.part_s, A.inst_task0, v.n_inst,
                        A.sums_s, v.err, A.spin_limit, red, nullptr, &go, v.inst, A.scal_inst))
        return;

    for (int n = 0;; ++n) {
        // s_n, 1/s_n, 1/s_{n-1} per instance, by step parity
        const double* sc_n = A.scal_inst + (n & 1) * 2 * v.n_inst;
        const double* sc_p = A.scal_inst + ((n & 1) ^ 1) * 2 * v.n_inst;
        // ------------------------------------------------------ phase A(n+1)
        int vs_sid = -1;  // subdomain whose v is in vs / vf (consecutive tasks of one subdomain share it)
        for (int j = 0; j < ntk; ++j) {
            __syncthreads();
            if (!alive[j]) continue;
            const TaskCache tc = tcs[j];
            const int K = tc.K, nr = tc.nr;
            const int t = A.cta_list[t_begin + j];
            const bool load = (tc.sid != vs_sid);
            // the warp's first block of rows travels to L2 while v and the partials are formed
            if (many && lane == 0 && n < tc.maxs)
                prefetch_rows<DF32>(v, tc, tc.r0 + 4 * warp, min(4, tc.r0 + nr - (tc.r0 + 4 * warp)));
            // one round trip: s_n, y^n, b'^{n+1}
            const double s_n = __ldcg(sc_n + tc.inst), is_n = __ldcg(sc_n + v.n_inst + tc.inst);
            const double is_p = n == 0 ? 1.0 : __ldcg(sc_p + v.n_inst + tc.inst);
            double yv[4], bv[4];
            if (load) {
                const double* yn = v.arena + tc.hist + (long long)n * K;
                const int wp = A.win_prev[tc.inst];
                const double* bsrc = (wp > 0) ? v.arena + tc.bvec + (long long)min(n + 1, wp) * K : nullptr;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int c = tid + i * WIN_THREADS;
                    yv[i] = (c < K) ? yn[c] : 0.0;
                    bv[i] = (c < K && bsrc) ? bsrc[c] : 0.0;
                }
            }
            if (tid == 0 && tc.first) A.snorm[(long long)tc.inst * (cap + 1) + n] = s_n;
            if (n >= tc.maxs || !isfinite(s_n) || s_n <= 0.0) continue;  // closed in phase B
            if (load) {
                // antisymmetric states: v <- (v - swap(v of the mirror subdomain)) / 2 on
                // a diagonal subdomain (its own mirror)
                const bool anti = diagonal_anti(v, tc);
                const double *ynm = nullptr, *bnm = nullptr;
                if (anti) {
                    const SubDev& ms = v.sub[mirror_sid(v, tc)];
                    const int wp = A.win_prev[tc.inst];
                    ynm = v.arena + ms.hist + (long long)n * K;
                    if (wp > 0) bnm = v.arena + ms.bvec + (long long)min(n + 1, wp) * K;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int c = tid + i * WIN_THREADS;
                    if (c < K) {
                        double val = yv[i] * is_n + tc.kdt * bv[i];
                        if (anti) {
                            const int sc = swap_index(c, tc.kd);
                            val = 0.5 * (val - (__ldcg(ynm + sc) * is_n + (bnm ? tc.kdt * __ldcg(bnm + sc) : 0.0)));
                        }
                        if (DF32) {
                            float h = (float)val;
                            vf[c] = make_float2(h, (float)(val - (double)h));
                        } else {
                            vs[c] = val;
                        }
                    } else if (DF32 && c < df32_ld(K)) {
                        vf[c] = make_float2(0.f, 0.f);  // padding columns of the FP32 planes
                    }
                }
                vs_sid = tc.sid;
            }
            // partial of delta_n^2 = || y^n/s_n - y^{n-1}/s_{n-1} ||^2_chi over own rows
            if (n >= 1 && tc.ngf_stop) {
                const double* y_n = own(j, n & 1);
                const double* y_p = own(j, (n - 1) & 1);
                const double* z_n = own(j, 2 + (n & 1));
                const double* z_p = own(j, 2 + ((n - 1) & 1));
                double acc = 0;
                for (int r = tid; r < nr; r += WIN_THREADS)
                    acc += (y_n[r] * is_n - y_p[r] * is_p) * (z_n[r] * is_n - z_p[r] * is_p);
                acc = wblock_sum(acc, red);
                if (tid == 0) A.part_d[t] = acc * mirror_weight(v, tc);
            } else {
                __syncthreads();
            }
            // rows of y^{n+1} = G v
            double* ynew = v.arena + tc.hist + (long long)(n + 1) * K;
            double* yslot = own(j, (n + 1) & 1);
            // each warp takes blocks of 4 consecutive rows
            const int ld = df32_ld(K);
            const float* Gh = (const float*)(v.arena + tc.Gf);
            const float* Gl = Gh + (long long)K * ld;
            for (int rb = tc.r0 + 4 * warp; rb < tc.r0 + nr; rb += 4 * nw) {
                const int nrow = min(4, tc.r0 + nr - rb);
                if (many && lane == 0) prefetch_rows<DF32>(v, tc, rb + 4 * nw, min(4, tc.r0 + nr - (rb + 4 * nw)));
                double y[4];
                if (DF32) df32_rows4(Gh, Gl, ld, vf, rb, nrow, lane, y);
                else fp64_rows4(v.arena + tc.Gm, K, vs, rb, nrow, lane, y);
                if (lane == 0) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (i < nrow) {
                            ynew[rb + i] = y[i];
                            yslot[rb + i - tc.r0] = y[i];
                        }
                    }
                }
            }
        }
        __syncthreads();
        target += gridDim.x;
        ++gen;
        if (!reduce_barrier(&A.bar->count, &A.bar->gen, target, gen, A.any_ngf_stop && n >= 1, A.part_d,
                            A.inst_task0, v.n_inst, A.sums_d, v.err, A.spin_limit, red, nullptr, &go))
            return;
        // ------------------------------------------------------ phase B(n+1)
        vs_sid = -1;  // vs now holds y^{n+1} of subdomain vs_sid
        for (int j = 0; j < ntk; ++j) {
            __syncthreads();
            if (!alive[j]) continue;
            const TaskCache tc = tcs[j];
            const int K = tc.K, nr = tc.nr;
            const int t = A.cta_list[t_begin + j];
            const double s_n = __ldcg(sc_n + tc.inst);
            bool stop = (n >= tc.maxs) || !isfinite(s_n) || s_n <= 0.0;
            double d2 = 0;
            const double* yn1 = v.arena + tc.hist + (long long)(n + 1) * K;
            if (!stop) {
                if (n >= 1 && tc.ngf_stop) d2 = __ldcg(A.sums_d + tc.inst);
                if (tc.sid != vs_sid)
                    for (int c = tid; c < K; c += WIN_THREADS) vs[c] = yn1[c];
                if (n >= 1 && tc.ngf_stop) stop = sqrt(fmax(d2, 0.0)) <= tc.ngf_tol;
            }
            if (stop) {
                __syncthreads();
                if (tid == 0) {
                    alive[j] = 0;
                    if (tc.first) {
                        A.win[tc.inst] = n;
                        if (!isfinite(s_n) || s_n <= 0.0) atomicOr(v.err, SWR_ERR_NUMERIC);
                        __threadfence();
                        atomicSub(A.n_active, 1);
                    }
                }
                continue;
            }
            vs_sid = tc.sid;
            __syncthreads();
            double* zslot = own(j, 2 + ((n + 1) & 1));
            z_rows(j, tc, zslot);
            const double* yslot = own(j, (n + 1) & 1);
            double acc = 0;
            for (int r = tid; r < nr; r += WIN_THREADS) acc += yslot[r] * zslot[r];
            acc = wblock_sum(acc, red);
            if (tid == 0) A.part_s[t] = acc * mirror_weight(v, tc);
        }
        __syncthreads();
        target += gridDim.x;
        ++gen;
        // the last CTA to arrive reads the active count after every decrement of
        // this phase and hands the verdict to all CTAs with the release
        if (!reduce_barrier(&A.bar->count, &A.bar->gen, target, gen, true, A.part_s, A.inst_task0, v.n_inst,
                            A.sums_s, v.err, A.spin_limit, red, A.n_active, &go, v.inst,
                            A.scal_inst + ((n + 1) & 1) * 2 * v.n_inst))
            return;
        if (!go) return;
    }
}

// ---------------------------------------------------- double-single window
//
// Mixed precision, ONE reduce-barrier per step.  z^{n+1} = (Pp (x) Pp) y^{n+1}
// is obtained as W v with W = (Pp (x) Pp) G precomputed at assembly, so the
// CTA that computes its rows of y^{n+1} = G v also has its rows of z^{n+1}
// and the partial of s_{n+1}^2 without waiting for the full y^{n+1}.  Phase
// P(n): decisions from the sums reduced at the last barrier (s_n^2 and
// D_{n-1} = ||c^{n-1} - c^{n-2}||^2 ... see below), v = y^n/s_n + kappa dt b',
// partial of D_n = ||c^n - c^{n-1}||^2 from the CTA's own rows, fused
// double-single pass over the rows of G and W, partial of s_{n+1}^2.  The
// barrier after P(n) reduces both partial arrays.  D_n is therefore known at
// P(n+1): when D_n <= tol^2 the window ends at n (the step n+1 already
// computed is dropped), which reproduces the stop of the plain algorithm.
// Shared-memory task state only (at most WIN_TPC tasks per CTA).
// Dynamic shared memory: vs[kmax] doubles | vf[kmax] float2 | tmp[rows_max + 2 kdmax]
// doubles | P[tasks_per_cta][2][kdmax^2] doubles | G_hi rows (floats, when resident).
// ONEP: only the hi planes of G and W are read (the FP32-rounded step matrix
// of SWR_PREC_FP32_REFINED before its switch), their lo terms taken as 0.
template <bool ONEP>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window_fused(SweepArgs A) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ TaskCache tcs[WIN_TPC];
    __shared__ double own[WIN_TPC][6][WIN_RB];  // y slots 0..2, z slots 3..5 (ring of 3)
    __shared__ double is_prev[WIN_TPC];
    __shared__ int alive[WIN_TPC];
    __shared__ double s_sc[2];
    __shared__ int s_stop;
    __shared__ double s2_sm[WIN_TPC], d2_sm[WIN_TPC];  // s^2 and D sums of each task's instance
    // partials double-buffered by barrier parity: a CTA that has passed a
    // barrier writes the next buffer while others still sum this one
    long long pofs = 0;
    int go = 1;
    const SwrDeviceView& v = A.v;
    const int t_begin = A.cta_task0[blockIdx.x];
    const int ntk = A.cta_task0[blockIdx.x + 1] - t_begin;
    const int cap = A.cap;
    const int kmax = df32_ld(A.kmax), kdmax = A.kdmax;
    double* vs = sm;
    float2* vf = (float2*)(sm + kmax);
    double* tmp = sm + 2 * kmax;
    double* Psm = tmp + A.rows_max + 2 * kdmax;
    // resident G_hi rows start on 16 bytes (16-byte vector loads)
    // (everything before it is an even number of doubles except tmp's rows_max)
    float* Gsm = (float*)(Psm + (long long)A.tasks_per_cta * 2 * kdmax * kdmax + (A.rows_max & 1));
    const bool gres = A.g_resident != 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = WIN_THREADS / 32;
    unsigned target = 0, gen = 0;

    // ------------------------------------------------------- set-up + step 0
    for (int j = 0; j < ntk; ++j) {
        const int t = A.cta_list[t_begin + j];
        if (tid == 0) {
            tcs[j] = make_task_cache(A, t);
            alive[j] = 1;
            is_prev[j] = 1.0;
        }
        __syncthreads();
        const TaskCache& tc = tcs[j];
        const int kd = tc.kd, K = tc.K, nr = tc.nr;
        double* P1 = Psm + (long long)j * 2 * kdmax * kdmax;
        double* P2 = P1 + (long long)kdmax * kdmax;
        const double* P1g = v.arena + tc.p1;
        const double* P2g = v.arena + tc.p2;
        for (int e = tid; e < kd * kd; e += WIN_THREADS) {
            P1[e] = P1g[e];
            P2[e] = P2g[e];
        }
        if (gres) {
            const float* Gh = (const float*)(v.arena + tc.Gf);
            const long long ld = df32_ld(K);
            for (long long e = tid; e < (long long)nr * ld; e += WIN_THREADS) Gsm[e] = Gh[(long long)tc.r0 * ld + e];
        }
        const double* c0 = v.arena + tc.c0;
        for (int c = tid; c < K; c += WIN_THREADS) vs[c] = c0[c];
        __syncthreads();
        double* h0 = v.arena + tc.hist;
        for (int r = tid; r < nr; r += WIN_THREADS) {
            h0[tc.r0 + r] = vs[tc.r0 + r];
            own[j][0][r] = vs[tc.r0 + r];  // y^0 in slot 0
        }
        z_rows_sm(tc, P1, P2, vs, own[j][3], tmp);  // z^0 in slot 3
        double acc = 0;
        for (int r = tid; r < nr; r += WIN_THREADS) acc += own[j][0][r] * own[j][3][r];
        acc = wblock_sum(acc, red);
        if (tid == 0) {
            A.part_s[pofs + t] = acc;
            A.part_d[pofs + t] = 0.0;
        }
    }
    // after each barrier: the sums of the CTA's instances, reduced locally
    auto task_sums = [&]() {
        for (int j = 0; j < ntk; ++j) {
            const int i = tcs[j].inst;
            if (j > 0 && tcs[j - 1].inst == i) {
                if (tid == 0) {
                    s2_sm[j] = s2_sm[j - 1];
                    d2_sm[j] = d2_sm[j - 1];
                }
                continue;
            }
            block_sums2(A.part_s + pofs, A.part_d + pofs, A.inst_task0[i], A.inst_task0[i + 1], red, &s2_sm[j],
                        &d2_sm[j]);
        }
        __syncthreads();
        pofs = pofs ? 0 : A.n_tasks;
    };
    target += gridDim.x;
    ++gen;
    if (!release_barrier(&A.bar->count, &A.bar->gen, target, gen, v.err, A.spin_limit, nullptr, &go)) return;
    task_sums();

    for (int n = 0;; ++n) {
        for (int j = 0; j < ntk; ++j) {
            __syncthreads();
            if (!alive[j]) continue;
            const TaskCache& tc = tcs[j];
            const int K = tc.K, nr = tc.nr;
            const int t = A.cta_list[t_begin + j];
            // one round trip: s_n^2, D_{n-1}, y^n, b'^{n+1}
            const double s2 = tc.normalize ? s2_sm[j] : 1.0;
            const double d2 = (n >= 2 && tc.ngf_stop) ? d2_sm[j] : 1.0e300;
            const double* yn = v.arena + tc.hist + (long long)n * K;
            const int wp = A.win_prev[tc.inst];
            const double* bsrc = (wp > 0) ? v.arena + tc.bvec + (long long)min(n + 1, wp) * K : nullptr;
            double yv[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int c = tid + i * WIN_THREADS;
                yv[i] = (c < K) ? yn[c] : 0.0;
                bv[i] = (c < K && bsrc) ? bsrc[c] : 0.0;
            }
            if (tid == 0) {
                const double is_n = tc.normalize ? rsqrt(s2) : 1.0;
                const double s_n = tc.normalize ? s2 * is_n : 1.0;
                int stop = 0, w = n;
                if (n >= 2 && tc.ngf_stop && sqrt(fmax(d2, 0.0)) <= tc.ngf_tol) {
                    stop = 1;
                    w = n - 1;
                } else if (n >= tc.maxs || !isfinite(s_n) || s_n <= 0.0) {
                    stop = 1;
                    w = n;
                }
                if (tc.first) A.snorm[(long long)tc.inst * (cap + 1) + n] = s_n;
                if (stop) {
                    alive[j] = 0;
                    if (tc.first) {
                        A.win[tc.inst] = w;
                        if (!isfinite(s_n) || s_n <= 0.0) atomicOr(v.err, SWR_ERR_NUMERIC);
                        __threadfence();
                        atomicSub(A.n_active, 1);
                    }
                } else {
                    s_sc[0] = is_n;
                    s_sc[1] = is_prev[j];
                    is_prev[j] = is_n;
                }
                s_stop = stop;
            }
            __syncthreads();
            if (s_stop) continue;
            const double is_n = s_sc[0], is_p = s_sc[1];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int c = tid + i * WIN_THREADS;
                if (c < K) {
                    double val = yv[i] * is_n + tc.kdt * bv[i];
                    vs[c] = val;
                    float h = (float)val;
                    vf[c] = make_float2(h, (float)(val - (double)h));
                } else if (c < df32_ld(K)) {
                    vf[c] = make_float2(0.f, 0.f);  // padding columns of the FP32 planes
                }
            }
            __syncthreads();
            // fused double-single rows of y^{n+1} = G v and z^{n+1} = W v, two rows
            // per warp at a time, 16-byte loads of the four FP32 planes
            double* ynew = v.arena + tc.hist + (long long)(n + 1) * K;
            double* yslot = own[j][(n + 1) % 3];
            double* zslot = own[j][3 + (n + 1) % 3];
            const long long ld = df32_ld(K);
            const float* Ghg = (const float*)(v.arena + tc.Gf);
            const float* Gl = Ghg + (long long)K * ld;
            const float* Wh = (const float*)(v.arena + tc.Wf);
            const float* Wl = Wh + (long long)K * ld;
            for (int rb = tc.r0 + 2 * warp; rb < tc.r0 + nr; rb += 2 * nw) {
                const int nrow = min(2, tc.r0 + nr - rb);
                float yh[2] = {0.f, 0.f}, yl[2] = {0.f, 0.f}, zh[2] = {0.f, 0.f}, zl[2] = {0.f, 0.f};
                for (int c = lane * 4; c < ld; c += 128) {
                    const float4 xa = *reinterpret_cast<const float4*>(vf + c);
                    const float4 xb = *reinterpret_cast<const float4*>(vf + c + 2);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        if (i < nrow) {
                            const long long o = (long long)(rb + i) * ld + c;
                            const float* ghp = gres ? Gsm + (long long)(rb + i - tc.r0) * ld + c : Ghg + o;
                            const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            const float4 g0 = *reinterpret_cast<const float4*>(ghp);
                            const float4 g1 = ONEP ? zero4 : *reinterpret_cast<const float4*>(Gl + o);
                            const float4 w0 = *reinterpret_cast<const float4*>(Wh + o);
                            const float4 w1 = ONEP ? zero4 : *reinterpret_cast<const float4*>(Wl + o);
                            df32_acc(yh[i], yl[i], g0.x, g1.x, xa.x, xa.y);
                            df32_acc(zh[i], zl[i], w0.x, w1.x, xa.x, xa.y);
                            df32_acc(yh[i], yl[i], g0.y, g1.y, xa.z, xa.w);
                            df32_acc(zh[i], zl[i], w0.y, w1.y, xa.z, xa.w);
                            df32_acc(yh[i], yl[i], g0.z, g1.z, xb.x, xb.y);
                            df32_acc(zh[i], zl[i], w0.z, w1.z, xb.x, xb.y);
                            df32_acc(yh[i], yl[i], g0.w, g1.w, xb.z, xb.w);
                            df32_acc(zh[i], zl[i], w0.w, w1.w, xb.z, xb.w);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float sh, eh;
                        float oh = __shfl_xor_sync(0xffffffffu, yh[i], o), ol = __shfl_xor_sync(0xffffffffu, yl[i], o);
                        two_sum(yh[i], oh, sh, eh);
                        yh[i] = sh;
                        yl[i] = yl[i] + ol + eh;
                        oh = __shfl_xor_sync(0xffffffffu, zh[i], o);
                        ol = __shfl_xor_sync(0xffffffffu, zl[i], o);
                        two_sum(zh[i], oh, sh, eh);
                        zh[i] = sh;
                        zl[i] = zl[i] + ol + eh;
                    }
                    if (lane == 0 && i < nrow) {
                        const double y = (double)yh[i] + (double)yl[i];
                        ynew[rb + i] = y;
                        yslot[rb + i - tc.r0] = y;
                        zslot[rb + i - tc.r0] = (double)zh[i] + (double)zl[i];
                    }
                }
            }
            __syncthreads();
            // partials of s_{n+1}^2 and of D_n = ||y^n/s_n - y^{n-1}/s_{n-1}||^2_chi (own rows)
            const bool dn = (n >= 1 && tc.ngf_stop);
            const double* y_n = own[j][n % 3];
            const double* y_p = own[j][(n + 2) % 3];
            const double* z_n = own[j][3 + n % 3];
            const double* z_p = own[j][3 + (n + 2) % 3];
            double acc = 0, accd = 0;
            for (int r = tid; r < nr; r += WIN_THREADS) {
                acc += yslot[r] * zslot[r];
                if (dn) accd += (y_n[r] * is_n - y_p[r] * is_p) * (z_n[r] * is_n - z_p[r] * is_p);
            }
            acc = warp_sum(acc);
            accd = warp_sum(accd);
            if (lane == 0) {
                red[warp] = acc;
                red[16 + warp] = accd;
            }
            __syncthreads();
            if (tid == 0) {
                double a = 0, b = 0;
                for (int i = 0; i < nw; ++i) {
                    a += red[i];
                    b += red[16 + i];
                }
                A.part_s[pofs + t] = a;
                if (dn) A.part_d[pofs + t] = b;
            }
        }
        __syncthreads();
        target += gridDim.x;
        ++gen;
        if (!release_barrier(&A.bar->count, &A.bar->gen, target, gen, v.err, A.spin_limit, A.n_active, &go)) return;
        if (!go) return;
        task_sums();
    }
}

// ------------------------------------------------ resident single-plane window
//
// The split recursion (u^{m+1} = G y^m and w^{m+1} = G (kappa dt b'^{m+1}) in
// one pass over G, y^{m+1} = u^{m+1} / s_m + w^{m+1} formed after the barrier,
// the NGF stop decided one step later) with the fused window's static tasks:
// every CTA keeps its tasks and the G_hi rows of its (single) task resident
// in shared memory for the whole window, so a step reads from L2 only the
// G_lo plane of its rows (nothing in the FP32 phase, ONEP), the u and w of its
// subdomain and the partials; no W = (Pp (x) Pp) G.  One release-only grid
// barrier per step; each CTA sums its instances' partials itself, in a fixed
// order.  At most WIN_TPC tasks of at most WIN_RB rows per CTA.
// Dynamic shared memory: vs[kmax4] doubles | vf[kmax4] float2 | bf[kmax4] float2
// | tmp[rows_max + 2 kdmax] | Psm[tasks][2][kdmax^2] | (16-byte aligned) G_hi rows.
template <bool ONEP>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window_resident(SweepArgs A) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ TaskCache tcs[WIN_TPC];
    __shared__ double own[WIN_TPC][6][WIN_RB];  // y slots 0..2, z slots 3..5 (ring of 3, by step)
    __shared__ double is1_sm[WIN_TPC], is2_sm[WIN_TPC];  // 1/s_{m-1}, 1/s_{m-2} of the task's instance
    __shared__ int alive[WIN_TPC];
    __shared__ int s_stop;
    __shared__ double s2_sm[WIN_TPC], d2_sm[WIN_TPC];  // s_{m-1}^2 and D_{m-2} of each task's instance
    long long pofs = 0;
    int go = 1;
    const SwrDeviceView& v = A.v;
    const int t_begin = A.cta_task0[blockIdx.x];
    const int ntk = A.cta_task0[blockIdx.x + 1] - t_begin;
    const int cap = A.cap;
    const int kmax = df32_ld(A.kmax), kdmax = A.kdmax;
    double* vs = sm;
    float2* vf = (float2*)(sm + kmax);
    float2* bf = (float2*)(sm + 2 * kmax);
    double* tmp = sm + 3 * kmax;
    double* Psm = tmp + A.rows_max + 2 * kdmax;
    float* Gsm = (float*)(Psm + (long long)A.tasks_per_cta * 2 * kdmax * kdmax + (A.rows_max & 1));
    const bool gres = A.g_resident != 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = WIN_THREADS / 32;
    unsigned target = 0, gen = 0;

    for (int j = 0; j < ntk; ++j) {
        const int t = A.cta_list[t_begin + j];
        if (tid == 0) {
            tcs[j] = make_task_cache(A, t);
            alive[j] = 1;
            is1_sm[j] = 1.0;
            is2_sm[j] = 1.0;
        }
        __syncthreads();
        const TaskCache& tc = tcs[j];
        double* P1 = Psm + (long long)j * 2 * kdmax * kdmax;
        double* P2 = P1 + (long long)kdmax * kdmax;
        for (int e = tid; e < tc.kd * tc.kd; e += WIN_THREADS) {
            P1[e] = v.arena[tc.p1 + e];
            P2[e] = v.arena[tc.p2 + e];
        }
        if (gres) {
            const float* Gh = (const float*)(v.arena + tc.Gf);
            const long long ld = df32_ld(tc.K);
            for (long long e = tid; e < (long long)tc.nr * ld; e += WIN_THREADS) Gsm[e] = Gh[(long long)tc.r0 * ld + e];
        }
    }
    __syncthreads();
    auto task_sums = [&]() {
        for (int j = 0; j < ntk; ++j) {
            const int i = tcs[j].inst;
            if (j > 0 && tcs[j - 1].inst == i) {
                if (tid == 0) {
                    s2_sm[j] = s2_sm[j - 1];
                    d2_sm[j] = d2_sm[j - 1];
                }
                continue;
            }
            block_sums2(A.part_s + pofs, A.part_d + pofs, A.inst_task0[i], A.inst_task0[i + 1], red, &s2_sm[j],
                        &d2_sm[j]);
        }
        __syncthreads();
        pofs = pofs ? 0 : A.n_tasks;
    };

    for (int m = 0;; ++m) {
        for (int j = 0; j < ntk; ++j) {
            __syncthreads();
            if (!alive[j]) continue;
            const TaskCache& tc = tcs[j];
            const int K = tc.K, nr = tc.nr, ld = df32_ld(K);
            const int t = A.cta_list[t_begin + j];
            const SubDev& sd = v.sub[tc.sid];
            if (tid == 0) {
                int stop = 0;
                if (m >= 1) {
                    // the plain algorithm's stop at n = m-2 (D_{m-2}), else at n = m-1
                    // (cap, or s_{m-1} not positive and finite)
                    const double s2 = tc.normalize ? s2_sm[j] : 1.0;
                    const double is1 = tc.normalize ? rsqrt(s2) : 1.0;
                    const double s1 = tc.normalize ? s2 * is1 : 1.0;
                    int win = 0;
                    const bool bad = !isfinite(s1) || s1 <= 0.0;
                    if (m >= 3 && tc.ngf_stop && sqrt(fmax(d2_sm[j], 0.0)) <= tc.ngf_tol) {
                        stop = 1;
                        win = m - 2;
                    } else if (m - 1 >= tc.maxs || bad) {
                        stop = 1;
                        win = m - 1;
                    }
                    if (tc.first) A.snorm[(long long)tc.inst * (cap + 1) + m - 1] = s1;
                    if (stop) {
                        alive[j] = 0;
                        if (tc.first) {
                            A.win[tc.inst] = win;
                            if (bad) atomicOr(v.err, SWR_ERR_NUMERIC);
                            __threadfence();
                            atomicSub(A.n_active, 1);
                        }
                    } else {
                        is2_sm[j] = is1_sm[j];
                        is1_sm[j] = is1;
                    }
                }
                s_stop = stop;
            }
            __syncthreads();
            if (s_stop) continue;
            const double is1 = is1_sm[j], is2 = is2_sm[j];
            // full y^m = u^m / s_{m-1} + w^m of the subdomain (y^0 = c0) and kappa dt b'^{m+1}
            const int wp = A.win_prev[tc.inst];
            const double* bsrc = (wp > 0) ? v.arena + tc.bvec + (long long)min(m + 1, wp) * K : nullptr;
            {
                const double* U = v.arena + sd.work + (long long)(m & 1) * 2 * K;
                const double* Wv = U + K;
                const double* c0 = v.arena + tc.c0;
                for (int c = tid; c < ld; c += WIN_THREADS) {
                    if (c < K) {
                        const double y = m == 0 ? c0[c] : __ldcg(U + c) * is1 + __ldcg(Wv + c);
                        vs[c] = y;
                        vf[c] = ds_split(y);
                        bf[c] = bsrc ? ds_split(tc.kdt * bsrc[c]) : make_float2(0.f, 0.f);
                    } else {
                        vf[c] = make_float2(0.f, 0.f);
                        bf[c] = make_float2(0.f, 0.f);
                    }
                }
            }
            __syncthreads();
            double* ym = own[j][m % 3];
            double* hrow = v.arena + tc.hist + (long long)m * K;
            for (int r = tid; r < nr; r += WIN_THREADS) {
                ym[r] = vs[tc.r0 + r];
                hrow[tc.r0 + r] = vs[tc.r0 + r];
            }
            double* P1 = Psm + (long long)j * 2 * kdmax * kdmax;
            double* P2 = P1 + (long long)kdmax * kdmax;
            double* zm = own[j][3 + m % 3];
            z_rows_sm(tc, P1, P2, vs, zm, tmp);  // ends with a block barrier
            // partials: s_m^2 (own rows of y^m . z^m) and D_{m-1} = ||c^{m-1} - c^{m-2}||_chi^2
            {
                const bool dn = m >= 2 && tc.ngf_stop;
                const double* y1 = own[j][(m + 2) % 3];
                const double* y2 = own[j][(m + 1) % 3];
                const double* z1 = own[j][3 + (m + 2) % 3];
                const double* z2 = own[j][3 + (m + 1) % 3];
                double acc = 0, accd = 0;
                for (int r = tid; r < nr; r += WIN_THREADS) {
                    acc += ym[r] * zm[r];
                    if (dn) accd += (y1[r] * is1 - y2[r] * is2) * (z1[r] * is1 - z2[r] * is2);
                }
                acc = warp_sum(acc);
                accd = warp_sum(accd);
                if (lane == 0) {
                    red[warp] = acc;
                    red[16 + warp] = accd;
                }
                __syncthreads();
                if (tid == 0) {
                    double a = 0, b = 0;
                    for (int i = 0; i < nw; ++i) {
                        a += red[i];
                        b += red[16 + i];
                    }
                    A.part_s[pofs + t] = a;
                    if (dn) A.part_d[pofs + t] = b;
                }
            }
            if (m >= tc.maxs) continue;  // no step beyond the cap
            // rows of u^{m+1} = G y^m and w^{m+1} = G (kappa dt b'^{m+1}): two rows per
            // warp at a time, G_hi from shared memory (or L2), G_lo from L2 (ONEP: none)
            double* Un = v.arena + sd.work + (long long)((m + 1) & 1) * 2 * K;
            double* Wn = Un + K;
            const float* Ghg = (const float*)(v.arena + tc.Gf);
            const float* Gl = Ghg + (long long)K * ld;
            const bool hasb = bsrc != nullptr;
            for (int rb = tc.r0 + 2 * warp; rb < tc.r0 + nr; rb += 2 * nw) {
                const int nrow = min(2, tc.r0 + nr - rb);
                float yh[2] = {0.f, 0.f}, yl[2] = {0.f, 0.f}, wh[2] = {0.f, 0.f}, wl[2] = {0.f, 0.f};
                for (int c = lane * 4; c < ld; c += 128) {
                    const float4 xa = *reinterpret_cast<const float4*>(vf + c);
                    const float4 xb = *reinterpret_cast<const float4*>(vf + c + 2);
                    const float4 ba = *reinterpret_cast<const float4*>(bf + c);
                    const float4 bb = *reinterpret_cast<const float4*>(bf + c + 2);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        if (i < nrow) {
                            const long long o = (long long)(rb + i) * ld + c;
                            const float* ghp = gres ? Gsm + (long long)(rb + i - tc.r0) * ld + c : Ghg + o;
                            const float4 g0 = *reinterpret_cast<const float4*>(ghp);
                            const float4 g1 = ONEP ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                   : *reinterpret_cast<const float4*>(Gl + o);
                            df32_acc(yh[i], yl[i], g0.x, g1.x, xa.x, xa.y);
                            df32_acc(yh[i], yl[i], g0.y, g1.y, xa.z, xa.w);
                            df32_acc(yh[i], yl[i], g0.z, g1.z, xb.x, xb.y);
                            df32_acc(yh[i], yl[i], g0.w, g1.w, xb.z, xb.w);
                            if (hasb) {
                                df32_acc(wh[i], wl[i], g0.x, g1.x, ba.x, ba.y);
                                df32_acc(wh[i], wl[i], g0.y, g1.y, ba.z, ba.w);
                                df32_acc(wh[i], wl[i], g0.z, g1.z, bb.x, bb.y);
                                df32_acc(wh[i], wl[i], g0.w, g1.w, bb.z, bb.w);
                            }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float sh, eh;
                        float oh = __shfl_xor_sync(0xffffffffu, yh[i], o), ol = __shfl_xor_sync(0xffffffffu, yl[i], o);
                        two_sum(yh[i], oh, sh, eh);
                        yh[i] = sh;
                        yl[i] = yl[i] + ol + eh;
                        oh = __shfl_xor_sync(0xffffffffu, wh[i], o);
                        ol = __shfl_xor_sync(0xffffffffu, wl[i], o);
                        two_sum(wh[i], oh, sh, eh);
                        wh[i] = sh;
                        wl[i] = wl[i] + ol + eh;
                    }
                    if (lane == 0 && i < nrow) {
                        Un[rb + i] = (double)yh[i] + (double)yl[i];
                        Wn[rb + i] = (double)wh[i] + (double)wl[i];
                    }
                }
            }
        }
        __syncthreads();
        target += gridDim.x;
        ++gen;
        if (!release_barrier(&A.bar->count, &A.bar->gen, target, gen, v.err, A.spin_limit, A.n_active, &go)) return;
        if (!go) return;
        task_sums();
    }
}

// ------------------------------------------------------- single-barrier window
//
// Mixed precision, batches of any size, ONE reduce-barrier per step, G streamed
// from HBM once per step (8 bytes per element) through shared memory.  With
// y^{n+1} = G (y^n / s_n + kappa dt b'^{n+1}) = u^{n+1} / s_n + w^{n+1},
// u^{n+1} = G y^n, w^{n+1} = G (kappa dt b'^{n+1}), neither product needs
// s_n: phase X(m) forms the full y^m = u^m / s_{m-1} + w^m of each of its
// tasks' subdomains (s_{m-1} reduced at the last barrier), writes its rows,
// computes z^m = (Pp (x) Pp) y^m and the partials of s_m^2 and
// D_{m-1} = ||c^{m-1} - c^{m-2}||_chi^2, and the rows of u^{m+1} and w^{m+1}
// in one double-single pass over G.  The stop of the plain algorithm at step
// n is decided at X(n+2) (D_n is reduced at the barrier after X(n+1)); the
// steps computed beyond it are dropped.  u and w live, double-buffered by step
// parity, in the subdomain's assembly scratch.  Task state in global memory.
//
// The rows of G reach shared memory by bulk copies (cp.async.bulk, both FP32
// planes of a stage of rows per copy pair) into a ring of n_stages stages
// (2..SPLIT_NS_MAX, a plan parameter), each completing on its own mbarrier;
// thread 0 issues the next stage as soon as a slot is consumed, along the
// CTA's fixed order of (step, task, rows), so the copies stay in flight
// through the prologues of the tasks (y, z, partials) and through the grid
// barrier (G is constant: the first stages of step m+1 load while the barrier
// after step m completes).  Step m+1 streams the tasks still stepping after
// the decisions of step m; a task found stopped at m+1 has its stages waited
// for and skipped.
// Dynamic shared memory: vs[kmax4] doubles | vf[kmax4] float2 | bf[kmax4] float2
// | tmp[rows_max + 2 kdmax] | Ps[2 kdmax^2] | (128-byte aligned) ring of
// n_stages stages of stage_floats floats.
#define SPLIT_NS_MAX 8
#define SPLIT_FIFO 8        // claimed tasks queued between the producer thread and the consumers
#define SPLIT_CLAIM_MAX 8   // list positions per claim (at most)

__device__ inline unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Bounded wait for the phase of parity `par` of an mbarrier.
__device__ inline bool mbar_wait(const unsigned long long* bar, unsigned par, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(par)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Rows per stage for rows of ld floats: a power of two <= 32 with `planes`
// planes (2: hi and lo; 1: hi only) in stage_floats.
__device__ inline int split_stage_rows(int ld, int stage_floats, int planes = 2) {
    const int r = stage_floats / (planes * ld);
    return r >= 32 ? 32 : r >= 16 ? 16 : r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1;
}

// Last-arriver reduction of two partial arrays per instance (warp per instance
// from 8 instances on), s = sqrt(sum_a) and 1/s per instance into scal_out,
// the reset of the work queue of parity `qpar` (its list is used up), then the
// release (go = 0 when `nact` shows no instance still stepping).
__device__ bool reduce_barrier_sd(unsigned* count, unsigned* release, unsigned target, unsigned gen,
                                  const double* part_a, const double* part_b, const int* inst_task0, int n_inst,
                                  double* sums_a, double* sums_b, const InstDev* inst, double* scal_out, int* err,
                                  long long limit, double* red, const int* nact, int* go_out, SplitQueue* q, int qpar) {
    __shared__ int s_last, s_ok, s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned old = atomicAdd(count, 1u);
        s_last = (old == target - 1);
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const int lane = threadIdx.x & 31;
        if (n_inst < 8) {
            for (int i = 0; i < n_inst; ++i) {
                double xa = 0, xb = 0;
                for (int u = inst_task0[i] + threadIdx.x; u < inst_task0[i + 1]; u += WIN_THREADS) {
                    xa += __ldcg(part_a + u);
                    xb += __ldcg(part_b + u);
                }
                xa = wblock_sum(xa, red);
                xb = wblock_sum(xb, red);
                if (threadIdx.x == 0) {
                    sums_a[i] = xa;
                    sums_b[i] = xb;
                }
            }
        } else {
            for (int i = threadIdx.x >> 5; i < n_inst; i += WIN_THREADS / 32) {
                double xa = 0, xb = 0;
#pragma unroll 4
                for (int u = inst_task0[i] + lane; u < inst_task0[i + 1]; u += 32) {
                    xa += __ldcg(part_a + u);
                    xb += __ldcg(part_b + u);
                }
                xa = warp_sum(xa);
                xb = warp_sum(xb);
                if (lane == 0) {
                    sums_a[i] = xa;
                    sums_b[i] = xb;
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n_inst; i += WIN_THREADS) {
            const double sn = inst[i].normalize ? sqrt(sums_a[i]) : 1.0;
            scal_out[i] = sn;
            scal_out[n_inst + i] = 1.0 / sn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            q->claim[qpar] = 0;
            q->count[qpar] = 0;
            const int go = nact ? (__ldcg(nact) > 0) : 1;
            s_go = go;
            __threadfence();
            st_release_u32(release, 2u * gen + (unsigned)go);
        }
    } else if (threadIdx.x == 0) {
        long long it = 0;
        unsigned w = 0;
        while ((w = ld_acquire_u32(release)) < 2u * gen) {
            if (++it > limit) { atomicOr(err, SWR_ERR_TIMEOUT); s_ok = 0; break; }
            if ((it & 255) == 0 && *(volatile int*)err) { s_ok = 0; break; }
            __nanosleep(20);
        }
        s_go = (int)(w & 1u);
        __threadfence();
    }
    if (threadIdx.x == 0 && *(volatile int*)err) s_ok = 0;  // one verdict for the whole CTA
    __syncthreads();
    *go_out = s_go;
    return s_ok != 0;
}

// Consumer-group barrier of the split window: warps 1..7 (named barrier 1).
__device__ inline void split_cbar() { asm volatile("bar.sync 1, %0;" ::"n"(WIN_THREADS - 32) : "memory"); }

// Consumer-group barrier that also ORs x over the group (the same result in
// every consumer thread).
__device__ inline int split_cbar_or(int x) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(x), "n"(WIN_THREADS - 32)
        : "memory");
    return r;
}

__device__ inline void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Rows [r0, r0+nr) of z = (P1 (x) P2) y (N = 2) or P1 y (N = 1) by the consumer
// group (threads ct = 0..CT-1): the factors are staged in shared memory (Ps),
// then every thread computes whole outputs of the two small products
//   tmp[bb][c] = sum_e Y[c][e] P2[b0+bb][e],   z[(a,b)] = sum_c P1[a][c] tmp[b-b0][c].
__device__ void z_rows_group(const TaskCache& tc, const double* P1g, const double* P2g, const double* ys, double* z,
                             double* tmp, double* Ps, int ct, int CT) {
    const int kd = tc.kd, r0 = tc.r0, r1 = tc.r0 + tc.nr, kk = kd * kd;
    double* P1 = Ps;
    double* P2 = Ps + kk;
    for (int e = ct; e < kk; e += CT) {
        P1[e] = P1g[e];
        if (tc.N == 2) P2[e] = P2g[e];
    }
    split_cbar();
    if (tc.N == 1) {
        for (int r = r0 + ct; r < r1; r += CT) {
            double acc = 0;
            for (int c = 0; c < kd; ++c) acc = fma(P1[r * kd + c], ys[c], acc);
            z[r - r0] = acc;
        }
        split_cbar();
        return;
    }
    const int b0 = r0 / kd, b1 = (r1 - 1) / kd, nb = b1 - b0 + 1;
    for (int item = ct; item < nb * kd; item += CT) {
        const int bb = item / kd, c = item - bb * kd;
        const double* p2 = P2 + (b0 + bb) * kd;
        double acc = 0;
        for (int e = 0; e < kd; ++e) acc = fma(ys[c + kd * e], p2[e], acc);
        tmp[item] = acc;
    }
    split_cbar();
    for (int r = r0 + ct; r < r1; r += CT) {
        const int b = r / kd, a = r - b * kd;
        const double* p1 = P1 + a * kd;
        const double* tb = tmp + (b - b0) * kd;
        double acc = 0;
        for (int c = 0; c < kd; ++c) acc = fma(p1[c], tb[c], acc);
        z[r - r0] = acc;
    }
    split_cbar();
}

// Rows [r0, r0+nr) of z = (P1 (x) P2) y (N = 2) or P1 y (N = 1) in
// double-single for the consumer group (CT threads from ct): y as pairs in
// shared memory, the Kronecker factors staged as pairs (split on the integer
// pipes), tmp[bb][c] = sum_e Y[c][e] P2[b0+bb][e] with 4 threads per entry,
// z[(a, b)] = sum_c P1[a][c] tmp[b-b0][c] with 8 threads per row; z to FP64.
__device__ void z_rows_group_ds(const TaskCache& tc, const double* P1g, const double* P2g, const float2* ys, double* z,
                                float2* tmp, float2* Ps, int ct, int CT) {
    const int kd = tc.kd, r0 = tc.r0, nr = tc.nr, kk = kd * kd;
    float2* P1 = Ps;
    float2* P2 = Ps + kk;
    for (int e = ct; e < kk; e += CT) {
        P1[e] = dsp_split_int(P1g[e]);
        if (tc.N == 2) P2[e] = dsp_split_int(P2g[e]);
    }
    split_cbar();
    if (tc.N == 2) {
        const int b0 = r0 / kd, nb = (r0 + nr - 1) / kd - b0 + 1, items = nb * kd;
        for (int base = 0; base < items; base += CT / 4) {
            const int it = base + (ct >> 2), g = ct & 3;
            float2 acc = make_float2(0.f, 0.f);
            if (it < items) {
                const int bb = it / kd, c = it - bb * kd;
                const float2* p2 = P2 + (b0 + bb) * kd;
                for (int e = g; e < kd; e += 4) ds_fma(acc.x, acc.y, ys[c + kd * e], p2[e]);
            }
            acc = dsp_shfl_add(acc, 1);
            acc = dsp_shfl_add(acc, 2);
            if (it < items && g == 0) tmp[it] = acc;
        }
        split_cbar();
        for (int base = 0; base < nr; base += CT / 8) {
            const int i = base + (ct >> 3), g = ct & 7;
            float2 acc = make_float2(0.f, 0.f);
            if (i < nr) {
                const int r = r0 + i, b = r / kd, a = r - b * kd;
                const float2* p1 = P1 + a * kd;
                const float2* tb = tmp + (b - b0) * kd;
                for (int c = g; c < kd; c += 8) ds_fma(acc.x, acc.y, p1[c], tb[c]);
            }
            acc = dsp_shfl_add(acc, 1);
            acc = dsp_shfl_add(acc, 2);
            acc = dsp_shfl_add(acc, 4);
            if (i < nr && g == 0) z[i] = dsp_to_double(acc);
        }
    } else {
        for (int base = 0; base < nr; base += CT / 8) {
            const int i = base + (ct >> 3), g = ct & 7;
            float2 acc = make_float2(0.f, 0.f);
            if (i < nr) {
                const float2* p1 = P1 + (r0 + i) * kd;
                for (int c = g; c < kd; c += 8) ds_fma(acc.x, acc.y, p1[c], ys[c]);
            }
            acc = dsp_shfl_add(acc, 1);
            acc = dsp_shfl_add(acc, 2);
            acc = dsp_shfl_add(acc, 4);
            if (i < nr && g == 0) z[i] = dsp_to_double(acc);
        }
    }
    split_cbar();
}

// One double-single chunk of 4 columns of a staged row into (yh, yl) and,
// with HASB, (wh, wl); ONEP: the row's lo plane is absent (taken as 0).
template <bool HASB, bool ONEP>
__device__ inline void split_chunk(const float* sh, const float* sl, const float2* vf, const float2* bf, int c,
                                   float& yh, float& yl, float& wh, float& wl) {
    const float4 g0 = *reinterpret_cast<const float4*>(sh + c);
    const float4 g1 = ONEP ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(sl + c);
    const float4 xa = *reinterpret_cast<const float4*>(vf + c);
    const float4 xb = *reinterpret_cast<const float4*>(vf + c + 2);
    df32_acc(yh, yl, g0.x, g1.x, xa.x, xa.y);
    df32_acc(yh, yl, g0.y, g1.y, xa.z, xa.w);
    df32_acc(yh, yl, g0.z, g1.z, xb.x, xb.y);
    df32_acc(yh, yl, g0.w, g1.w, xb.z, xb.w);
    if (HASB) {
        const float4 ba = *reinterpret_cast<const float4*>(bf + c);
        const float4 bb = *reinterpret_cast<const float4*>(bf + c + 2);
        df32_acc(wh, wl, g0.x, g1.x, ba.x, ba.y);
        df32_acc(wh, wl, g0.y, g1.y, ba.z, ba.w);
        df32_acc(wh, wl, g0.z, g1.z, bb.x, bb.y);
        df32_acc(wh, wl, g0.w, g1.w, bb.z, bb.w);
    }
}

// (h, l) += (oh, ol) in double-single.
__device__ inline void ds_add(float& h, float& l, float oh, float ol) {
    float s, e;
    two_sum(h, oh, s, e);
    h = s;
    l = l + ol + e;
}

// One staged row by one warp: lanes over groups of 4 columns, two accumulator
// pairs per product (alternate column groups), shuffle sum; the row's values of
// G y and G b to all lanes.
template <bool HASB, bool ONEP>
__device__ inline void split_row(const float* sh, const float* sl, const float2* vf, const float2* bf, int ld,
                                 int lane, float2& y, float2& w) {
    float yh0 = 0.f, yl0 = 0.f, wh0 = 0.f, wl0 = 0.f, yh1 = 0.f, yl1 = 0.f, wh1 = 0.f, wl1 = 0.f;
    int c = lane * 4;
    for (; c + 128 < ld; c += 256) {
        split_chunk<HASB, ONEP>(sh, sl, vf, bf, c, yh0, yl0, wh0, wl0);
        split_chunk<HASB, ONEP>(sh, sl, vf, bf, c + 128, yh1, yl1, wh1, wl1);
    }
    if (c < ld) split_chunk<HASB, ONEP>(sh, sl, vf, bf, c, yh0, yl0, wh0, wl0);
    ds_add(yh0, yl0, yh1, yl1);
    if (HASB) ds_add(wh0, wl0, wh1, wl1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ds_add(yh0, yl0, __shfl_xor_sync(0xffffffffu, yh0, o), __shfl_xor_sync(0xffffffffu, yl0, o));
        if (HASB) ds_add(wh0, wl0, __shfl_xor_sync(0xffffffffu, wh0, o), __shfl_xor_sync(0xffffffffu, wl0, o));
    }
    y = dsp_norm(yh0, yl0);
    w = HASB ? dsp_norm(wh0, wl0) : make_float2(0.f, 0.f);
}

// ONEP: only the hi plane of G is staged (the FP32-rounded step matrix of
// SWR_PREC_FP32_REFINED before its switch): one bulk copy per stage, twice the
// rows per stage, the lo terms taken as 0.
template <bool ONEP>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window_split(SweepArgs A) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ __align__(8) unsigned long long full[SPLIT_NS_MAX], empty[SPLIT_NS_MAX];
    __shared__ __align__(8) unsigned long long ff[SPLIT_FIFO], fe[SPLIT_FIFO];
    __shared__ int fifo[SPLIT_FIFO];
    __shared__ int cbuf[SPLIT_CLAIM_MAX];
    int go = 1;
    const SwrDeviceView& v = A.v;
    const int cap = A.cap, ni = v.n_inst, SC = A.stage_floats, nt = A.n_tasks;
    const unsigned NS = (unsigned)A.n_stages;
    const int kmax = df32_ld(A.kmax), kdmax = A.kdmax;
    double* vs = sm;
    float2* vf = (float2*)(sm + kmax);
    float2* bf = (float2*)(sm + 2 * kmax);
    double* tmp = sm + 3 * kmax;
    double* Ps = tmp + A.rows_max + 2 * kdmax;
    float* ring = (float*)(sm + ((3 * kmax + A.rows_max + 2 * kdmax + 2 * kdmax * kdmax + 15) & ~15));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NCW = WIN_THREADS / 32 - 1, CT = WIN_THREADS - 32;  // consumer warps, threads
    const long long wait_limit = A.spin_limit >> 4;
    // the waits for this CTA's own bulk copies before it ends do not follow the
    // caller's spin limit: a CTA must not exit while a copy still writes its
    // shared memory, and a copy of a few KB completes within microseconds
    const long long copy_limit = wait_limit > (1LL << 20) ? wait_limit : (1LL << 20);
    SplitQueue* q = A.q;
    unsigned target = 0, gen = 0;
    bool failed = false;  // a bounded wait gave up: the rest of the window skips its waits
    // producer (warp 0, lane 0)
    unsigned issued = 0, pushed = 0;
    int c_next = 0, c_end = 0;
    unsigned c_hint = 0;
    // consumers (warps 1..7)
    unsigned taken = 0, used = 0;  // FIFO entries taken, stages used
    auto own = [&](const TaskCache& tc, int slot) -> double* { return A.g_own + tc.own + (long long)slot * tc.nr; };
    auto wait = [&](unsigned long long* bar, unsigned par) {
        if (failed) return;
        if (!mbar_wait(bar, par, wait_limit)) {
            atomicOr(v.err, SWR_ERR_TIMEOUT);
            failed = true;
        }
    };

    if (tid == 0) {
        for (unsigned i = 0; i < NS; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(NCW) : "memory");
        }
        for (int i = 0; i < SPLIT_FIFO; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ff[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fe[i])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    for (int m = 0;; ++m) {
        const double* sc1 = A.scal_inst + ((m - 1) & 1) * 2 * ni;  // s_{m-1}, 1/s_{m-1}
        const double* sc2 = A.scal_inst + ((m - 2) & 1) * 2 * ni;  // s_{m-2}, 1/s_{m-2}
        if (warp == 0) {
            if (lane == 0) {
                // ------------------------------------------------ producer
                auto push = [&](int val) {
                    const unsigned s = pushed % SPLIT_FIFO;
                    if (pushed >= SPLIT_FIFO) wait(&fe[s], (pushed / SPLIT_FIFO - 1) & 1u);
                    if (failed) return;  // a wait gave up: the consumers leave on their own bounded waits
                    fifo[s] = val;
                    mbar_arrive(&ff[s]);
                    ++pushed;
                };
                c_next = c_end = 0;
                c_hint = 0;
                unsigned a_pos = 0;
                int a_t = -1, a_par = 0;
                for (;;) {
                    if (failed) break;  // a wait gave up: claim and issue nothing more
                    // next task of step m: guided chunks of the step's list
                    if (c_next == c_end) {
                        const unsigned n = m == 0 ? (unsigned)nt : __ldcg(&q->count[m & 1]);
                        unsigned b = c_hint < n ? (n - c_hint) / (2u * gridDim.x) : 1u;
                        b = b < 1u ? 1u : (b > SPLIT_CLAIM_MAX ? SPLIT_CLAIM_MAX : b);
                        const unsigned i = atomicAdd(&q->claim[m & 1], b);
                        c_hint = i + b;
                        if (i >= n) break;
                        const unsigned e = i + b < n ? i + b : n;
                        for (unsigned k = i; k < e; ++k)
                            cbuf[k - i] = m == 0 ? (int)k : __ldcg(A.q_list + (size_t)(m & 1) * nt + k);
                        c_next = 0;
                        c_end = (int)(e - i);
                    }
                    const int t = cbuf[c_next++];
                    const TaskCache tc = make_task_cache(A, t);
                    if (m >= 1) {
                        // the plain algorithm's stop at n = m-2 (D_{m-2}), else at n = m-1
                        // (cap, or s_{m-1} not positive and finite)
                        const double s1 = __ldcg(sc1 + tc.inst);
                        int stop = 0, win = 0, bad = 0;
                        if (m >= 3 && tc.ngf_stop && sqrt(fmax(__ldcg(A.sums_d + tc.inst), 0.0)) <= tc.ngf_tol) {
                            stop = 1;
                            win = m - 2;
                        } else if (m - 1 >= tc.maxs || !isfinite(s1) || s1 <= 0.0) {
                            stop = 1;
                            win = m - 1;
                            bad = !isfinite(s1) || s1 <= 0.0;
                        }
                        if (tc.first) A.snorm[(long long)tc.inst * (cap + 1) + m - 1] = s1;
                        if (stop) {
                            if (tc.first) {
                                A.win[tc.inst] = win;
                                if (bad) atomicOr(v.err, SWR_ERR_NUMERIC);
                                __threadfence();
                                atomicSub(A.n_active, 1);
                            }
                            continue;
                        }
                    }
                    // still stepping after the decisions of step m: a member of step
                    // m+1's list (the entry is stored one append later, or at the end
                    // of the step, so that the atomic's round trip overlaps other work)
                    if (a_t >= 0) A.q_list[(size_t)a_par * nt + a_pos] = a_t;
                    a_par = (m + 1) & 1;
                    a_pos = atomicAdd(&q->count[a_par], 1u);
                    a_t = t;
                    const bool str = m < tc.maxs;
                    push(2 * t + (str ? 1 : 0));
                    if (!str) continue;
                    // the task's stages: rows [rb, rb + rs) of both planes per stage
                    const int ld = df32_ld(tc.K), rs = split_stage_rows(ld, SC, ONEP ? 1 : 2);
                    const float* Gh = (const float*)(v.arena + tc.Gf);
                    const long long plane = (long long)tc.K * ld;
                    for (int rb = tc.r0; rb < tc.r0 + tc.nr; rb += rs) {
                        const unsigned s = issued % NS;
                        if (issued >= NS) wait(&empty[s], (issued / NS - 1) & 1u);
                        if (failed) break;  // never a copy into a slot whose release was not seen
                        const int nrow = min(rs, tc.r0 + tc.nr - rb);
                        const unsigned bytes = (unsigned)nrow * ld * 4u, mb = smem_u32(&full[s]);
                        float* dst = ring + (size_t)s * SC;
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                                     "r"((ONEP ? 1u : 2u) * bytes)
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                            "[%3];" ::"r"(smem_u32(dst)),
                            "l"(Gh + (long long)rb * ld), "r"(bytes), "r"(mb)
                            : "memory");
                        if (!ONEP)
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(dst + rs * ld)),
                                "l"(Gh + plane + (long long)rb * ld), "r"(bytes), "r"(mb)
                                : "memory");
                        ++issued;
                    }
                }
                if (a_t >= 0) A.q_list[(size_t)a_par * nt + a_pos] = a_t;
                push(-1);  // end of the step's tasks
            }
            __syncwarp();
        } else {
            // ------------------------------------------------ consumers
            const int ct = tid - 32, cw = warp - 1;
            for (;;) {
                const unsigned fs = taken % SPLIT_FIFO;
                wait(&ff[fs], (taken / SPLIT_FIFO) & 1u);
                // every consumer has the entry and the previous task's rows are done; a
                // wait that gave up anywhere in the group ends the step for all of it
                const int e = split_cbar_or(failed ? 1 : 0) ? -1 : fifo[fs];
                ++taken;
                split_cbar();
                if (ct == 0) mbar_arrive(&fe[fs]);
                if (e < 0) break;
                const int t = e >> 1;
                const bool str = (e & 1) != 0;
                const TaskCache tc = make_task_cache(A, t);
                const int K = tc.K, nr = tc.nr, ld = df32_ld(K);
                const SubDev& sd = v.sub[tc.sid];
                const int wp = A.win_prev[tc.inst];
                const double* bsrc = (wp > 0) ? v.arena + tc.bvec + (long long)min(m + 1, wp) * K : nullptr;
                // full y^m = u^m / s_{m-1} + w^m (y^0 = c0) and kappa dt b'^{m+1} as
                // double-single pairs on the FP32 and integer pipes (u, w are
                // stored as pairs; the FP64 unit of this part is slow)
                const double is1 = m >= 1 ? __ldcg(sc1 + ni + tc.inst) : 1.0;
                const double is2 = m >= 2 ? __ldcg(sc2 + ni + tc.inst) : 1.0;
                float2* ys2 = reinterpret_cast<float2*>(vs);  // y^m as pairs (the matvec input is vf)
                {
                    const float2 isf = ds_split(is1), kdt2 = ds_split(tc.kdt);
                    const float2* U = reinterpret_cast<const float2*>(v.arena + sd.work + (long long)(m & 1) * 2 * K);
                    // w^m: formed by this kernel at step m - 1 (G times kappa dt b'^m), or
                    // read from the Robin response precomputed for every step
                    // (swr_robin.cu; no antisymmetric instance then), zero
                    // without Robin data
                    const float2* Wv = U + K;
                    const float2* Wpre = nullptr;
                    if (A.robin_w && m >= 1 && wp > 0)
                        Wpre = reinterpret_cast<const float2*>(v.arena + sd.Wr) + (long long)min(m, wp) * ld;
                    const double* c0 = v.arena + tc.c0;
                    // antisymmetric states: on a diagonal subdomain (its own mirror) the
                    // products act on (y - swap(y)) / 2 and likewise b'; y itself is kept
                    // for the history and z
                    const bool anti = diagonal_anti(v, tc);
                    const float2 *Um = nullptr, *Wm = nullptr;
                    const double *c0m = nullptr, *bm = nullptr;
                    if (anti) {
                        const SubDev& ms = v.sub[mirror_sid(v, tc)];
                        Um = reinterpret_cast<const float2*>(v.arena + ms.work + (long long)(m & 1) * 2 * K);
                        Wm = Um + K;
                        c0m = v.arena + ms.c0;
                        if (bsrc) bm = v.arena + ms.bvec + (long long)min(m + 1, wp) * K;
                    }
                    const float2 half = make_float2(0.5f, 0.f);
                    for (int c = ct; c < ld; c += CT) {
                        if (c < K) {
                            auto ld2 = [](const float2* p) {
                                const unsigned long long u = __ldcg(reinterpret_cast<const unsigned long long*>(p));
                                return make_float2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
                            };
                            const float2 wm = A.robin_w ? (Wpre ? ld2(Wpre + c) : make_float2(0.f, 0.f)) : ld2(Wv + c);
                            const float2 y = m == 0 ? dsp_split_int(c0[c]) : dsp_add(dsp_mul(ld2(U + c), isf), wm);
                            float2 yp = y, bp = (bsrc && !A.robin_w) ? dsp_split_int(bsrc[c]) : make_float2(0.f, 0.f);
                            if (anti) {
                                const int sc = swap_index(c, tc.kd);
                                const float2 ym_ = m == 0 ? dsp_split_int(c0m[sc])
                                                          : dsp_add(dsp_mul(ld2(Um + sc), isf), ld2(Wm + sc));
                                yp = dsp_mul(half, dsp_add(y, dsp_neg(ym_)));
                                if (bsrc) bp = dsp_mul(half, dsp_add(bp, dsp_neg(dsp_split_int(__ldcg(bm + sc)))));
                            }
                            ys2[c] = y;
                            vf[c] = yp;
                            bf[c] = (bsrc && !A.robin_w) ? dsp_mul(kdt2, bp) : make_float2(0.f, 0.f);
                        } else {
                            ys2[c] = make_float2(0.f, 0.f);
                            vf[c] = make_float2(0.f, 0.f);
                            bf[c] = make_float2(0.f, 0.f);
                        }
                    }
                }
                split_cbar();
                double* ym = own(tc, m % 3);
                double* hrow = v.arena + tc.hist + (long long)m * K;
                for (int r = ct; r < nr; r += CT) {
                    const double yd = m == 0 ? v.arena[tc.c0 + tc.r0 + r] : dsp_to_double(ys2[tc.r0 + r]);
                    ym[r] = yd;
                    hrow[tc.r0 + r] = yd;
                }
                double* zm = own(tc, 3 + m % 3);
                z_rows_group_ds(tc, v.arena + tc.p1, v.arena + tc.p2, ys2, zm, reinterpret_cast<float2*>(tmp),
                                reinterpret_cast<float2*>(Ps), ct, CT);
                // partials: s_m^2 (own rows of y^m . z^m) and D_{m-1}
                {
                    const bool dn = m >= 2 && tc.ngf_stop;
                    const double* y1 = own(tc, (m + 2) % 3);
                    const double* y2 = own(tc, (m + 1) % 3);
                    const double* z1 = own(tc, 3 + (m + 2) % 3);
                    const double* z2 = own(tc, 3 + (m + 1) % 3);
                    double acc = 0, accd = 0;
                    for (int r = ct; r < nr; r += CT) {
                        acc += ym[r] * zm[r];
                        if (dn) accd += (y1[r] * is1 - y2[r] * is2) * (z1[r] * is1 - z2[r] * is2);
                    }
                    acc = warp_sum(acc);
                    accd = warp_sum(accd);
                    if (lane == 0) {
                        red[warp] = acc;
                        red[16 + warp] = accd;
                    }
                    split_cbar();
                    if (ct == 0) {
                        double a = 0, b = 0;
                        for (int i = 1; i <= NCW; ++i) {
                            a += red[i];
                            b += red[16 + i];
                        }
                        const double w = mirror_weight(v, tc);
                        A.part_s[t] = a * w;
                        if (dn) A.part_d[t] = b * w;
                    }
                }
                if (!str) continue;
                // rows of u^{m+1} = G y^m and w^{m+1} = G (kappa dt b'^{m+1}) from the
                // staged rows: row r0 + o of the task to consumer warp o mod 7, whole
                // rows per warp, no block barrier between stages
                const int rs = split_stage_rows(ld, SC, ONEP ? 1 : 2);
                float2* Un = reinterpret_cast<float2*>(v.arena + sd.work + (long long)((m + 1) & 1) * 2 * K);
                float2* Wn = Un + K;
                const bool hasb = bsrc != nullptr && !A.robin_w;  // else u = G y^m only
                for (int rb = tc.r0; rb < tc.r0 + nr; rb += rs) {
                    const int nrow = min(rs, tc.r0 + nr - rb);
                    const unsigned s = used % NS;
                    wait(&full[s], (used / NS) & 1u);
                    const float* stage = ring + (size_t)s * SC;
                    int r = ((cw - (rb - tc.r0)) % NCW + NCW) % NCW;
                    for (; r < nrow; r += NCW) {
                        float2 y, w;
                        if (hasb)
                            split_row<true, ONEP>(stage + (size_t)r * ld, stage + (size_t)(rs + r) * ld, vf, bf, ld,
                                                  lane, y, w);
                        else
                            split_row<false, ONEP>(stage + (size_t)r * ld, stage + (size_t)(rs + r) * ld, vf, bf, ld,
                                                   lane, y, w);
                        if (lane == 0) {
                            Un[rb + r] = y;
                            Wn[rb + r] = w;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    ++used;
                }
            }
        }
        __syncthreads();
        target += gridDim.x;
        ++gen;
        const bool ok = reduce_barrier_sd(&A.bar->count, &A.bar->gen, target, gen, A.part_s, A.part_d, A.inst_task0,
                                          ni, A.sums_s, A.sums_d, v.inst, A.scal_inst + (m & 1) * 2 * ni, v.err,
                                          A.spin_limit, red, A.n_active, &go, q, m & 1);
        if (!ok || !go) {
            // every stage issued has been consumed (each step's list ends with its
            // stages), except after a wait that gave up: the producer waits
            // (bounded) for the last copy into each slot before the CTA ends
            if (tid == 0)
                for (unsigned i = issued > NS ? issued - NS : 0; i < issued; ++i)
                    mbar_wait(&full[i % NS], (i / NS) & 1u, copy_limit);
            __syncthreads();
            return;
        }
    }
}

__global__ void k_window_reset(SweepArgs A, int n_inst) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.bar->count = 0;
        A.bar->gen = 0;
        *A.n_active = n_inst;
        A.q->claim[0] = A.q->claim[1] = 0;
        A.q->count[0] = A.q->count[1] = 0;
    }
    if (blockIdx.x == 0 && A.cl_slots)
        for (int i = threadIdx.x; i < 8 * A.n_tasks; i += blockDim.x) A.cl_slots[i] = 0ULL;
}

// Split of the FP64 step-matrix inverse into FP32 pairs (mixed precision).
// G_hi = fl32(G), G_lo = fl32(G - G_hi), rows padded to df32_ld(K) columns with zeros.
__global__ void k_split_df32(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, ld = df32_ld(K);
    const long long n = (long long)K * ld;
    const double* G = v.arena + s.Gm;
    float* Gh = (float*)(v.arena + s.Gf);
    float* Gl = Gh + n;
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < n; e += (long long)blockDim.x * gridDim.x) {
        const long long r = e / ld;
        const int c = (int)(e - r * ld);
        const double g = c < K ? G[r * K + c] : 0.0;
        const float h = (float)g;
        Gh[e] = h;
        Gl[e] = (float)(g - (double)h);
        if (c >= K && s.Wf) {  // padding columns of W (its other columns come from k_make_w)
            float* Wh = (float*)(v.arena + s.Wf);
            Wh[e] = 0.f;
            Wh[n + e] = 0.f;
        }
    }
}

// W = (Pp1 (x) Pp2) G (N = 2) or Pp1 G (N = 1), column by column in FP64, stored
// as FP32 pairs.  Column j of G reshaped Y[c][e] = G[c + kd e][j]:
// W[(a,b), j] = sum_{c,e} P1[a][c] Y[c][e] P2[b][e].
__global__ void k_make_w(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, kd = s.kd;
    T1Layout lay(s.q, kd);
    const double* P1 = v.arena + s.t1[0] + lay.mat(M_PP);
    const double* P2 = v.arena + s.t1[s.N == 2 ? 1 : 0] + lay.mat(M_PP);
    const double* G = v.arena + s.Gm;
    const long long ld = df32_ld(K);
    float* Wh = (float*)(v.arena + s.Wf);
    float* Wl = Wh + (long long)K * ld;
    extern __shared__ double sw[];
    double* Y = sw;            // K
    double* T = sw + K;        // kd * kd (N = 2)
    for (int j = blockIdx.x; j < K; j += gridDim.x) {
        for (int r = threadIdx.x; r < K; r += blockDim.x) Y[r] = G[(long long)r * K + j];
        __syncthreads();
        if (s.N == 1) {
            for (int a = threadIdx.x; a < K; a += blockDim.x) {
                double acc = 0;
                for (int c = 0; c < K; ++c) acc += P1[a * kd + c] * Y[c];
                float h = (float)acc;
                Wh[(long long)a * ld + j] = h;
                Wl[(long long)a * ld + j] = (float)(acc - (double)h);
            }
        } else {
            for (int e2 = threadIdx.x; e2 < kd * kd; e2 += blockDim.x) {  // T[a][e] = sum_c P1[a][c] Y[c][e]
                int a = e2 / kd, e = e2 % kd;
                double acc = 0;
                for (int c = 0; c < kd; ++c) acc += P1[a * kd + c] * Y[c + kd * e];
                T[a * kd + e] = acc;
            }
            __syncthreads();
            for (int m = threadIdx.x; m < K; m += blockDim.x) {  // W[(a,b)] = sum_e T[a][e] P2[b][e]
                int a = m % kd, b = m / kd;
                double acc = 0;
                for (int e = 0; e < kd; ++e) acc += T[a * kd + e] * P2[b * kd + e];
                float h = (float)acc;
                Wh[(long long)m * ld + j] = h;
                Wl[(long long)m * ld + j] = (float)(acc - (double)h);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- host side

size_t window_smem(int kmax, int kdmax, int rows_max, int tasks_in_smem, long long g_resident_floats) {
    return (2 * (size_t)df32_ld(kmax) + (size_t)rows_max + 2 * (size_t)kdmax + (size_t)tasks_in_smem * 2 * kdmax * kdmax +
            1) * sizeof(double) +
           (size_t)g_resident_floats * sizeof(float);
}

size_t window_smem_split(int kmax, int kdmax, int rows_max, int stage_floats, int n_stages) {
    return (((3 * (size_t)df32_ld(kmax) + (size_t)rows_max + 2 * (size_t)kdmax + 2 * (size_t)kdmax * kdmax + 15) &
             ~(size_t)15) *
            sizeof(double)) +
           (size_t)n_stages * stage_floats * sizeof(float);
}

// Resident window: vs, vf, bf (3 kmax4 doubles), tmp, the tasks' Kronecker
// factors and the resident G_hi rows.
size_t window_smem_resident(int kmax, int kdmax, int rows_max, int tasks_in_smem, long long g_resident_floats) {
    return (3 * (size_t)df32_ld(kmax) + (size_t)rows_max + 2 * (size_t)kdmax +
            (size_t)tasks_in_smem * 2 * kdmax * kdmax + 1) * sizeof(double) +
           (size_t)g_resident_floats * sizeof(float);
}

int window_tasks_per_cta_max() { return WIN_TPC; }
int window_rows_per_task_max() { return WIN_RB; }

static const void* window_kernel(int variant, bool df32, bool onep) {
    if (variant == WIN_RESIDENT)
        return onep ? (const void*)k_window_resident<true> : (const void*)k_window_resident<false>;
    if (variant == WIN_FUSED) return onep ? (const void*)k_window_fused<true> : (const void*)k_window_fused<false>;
    if (variant == WIN_SPLIT) return onep ? (const void*)k_window_split<true> : (const void*)k_window_split<false>;
    return df32 ? (const void*)k_window_2ph<true> : (const void*)k_window_2ph<false>;
}

// Resident CTAs per SM of the window kernel: the smaller of its two instantiations
// (both planes, hi plane only) where the variant has both.
cudaError_t window_occupancy(int* blocks_per_sm, size_t smem, int variant, bool df32) {
    int best = 1 << 30;
    for (int o = 0; o < 2; ++o) {
        if (o == 1 && variant != WIN_FUSED && variant != WIN_SPLIT && variant != WIN_RESIDENT) break;
        const void* f = window_kernel(variant, df32, o == 1);
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, WIN_THREADS, smem);
        if (e != cudaSuccess) return e;
        best = b < best ? b : best;
    }
    *blocks_per_sm = best;
    return cudaSuccess;
}

cudaError_t launch_split_df32(const SwrDeviceView& v, cudaStream_t st, int max_K, bool make_w) {
    long long kk = (long long)max_K * df32_ld(max_K);
    unsigned gx = (unsigned)((kk + 256 * 8 - 1) / (256 * 8));
    k_split_df32<<<dim3(gx, v.n_sub), 256, 0, st>>>(v);
    if (!make_w) return cudaGetLastError();
    size_t sm = ((size_t)max_K + 32 * 32) * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_make_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_make_w<<<dim3(max_K < 512 ? max_K : 512, v.n_sub), 256, sm, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_window(SweepArgs& a, int grid, size_t smem, cudaStream_t st, int n_inst, int variant, bool df32,
                          bool onep, cudaEvent_t ev_begin, cudaEvent_t ev_end) {
    k_window_reset<<<1, 32, 0, st>>>(a, n_inst);
    cudaError_t e = record_event(ev_begin, st);
    if (e != cudaSuccess) return e;
    if (variant == WIN_CLUSTER) {
        e = launch_cluster_window(a, grid, a.cl_size, smem, st, onep);
    } else {
        void* params[] = {&a};
        e = cudaLaunchCooperativeKernel(window_kernel(variant, df32, onep), dim3(grid), dim3(WIN_THREADS), params,
                                        smem, st);
    }
    if (e != cudaSuccess) return e;
    return record_event(ev_end, st);
}

}  // namespace swr
