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
// One persistent cooperative launch runs the whole window.  Work unit: a task
// = a block of rows of one subdomain's G; tasks are sized so that every SM
// gets the same number of rows.  Per step, two bounded grid barriers:
//   phase A(n+1): s_n from the per-task partials (deterministic order), the
//                 partial of delta_n^2 from rows this task owns, then the
//                 rows of y^{n+1} = G v (v = y^n/s_n + kappa dt b');
//   phase B(n+1): stop decisions, z^{n+1} rows = (Pp (x) Pp) y^{n+1} by the
//                 Kronecker form, and the partial of s_{n+1}^2.
// Each phase costs one dependent round trip to L2; the task's own rows of
// y^n, y^{n-1}, z^n, z^{n-1} stay in a per-task ring that only this CTA
// touches.
//
// Precision: FP64 (DFMA), or "double-single" (SWR_PREC_MIXED): G is stored
// as FP32 pairs G = G_hi + G_lo and v = v_hi + v_lo; the products run on the
// FP32 pipes with error-free TwoProduct/TwoSum accumulation into a
// (hi, lo) pair, which keeps the FP64 accuracy of the step (error ~1e-14)
// while using the FP32 units (64x the FP64 rate on GB300).
#include <math.h>

#include "swr_internal.cuh"

namespace swr {

#define WIN_THREADS 256

__device__ inline unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Monotone-counter grid barrier: the m-th barrier of a launch completes when
// the counter reaches m * gridDim.x.  At most `limit` polls, then error.
__device__ inline bool grid_barrier_mono(unsigned* count, unsigned target, int* err, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        long long it = 0;
        while (ld_acquire_u32(count) < target) {
            if (++it > limit) { atomicOr(err, SWR_ERR_TIMEOUT); ok = 0; break; }
            if ((it & 255) == 0 && *(volatile int*)err) { ok = 0; break; }
            __nanosleep(20);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

__device__ inline void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// rows [r0, r1) of z = (Pp1 (x) Pp2) y  (N = 2) or Pp1 y (N = 1); y in shared memory
__device__ void z_rows(const SwrDeviceView& v, const SubDev& s, const double* ys, int r0, int r1, double* z,
                       double* tmp) {
    const int kd = s.kd;
    T1Layout lay(s.q, kd);
    const double* P1 = v.arena + s.t1[0] + lay.mat(M_PP);
    if (s.N == 1) {
        for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            double acc = 0;
            for (int c = 0; c < kd; ++c) acc += P1[r * kd + c] * ys[c];
            z[r - r0] = acc;
        }
        __syncthreads();
        return;
    }
    const double* P2 = v.arena + s.t1[1] + lay.mat(M_PP);
    const int b0 = r0 / kd, b1 = (r1 - 1) / kd;
    for (int b = b0; b <= b1; ++b) {
        for (int c = threadIdx.x; c < kd; c += blockDim.x) {
            double acc = 0;
            for (int e = 0; e < kd; ++e) acc += ys[c + kd * e] * P2[b * kd + e];
            tmp[c] = acc;
        }
        __syncthreads();
        int lo = max(r0, b * kd), hi = min(r1, (b + 1) * kd);
        for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
            int a = r - b * kd;
            double acc = 0;
            for (int c = 0; c < kd; ++c) acc += P1[a * kd + c] * tmp[c];
            z[r - r0] = acc;
        }
        __syncthreads();
    }
}

// Dynamic shared memory: vs[Kmax] doubles, vf[Kmax] float2 (mixed only), tmp[kdmax].
template <bool DF32>
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window(SweepArgs A) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ int s_nact;
    const SwrDeviceView& v = A.v;
    const int t_begin = blockIdx.x * A.tasks_per_cta;
    const int t_end = min(A.n_tasks, t_begin + A.tasks_per_cta);
    const int cap = A.cap;
    double* vs = sm;
    float2* vf = (float2*)(sm + A.kmax);
    double* tmp = sm + 2 * A.kmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = WIN_THREADS / 32;
    unsigned target = 0;
    // ---------------------------------------------------------------- step 0
    for (int t = t_begin; t < t_end; ++t) {
        const Task tk = A.tasks[t];
        const SubDev& s = v.sub[tk.sid];
        const int K = s.K, nr = tk.r1 - tk.r0;
        const double* c0 = v.arena + s.c0;
        for (int c = tid; c < K; c += WIN_THREADS) vs[c] = c0[c];
        __syncthreads();
        double* own = A.own + tk.own;  // [4][nr]: y slot 0/1, z slot 0/1
        double* h0 = v.arena + s.hist;
        for (int r = tk.r0 + tid; r < tk.r1; r += WIN_THREADS) {
            h0[r] = vs[r];
            own[r - tk.r0] = vs[r];  // y^0 in slot 0
        }
        z_rows(v, s, vs, tk.r0, tk.r1, own + 2 * nr, tmp);  // z^0 in slot 0
        double acc = 0;
        for (int r = tid; r < nr; r += WIN_THREADS) acc += own[r] * own[2 * nr + r];
        acc = wblock_sum(acc, red);
        if (tid == 0) {
            A.part_s[t] = acc;
            A.alive[t] = 1;
            A.s_prev[t] = 1.0;
        }
    }
    target += gridDim.x;
    if (!grid_barrier_mono(&A.bar->count, target, v.err, A.spin_limit)) return;

    for (int n = 0;; ++n) {
        if (tid == 0) s_nact = __ldcg(A.n_active);
        __syncthreads();
        if (s_nact == 0) return;  // stable here: instances close only in phase B
        // ------------------------------------------------------ phase A(n+1)
        for (int t = t_begin; t < t_end; ++t) {
            if (!A.alive[t]) continue;  // written by this CTA only
            const Task tk = A.tasks[t];
            const SubDev& s = v.sub[tk.sid];
            const InstDev& in = v.inst[tk.inst];
            const int K = s.K, nr = tk.r1 - tk.r0;
            const int t0 = A.inst_task0[tk.inst], t1 = A.inst_task0[tk.inst + 1];
            const int fixed = in.window_cap, maxs = fixed > 0 ? fixed : in.max_steps;
            const bool ngf_stop = fixed == 0 && in.ngf_tol > 0.0;
            // issue the independent loads together: partials of s_n, y^n, b'^{n+1}
            double ps = 0;
            if (in.normalize)
                for (int u = t0 + tid; u < t1; u += WIN_THREADS) ps += __ldcg(A.part_s + (n & 1) * A.n_tasks + u);
            const double* yn = v.arena + s.hist + (long long)n * K;
            const int wp = A.win_prev[tk.inst];
            const double* bsrc = (wp > 0) ? v.arena + s.bvec + (long long)min(n + 1, wp) * K : nullptr;
            double bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int c = tid + i * WIN_THREADS;
                double yv = 0, bb = 0;
                if (c < K) {
                    yv = yn[c];
                    if (bsrc) bb = bsrc[c];
                }
                if (c < K) vs[c] = yv;
                bv[i] = bb;
            }
            const double s_n = in.normalize ? sqrt(wblock_sum(ps, red)) : 1.0;
            const double sp = A.s_prev[t];  // s_{n-1}
            __syncthreads();
            if (tid == 0) {
                A.s_prev[t] = s_n;
                if (t == t0) A.snorm[(long long)tk.inst * (cap + 1) + n] = s_n;
            }
            if (n >= maxs || !isfinite(s_n) || s_n <= 0.0) continue;  // closed in phase B
            const double kdt = in.kappa * in.dt;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int c = tid + i * WIN_THREADS;
                if (c < K) {
                    double val = vs[c] / s_n + kdt * bv[i];
                    vs[c] = val;
                    if (DF32) {
                        float h = (float)val;
                        vf[c] = make_float2(h, (float)(val - (double)h));
                    }
                }
            }
            double* own = A.own + tk.own;
            // partial of delta_n^2 = || y^n/s_n - y^{n-1}/s_{n-1} ||^2_chi over own rows
            if (n >= 1 && ngf_stop) {
                const double* y_n = own + (n & 1) * nr;
                const double* y_p = own + ((n - 1) & 1) * nr;
                const double* z_n = own + (2 + (n & 1)) * nr;
                const double* z_p = own + (2 + ((n - 1) & 1)) * nr;
                double acc = 0;
                for (int r = tid; r < nr; r += WIN_THREADS)
                    acc += (y_n[r] / s_n - y_p[r] / sp) * (z_n[r] / s_n - z_p[r] / sp);
                acc = wblock_sum(acc, red);
                if (tid == 0) A.part_d[(n & 1) * A.n_tasks + t] = acc;
            } else {
                __syncthreads();
            }
            // rows of y^{n+1} = G v
            double* ynew = v.arena + s.hist + (long long)(n + 1) * K;
            double* yslot = own + ((n + 1) & 1) * nr;
            if (DF32) {
                const float* Gh = (const float*)(v.arena + s.Gf);
                const float* Gl = Gh + (long long)K * K;
                for (int r = tk.r0 + warp; r < tk.r1; r += nw) {
                    const float* gh = Gh + (long long)r * K;
                    const float* gl = Gl + (long long)r * K;
                    float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
                    int c = lane;
                    for (; c + 32 < K; c += 64) {
                        float h0 = gh[c], l0 = gl[c], h1 = gh[c + 32], l1 = gl[c + 32];
                        float2 v0 = vf[c], v1 = vf[c + 32];
                        float p0 = h0 * v0.x, e0 = fmaf(h0, v0.x, -p0);
                        float p1 = h1 * v1.x, e1 = fmaf(h1, v1.x, -p1);
                        float s0, q0, s1, q1;
                        two_sum(ah0, p0, s0, q0);
                        two_sum(ah1, p1, s1, q1);
                        ah0 = s0;
                        ah1 = s1;
                        al0 += (q0 + e0) + fmaf(h0, v0.y, l0 * v0.x);
                        al1 += (q1 + e1) + fmaf(h1, v1.y, l1 * v1.x);
                    }
                    if (c < K) {
                        float h0 = gh[c], l0 = gl[c];
                        float2 v0 = vf[c];
                        float p0 = h0 * v0.x, e0 = fmaf(h0, v0.x, -p0);
                        float s0, q0;
                        two_sum(ah0, p0, s0, q0);
                        ah0 = s0;
                        al0 += (q0 + e0) + fmaf(h0, v0.y, l0 * v0.x);
                    }
                    float sh, eh;
                    two_sum(ah0, ah1, sh, eh);
                    float ah = sh, al = al0 + al1 + eh;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float oh = __shfl_xor_sync(0xffffffffu, ah, o);
                        float ol = __shfl_xor_sync(0xffffffffu, al, o);
                        two_sum(ah, oh, sh, eh);
                        ah = sh;
                        al = al + ol + eh;
                    }
                    if (lane == 0) {
                        double y = (double)ah + (double)al;
                        ynew[r] = y;
                        yslot[r - tk.r0] = y;
                    }
                }
            } else {
                const double* G = v.arena + s.Gm;
                for (int r = tk.r0 + warp; r < tk.r1; r += nw) {
                    const double* g = G + (long long)r * K;
                    double a0 = 0, a1 = 0;
                    int c = lane;
                    for (; c + 32 < K; c += 64) {
                        a0 = fma(g[c], vs[c], a0);
                        a1 = fma(g[c + 32], vs[c + 32], a1);
                    }
                    if (c < K) a0 = fma(g[c], vs[c], a0);
                    double y = warp_sum(a0 + a1);
                    if (lane == 0) {
                        ynew[r] = y;
                        yslot[r - tk.r0] = y;
                    }
                }
            }
            __syncthreads();
        }
        target += gridDim.x;
        if (!grid_barrier_mono(&A.bar->count, target, v.err, A.spin_limit)) return;
        // ------------------------------------------------------ phase B(n+1)
        for (int t = t_begin; t < t_end; ++t) {
            if (!A.alive[t]) continue;
            const Task tk = A.tasks[t];
            const SubDev& s = v.sub[tk.sid];
            const InstDev& in = v.inst[tk.inst];
            const int K = s.K, nr = tk.r1 - tk.r0;
            const int t0 = A.inst_task0[tk.inst], t1 = A.inst_task0[tk.inst + 1];
            const int fixed = in.window_cap, maxs = fixed > 0 ? fixed : in.max_steps;
            const bool ngf_stop = fixed == 0 && in.ngf_tol > 0.0;
            const double s_n = A.s_prev[t];
            double pd = 0;
            if (n >= 1 && ngf_stop)
                for (int u = t0 + tid; u < t1; u += WIN_THREADS) pd += __ldcg(A.part_d + (n & 1) * A.n_tasks + u);
            const double* yn1 = v.arena + s.hist + (long long)(n + 1) * K;
            bool early = (n >= maxs) || !isfinite(s_n) || s_n <= 0.0;
            if (!early)
                for (int c = tid; c < K; c += WIN_THREADS) vs[c] = yn1[c];
            bool stop = early;
            if (!stop && n >= 1 && ngf_stop) {
                double d2 = wblock_sum(pd, red);
                stop = sqrt(fmax(d2, 0.0)) <= in.ngf_tol;
            }
            if (stop) {
                if (tid == 0) {
                    A.alive[t] = 0;
                    if (t == t0) {
                        A.win[tk.inst] = n;
                        if (!isfinite(s_n) || s_n <= 0.0) atomicOr(v.err, SWR_ERR_NUMERIC);
                        __threadfence();
                        atomicSub(A.n_active, 1);
                    }
                }
                __syncthreads();
                continue;
            }
            __syncthreads();
            double* own = A.own + tk.own;
            double* zslot = own + (2 + ((n + 1) & 1)) * nr;
            z_rows(v, s, vs, tk.r0, tk.r1, zslot, tmp);
            const double* yslot = own + ((n + 1) & 1) * nr;
            double acc = 0;
            for (int r = tid; r < nr; r += WIN_THREADS) acc += yslot[r] * zslot[r];
            acc = wblock_sum(acc, red);
            if (tid == 0) A.part_s[((n + 1) & 1) * A.n_tasks + t] = acc;
        }
        target += gridDim.x;
        if (!grid_barrier_mono(&A.bar->count, target, v.err, A.spin_limit)) return;
    }
}

__global__ void k_window_reset(SweepArgs A, int n_inst) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.bar->count = 0;
        *A.n_active = n_inst;
    }
}

// Split of the FP64 step-matrix inverse into FP32 pairs (mixed precision).
__global__ void k_split_df32(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const long long KK = (long long)s.K * s.K;
    const double* G = v.arena + s.Gm;
    float* Gh = (float*)(v.arena + s.Gf);
    float* Gl = Gh + KK;
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < KK; e += (long long)blockDim.x * gridDim.x) {
        double g = G[e];
        float h = (float)g;
        Gh[e] = h;
        Gl[e] = (float)(g - (double)h);
    }
}

// ------------------------------------------------------------- host side

size_t window_smem(int kmax, int kdmax) { return (2 * (size_t)kmax + (size_t)kdmax + 8) * sizeof(double); }

cudaError_t window_occupancy(int* blocks_per_sm, size_t smem, bool df32) {
    const void* f = df32 ? (const void*)k_window<true> : (const void*)k_window<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, WIN_THREADS, smem);
}

cudaError_t launch_split_df32(const SwrDeviceView& v, cudaStream_t st, int max_K) {
    long long kk = (long long)max_K * max_K;
    unsigned gx = (unsigned)((kk + 256 * 8 - 1) / (256 * 8));
    k_split_df32<<<dim3(gx, v.n_sub), 256, 0, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_window(SweepArgs& a, int grid, size_t smem, cudaStream_t st, int n_inst, bool df32,
                          cudaEvent_t ev_begin, cudaEvent_t ev_end) {
    k_window_reset<<<1, 32, 0, st>>>(a, n_inst);
    cudaError_t e = cudaEventRecord(ev_begin, st);
    if (e != cudaSuccess) return e;
    void* params[] = {&a};
    const void* f = df32 ? (const void*)k_window<true> : (const void*)k_window<false>;
    e = cudaLaunchCooperativeKernel(f, dim3(grid), dim3(WIN_THREADS), params, smem, st);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(ev_end, st);
}

}  // namespace swr
