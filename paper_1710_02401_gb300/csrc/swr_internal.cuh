// swr_internal.cuh -- device-side data layout and helpers shared by the CUDA
// translation units of the SWR-Galerkin library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swr.h"

#define SWR_MAX_NUC 3
#define SWR_MAX_QP 64
#define SWR_NLINE_KINDS 16   // 2 coordinates x 4 lines x {value, derivative}

// Complex number in FP64 (real-time path); a plain aggregate so that it can
// live in __shared__ memory.
struct cplx {
    double re, im;
};
__host__ __device__ inline cplx mkc(double r, double i = 0.0) { cplx z; z.re = r; z.im = i; return z; }
__host__ __device__ inline cplx operator+(cplx a, cplx b) { return mkc(a.re + b.re, a.im + b.im); }
__host__ __device__ inline cplx operator-(cplx a, cplx b) { return mkc(a.re - b.re, a.im - b.im); }
__host__ __device__ inline cplx operator*(cplx a, cplx b) {
    return mkc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__host__ __device__ inline cplx operator*(double s, cplx a) { return mkc(s * a.re, s * a.im); }
__host__ __device__ inline cplx conj(cplx a) { return mkc(a.re, -a.im); }

// Per-instance constants (device copy).
struct InstDev {
    int N, L, kd_uniform, q_p, n_mid, q, mode, normalize, n_nuc;
    int sub_base, n_sub;          // first global subdomain index, count
    int n_steps, max_steps, window_cap;
    double a, b, H, eps;
    double x_nuc[SWR_MAX_NUC], Z_nuc[SWR_MAX_NUC];
    double eta_en, eta_ee, ee_coef, harmonic, kappa;
    double mu_re, mu_im, dt, ngf_tol;
    double E0, T, omega, phase;
    double gamma0, x0[2];
    double orth_tau;              // Cholesky acceptance / canonical cut-off of the 1-D overlaps
    int tc;                       // transmission condition (swr_tc)
    int anti;                     // antisymmetric states: steps act on the antisymmetric part (swr_symmetry)
};

// Per-subdomain descriptor.  Offsets are in doubles from the arena base.
struct SubDev {
    int inst, N, kd, K, q, ngam;
    int idx[2];                   // 1-D subdomain indices (i1, i2)
    int edge_mask;                // bit 2*d+side: edge (coordinate d, side lo=0/hi=1) is interior
    int gam_off[4];               // first Gamma node of edge slot 2*d+side (-1 when absent)
    double lo[2], hi[2], delta;
    long long t1[2];              // 1-D table block of coordinate d
    long long Hm;                 // K*K  H' (real part), orthonormal basis
    long long Gm;                 // K*K step-matrix inverse (x2 doubles when complex)
    long long c0;                 // initial coefficients (K, x2 when complex)
    long long hist;               // (cap+1)*K iterates before normalisation (x2 complex)
    long long bvec;               // (cap+1)*K Robin source b' per step (x2 complex)
    long long line;               // (cap+1)*nline line traces (x2 complex)
    long long u[2];               // (cap+1)*ngam own traces, two iteration parities (x2 complex)
    long long g;                  // (cap+1)*ngam averaged Robin data (x2 complex)
    long long work;               // scratch for assembly (see swr_assemble.cu)
    long long Gf;                 // mixed precision: G as FP32 pairs (G_hi [K*K] then G_lo [K*K])
    long long Wf;                 // mixed precision: W = (Pp (x) Pp) G as FP32 pairs
    long long GE;                 // Robin response (swr_robin.cu): G times the edge-load columns, K x J pairs
    long long Hr;                 // Robin response: (cap+1) x J tangential sums of b' per step (pairs)
    long long Wr;                 // Robin response: (cap+1) x df32_ld(K) pairs, w^n = kappa dt G b'^n
    int nline;                    // values per step in `line`
};

// 1-D table layout for one coordinate of one subdomain (offsets in doubles).
struct T1Layout {
    int q, kd;
    __host__ __device__ T1Layout(int q_, int kd_) : q(q_), kd(kd_) {}
    __host__ __device__ long long x() const { return 0; }
    __host__ __device__ long long w() const { return q; }
    __host__ __device__ long long chi() const { return 2LL * q; }
    __host__ __device__ long long v1() const { return 3LL * q; }          // 1-D external potential
    __host__ __device__ long long alpha() const { return 4LL * q; }       // centres [kd]
    __host__ __device__ long long B() const { return 4LL * q + kd; }      // [q][kd] values (-> orthonormal)
    __host__ __device__ long long D() const { return B() + (long long)q * kd; }  // [q][kd] derivatives
    __host__ __device__ long long Lv() const { return D() + (long long)q * kd; } // [4][kd] line values
    __host__ __device__ long long Ld() const { return Lv() + 4LL * kd; }         // [4][kd] line derivatives
    __host__ __device__ long long mat(int i) const { return Ld() + 4LL * kd + (long long)i * kd * kd; }
    // matrices: 0 S, 1 Kf, 2 Xpos, 3 U, 4 Schi, 5 Xo (orth transform), 6 Tp, 7 Up, 8 Pp, 9 Xp', 10 Rp
    __host__ __device__ long long size() const { return mat(11); }
};
enum { M_S = 0, M_KF, M_XPOS, M_U, M_SCHI, M_XO, M_TP, M_UP, M_PP, M_XP, M_RP };

// Line positions of a subdomain interval: lo, lo+eps, hi-eps, hi.
__host__ __device__ inline double line_pos(double lo, double hi, double eps, int l) {
    return l == 0 ? lo : (l == 1 ? lo + eps : (l == 2 ? hi - eps : hi));
}

// ---------------------------------------------------------------- errors
#define SWR_ERR_TIMEOUT 1
#define SWR_ERR_NUMERIC 2
#define SWR_ERR_SINGULAR 4

// Bounded sense-reversal grid barrier for a cooperative launch.  Spins at most
// `limit` polls; on timeout it raises SWR_ERR_TIMEOUT in *err and returns false.
// Arrival counter and release word on separate 128-byte lines: the CTAs that
// poll the release word do not contend with the arrivals' atomics.
struct GridBarrier {
    unsigned int count;
    unsigned int pad0[31];
    unsigned int gen;
    unsigned int pad1[31];
};

// Work queue of the split window, by step parity p: list[p] holds the tasks
// still stepping at a step of parity p (appended during the step before),
// count[p] its length, claim[p] the next list position to hand out.
struct SplitQueue {
    unsigned int claim[2];
    unsigned int pad0[30];
    unsigned int count[2];
    unsigned int pad1[30];
};

__device__ inline bool grid_sync_bounded(GridBarrier* bar, unsigned int nblocks, int* err,
                                         long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &bar->gen;
        unsigned int g = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (++it > limit) { atomicOr(err, SWR_ERR_TIMEOUT); ok = 0; break; }
                if ((it & 63) == 0 && *(volatile int*)err) { ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int*)err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Warp reduction.
// Double-single arithmetic (FP32 pairs carrying FP64-level accuracy on the
// FP32 pipes): split of a double, and (h, l) += a b with TwoProduct of the
// leading terms, TwoSum into (h, l) and the cross terms into l.
__device__ inline float2 ds_split(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
__device__ inline void ds_fma(float& h, float& l, float2 a, float2 b) {
    const float p = a.x * b.x, e = fmaf(a.x, b.x, -p);
    const float sm = h + p, bb = sm - h, err = (h - (sm - bb)) + (p - bb);
    h = sm;
    l += (err + e) + fmaf(a.x, b.y, a.y * b.x);
}

// Double-single pairs (h, l) as float2 on the FP32 pipes: error-free sum and
// product of the leading terms, renormalised results.
__device__ inline void dsp_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ inline float2 dsp_norm(float h, float l) {
    const float s = h + l;
    return make_float2(s, l - (s - h));
}
__device__ inline float2 dsp_add(float2 a, float2 b) {
    float s, e;
    dsp_two_sum(a.x, b.x, s, e);
    return dsp_norm(s, e + (a.y + b.y));
}
__device__ inline float2 dsp_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return dsp_norm(p, e);
}
__device__ inline float2 dsp_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ inline float2 dsp_shfl_add(float2 a, int o) {
    return dsp_add(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
}
__device__ inline double dsp_to_double(float2 a) { return (double)a.x + (double)a.y; }

// Split of a double into a double-single pair on the integer pipes: hi = x
// truncated to 24 significant bits, lo = the remainder truncated to 24 bits,
// |x - hi - lo| <= 2^-46 |x|.  |x| < 2^-100 gives (0, 0); NaN, infinities and
// |x| >= 2^128 take the FP64 conversion (and propagate).
__device__ inline float2 dsp_split_int(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ffULL) - 1023;
    if (e < -100) return make_float2(0.f, 0.f);
    if (e > 127) return make_float2((float)x, 0.f);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const unsigned long long mant = u & 0xFFFFFFFFFFFFFULL;
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
    const unsigned long long r = mant & 0x1FFFFFFFULL;  // the 29 bits below hi
    float lo = 0.f;
    if (r != 0) {
        const int p = 63 - __clzll((long long)r);  // leading bit of r, 0..28
        const int le = e - 52 + p;                 // its binary exponent
        if (le >= -126) {
            const unsigned m = p >= 23 ? (unsigned)(r >> (p - 23)) : (unsigned)(r << (23 - p));
            lo = __uint_as_float(sign | ((unsigned)(le + 127) << 23) | (m & 0x7FFFFFu));
        }
    }
    return make_float2(hi, lo);
}

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Host-side launch helpers implemented in swr_assemble.cu / swr_sweep.cu.
struct SwrDeviceView {
    double* arena;
    const InstDev* inst;
    const SubDev* sub;
    int n_inst, n_sub;
    int* err;                     // device error flags
};

namespace swr {
// Batched FP64 GEMM job (one per subdomain): C = op(A) * B.
struct GemmJob {
    long long a, b, c;   // offsets (doubles) into the arena
    int M, N, K;         // C is M x N
    int lda, ldb, ldc;
    int transA;          // op(A) = A^T when set (A stored K x M)
    int mode;            // 0: C = AB;  1: scatter the e-e block into H' (index permutation)
    int kd;              // for mode 1
};

// Row block [r0, r1) of the step matrix of subdomain sid (persistent task).
struct Task {
    int sid, r0, r1, inst;
    long long own;              // offset of the task's ring [6][r1-r0] in SweepArgs::g_own
};

// Leading dimension of the real step matrix's FP32 planes (mixed precision):
// K rounded up to 4 columns, zero-padded, so that every row starts on 16 bytes.
__host__ __device__ inline int df32_ld(int K) { return (K + 3) & ~3; }

// Constants of one row task, gathered once per window.
struct TaskCache {
    int inst, sid, r0, nr, K, kd, N, t0, first, maxs, ngf_stop, normalize;
    long long hist, bvec, Gm, Gf, Wf, c0, p1, p2, own;
    double kdt, ngf_tol;
};

// Window kernel variants.
enum WindowVariant { WIN_TWO_PHASE = 1, WIN_FUSED = 2, WIN_SPLIT = 3, WIN_RESIDENT = 4, WIN_CLUSTER = 5 };

// Event record that becomes an event-record node of the graph under stream
// capture (external record) and is a plain record otherwise.
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

struct SweepArgs {
    SwrDeviceView v;
    const Task* tasks;
    const int* cta_task0;       // [grid+1] first position of each CTA in cta_list
    const int* cta_list;        // [n_tasks] task indices, CTA by CTA (cost-balanced, instances spread)
    int n_tasks, tasks_per_cta, kmax, kdmax, rows_max;
    int many;                   // per-task state in global memory (more tasks per CTA than shared memory holds)
    int tune_steps;             // > 0: fixed window of this many steps without the NGF stop (timing runs)
    TaskCache* g_tc;            // [n_tasks] by position in cta_list (many)
    double* scal_inst;          // [2][2][n_inst] s_n and 1/s_n per instance, by step parity (two-phase)
    int* g_alive;               // [n_tasks] by position (many)
    double* g_own;              // [sum of 6 x task rows] (many)
    int g_resident;             // mixed precision: G_hi rows of the CTA's task kept in shared memory
    int any_ngf_stop;           // some instance stops its window on ||c^{n+1} - c^n||
    const int* inst_task0;      // [n_inst+1] first task of each instance
    double* part_s;             // [n_tasks] partials of s^2
    double* part_d;             // [n_tasks] partials of delta^2
    double* sums_s;             // [n_inst] s^2 per instance (reduced at the grid barrier)
    double* sums_d;             // [n_inst] delta^2 per instance
    double* snorm;              // [n_inst][cap+1] normalisation factors s_n
    int* n_active;              // instances still stepping
    int* win;                   // [n_inst] window length of this iteration
    const int* win_prev;        // [n_inst] window of the previous iteration (0: none)
    int cap;                    // max window stored
    GridBarrier* bar;
    long long spin_limit;
    int stage_floats;           // split window: floats per stage of staged step-matrix rows (both planes)
    int n_stages;               // split window: stages in the ring (2..8)
    SplitQueue* q;              // split window: work queue counters
    int* q_list;                // split window: [2][n_tasks] task lists by step parity
    unsigned long long* cl_slots;  // cluster window: [2][n_tasks][4] tagged partials (step parity, task)
    int tmem_cols;              // cluster window: tensor-memory columns per CTA (power of two, 0: none)
    int cl_size;                // cluster window: CTAs per cluster (one subdomain each)
    int cl_hs;                  // cluster window: G_hi elements per thread in shared memory (rest: tensor memory)
    int robin_w;                // the Robin response w^n = kappa dt G b'^n is precomputed (split window: one product)
};

// Constants of task t, gathered once per window.
__device__ inline TaskCache make_task_cache(const SweepArgs& A, int t) {
    const Task tk = A.tasks[t];
    const SubDev& s = A.v.sub[tk.sid];
    const InstDev& in = A.v.inst[tk.inst];
    TaskCache c;
    c.inst = tk.inst;
    c.sid = tk.sid;
    c.r0 = tk.r0;
    c.nr = tk.r1 - tk.r0;
    c.K = s.K;
    c.kd = s.kd;
    c.N = s.N;
    c.t0 = A.inst_task0[tk.inst];
    c.first = (t == c.t0);
    c.maxs = in.window_cap > 0 ? in.window_cap : in.max_steps;
    c.ngf_stop = (in.window_cap == 0 && in.ngf_tol > 0.0);
    if (A.tune_steps > 0) {
        c.maxs = min(c.maxs, A.tune_steps);
        c.ngf_stop = 0;
    }
    c.normalize = in.normalize;
    c.hist = s.hist;
    c.bvec = s.bvec;
    c.Gm = s.Gm;
    c.Gf = s.Gf;
    c.Wf = s.Wf;
    c.c0 = s.c0;
    T1Layout lay(s.q, s.kd);
    c.p1 = s.t1[0] + lay.mat(M_PP);
    c.p2 = s.t1[s.N == 2 ? 1 : 0] + lay.mat(M_PP);
    c.own = tk.own;
    c.kdt = in.kappa * in.dt;
    c.ngf_tol = in.ngf_tol;
    return c;
}

// What the allocation-free residual entry point needs from a context.
struct ResidualInputs {
    SwrDeviceView v;
    cudaStream_t stream;
    int k, parity_last, n_inst, n_sub;
    const int* win_last;   // host, windows of the last iteration
    const int* win_before; // host, windows of the iteration before it
};
bool residual_inputs(swr_ctx* c, ResidualInputs* r);
// Cluster window (swr_cluster.cu): dynamic shared memory, tensor-memory
// columns per CTA (0: does not fit), clusters of cs CTAs the device holds at
// once, and the launch.
size_t window_smem_cluster(int kmax, int kdmax, int rows_max, int hs);
int cluster_hi_smem(int kmax, int kdmax, int rows_max);
int cluster_tmem_cols(int kmax, int rows_max, int hs);
cudaError_t cluster_occupancy(int* clusters, int rows_max, size_t smem, int cs, int grid);
cudaError_t launch_cluster_window(SweepArgs& a, int grid, int cs, size_t smem, cudaStream_t st, bool onep);
// Robin response w^n = kappa dt G b'^n (swr_robin.cu): columns of GE per
// subdomain, GE at assembly, H and W before each cluster window.
int robin_columns(const SubDev& s);
cudaError_t launch_robin_ge(const SwrDeviceView& v, cudaStream_t st, int max_K, int max_J);
cudaError_t launch_robin_w(const SwrDeviceView& v, cudaStream_t st, const int* d_win_prev, int kd2, int nsm,
                           int* d_tiles);
void set_error(swr_ctx* c, const char* msg);
void set_setup_error(const char* msg);
// Blocks per subdomain of the energy kernel (partials [n_sub][ENERGY_BLOCKS][3]).
#define ENERGY_BLOCKS 16
cudaError_t launch_residual(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const int* d_win_prev,
                            int parity, int first_iter, double* d_part, int res_blocks, double* d_res);
}  // namespace swr
