// swr_api.cu -- host side of the C ABI declared in include/swr.h.
//
// Owns the context: validated copy of the problem, the subdomain descriptors,
// the device arena (one allocation, or the caller's workspace), and the order
// of launches of an assembly (swr_assemble) and of a Schwarz iteration
// (swr_step).  Geometry follows the opening of Sec. 6 of the paper: subdomain
// i_e of coordinate e covers [a + i_e H - eps/2, a + (i_e + 1) H + eps/2].
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <queue>
#include <vector>

#include "swr_internal.cuh"

namespace swr {
struct TgState;
cudaError_t launch_assemble(const SwrDeviceView& v, cudaStream_t st, int max_q, int max_kd, int max_K,
                            bool any_ee, bool any_tdse, bool any_tise, const GemmJob* d_jobs1,
                            const GemmJob* d_jobs2, double* d_norm_part, const TgState* tg);
size_t tg_scratch_bytes(const int* Ks, const int* qs, const int* kds, const int* nel, int n_sub, bool cplx_data,
                        bool any_ee);
cudaError_t tg_setup(TgState** out, void* base, const int* Ks, const int* qs, const int* kds, const int* nel, int n_sub,
                     bool cplx_data, bool any_ee, cudaStream_t st);
void tg_release(TgState* g);
size_t window_smem(int kmax, int kdmax, int rows_max, int tasks_in_smem, long long g_resident_floats);
size_t window_smem_split(int kmax, int kdmax, int rows_max, int stage_floats, int n_stages);
size_t window_smem_resident(int kmax, int kdmax, int rows_max, int tasks_in_smem, long long g_resident_floats);
int window_tasks_per_cta_max();
int window_rows_per_task_max();
cudaError_t window_occupancy(int* blocks_per_sm, size_t smem, int variant, bool df32);
cudaError_t launch_split_df32(const SwrDeviceView& v, cudaStream_t st, int max_K, bool make_w);
cudaError_t launch_window(SweepArgs& a, int grid, size_t smem, cudaStream_t st, int n_inst, int variant, bool df32,
                          bool onep, cudaEvent_t ev_begin, cudaEvent_t ev_end);
extern const int kAssembleLaunchesFixed, kStepLaunches;
cudaError_t launch_post(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const int* d_win_prev,
                        const double* d_snorm, int cap, int parity, int first_iter, double* d_res_part,
                        int res_blocks, double* d_res, int max_cap_hint, int lt_kmax, int lt_kdmax, int lt_qmax,
                        bool any_anti, double* d_cv_part, double* d_cvtot, bool with_cvtot);
size_t cvtot_part_doubles(int n_inst);
cudaError_t launch_cvtot(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const double* d_snorm, int cap,
                         double* d_cv_part, double* d_cvtot);
cudaError_t launch_energy(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const double* d_snorm,
                          int cap, double* d_part, double* d_energy, double* d_norm2, double* d_dipole,
                          double* psi_out, const long long* psi_off, size_t smem);
size_t energy_smem(const SubDev& s);
cudaError_t launch_tdse_window(const SwrDeviceView& v, cudaStream_t st, const long long* d_boff, const int* d_win_prev,
                               int n_steps, const unsigned char* h_need, const unsigned char* d_need, int max_K,
                               int max_kd, bool df32, bool onep, long long* launches);
cudaError_t launch_split_c_df32(const SwrDeviceView& v, cudaStream_t st, int max_K);
}  // namespace swr

using namespace swr;

static const int GJ_NB_HOST = 32;     // Gauss-Jordan block (matches swr_assemble.cu)
static const int RES_BLOCKS = 32;     // residual partial blocks per subdomain
static const double ORTH_TAU_DEFAULT = 1e-12;  // basis reduction threshold when an instance gives 0
static const long long SPIN_LIMIT = 1LL << 24;  // default polls (x ~64 ns) before a device-side wait gives up

struct swr_ctx {
    std::string err;
    swr_problem prob;
    std::vector<swr_instance> inst_h;
    std::vector<std::vector<int>> kd_h;
    std::vector<std::vector<double>> delta_h;
    std::vector<InstDev> inst;
    std::vector<SubDev> sub;
    std::vector<long long> psi_off;
    std::vector<Task> tasks;
    std::vector<int> inst_task0;
    size_t arena_doubles = 0, aux_bytes = 0;
    int cap = 0, max_K = 0, max_kd = 0, max_q = 0, max_ngam = 0;
    bool any_ee = false, tdse = false;
    long long psi_total = 0, own_total = 0;
    bool df32 = false, g_resident = false, any_ngf_stop = false, any_anti = false;
    int stage_floats = 0;           // split window: floats per stage of staged rows
    size_t energy_smem = 0;         // dynamic shared memory of the energy / node-value kernel
    int n_stages = 0;               // split window: stages in the ring
    int cl_size = 0, tmem_cols = 0; // cluster window: CTAs per cluster, tensor-memory columns per CTA
    unsigned long long* d_clslots = nullptr;  // cluster window: tagged partials [2][tasks][4]
    int cl_hs = 0;                  // cluster window: G_hi elements per thread in shared memory
    int cn_iters = 0;
    std::vector<long long> boff;  // real time: per subdomain r, u, x work vectors
    long long* d_boff = nullptr;
    std::vector<unsigned char> cn_need;  // real time: fixed-point iterations [step][subdomain]
    std::vector<double> cn_sweeps;       // real time: matvecs with G0 per subdomain over the whole window
    unsigned char* d_cn_need = nullptr;
    int* d_rtiles = nullptr;        // Robin response: first product tile of every subdomain
    double* d_dipole = nullptr;
    std::vector<double> dipole_h;
    int nsm = 0, bps = 0, tasks_per_cta = 1, max_rows = 0;
    // window plan: kernel variant, row-task target, CTA ranges, task state in global memory
    int variant = WIN_TWO_PHASE, rows_target = 0, many = 0;
    bool has_w = false;             // W = (Pp (x) Pp) G allocated (fused variant possible)
    bool robin_w = false;           // Robin response GE, H, W allocated (cluster window possible)
    int max_J = 0;                  // Robin response: largest column count of GE
    std::vector<int> cta_task0, cta_list;
    long long tasks_cap = 0;        // capacity of the task arrays (row target 8)
    int *d_cta_task0 = nullptr, *d_cta_list = nullptr;
    // launch of one Schwarz iteration: a CUDA graph per (parity, first iteration), captured once
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2][2][2] = {};     // [parity][first iteration][FP32 matrices]
    long long g_win_launches[2][2][2] = {};
    bool graph_failed = false;
    int* d_wfix = nullptr;          // real time: the fixed window of every instance
    TaskCache* d_tc = nullptr;
    double *d_scal = nullptr, *d_own = nullptr;
    int* d_alive = nullptr;
    // device memory
    void* base = nullptr;
    bool owns = false;
    double* arena = nullptr;
    InstDev* d_inst = nullptr;
    SubDev* d_sub = nullptr;
    int* d_err = nullptr;
    GemmJob *d_jobs1 = nullptr, *d_jobs2 = nullptr;
    double* d_norm_part = nullptr;
    Task* d_tasks = nullptr;
    int* d_inst_task0 = nullptr;
    double *d_part_s = nullptr, *d_part_d = nullptr, *d_snorm = nullptr, *d_sums_s = nullptr, *d_sums_d = nullptr;
    int *d_n_active = nullptr, *d_win = nullptr, *d_win_prev = nullptr;
    GridBarrier* d_bar = nullptr;
    SplitQueue* d_queue = nullptr;
    int* d_qlist = nullptr;
    double *d_res_part = nullptr, *d_res = nullptr, *d_epart = nullptr, *d_energy = nullptr, *d_norm2 = nullptr;
    double *d_cv_part = nullptr, *d_cvtot = nullptr;
    bool cvtot_valid = false;     // cvtot_h holds the CVTOT of the last iteration
    double* d_psi = nullptr;
    long long* d_psi_off = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // state
    bool assembled = false;
    int k = 0, parity = 0;
    bool step_done = false;       // a swr_step has completed since the last assembly or trace restore
    bool use_tg = false;          // Gauss-Jordan trailing updates on the tensor cores
    TgState* tg = nullptr;
    void* d_tg = nullptr;
    bool refined = false;         // SWR_PREC_FP32_REFINED: switched to the double-single step matrices
    double res_peak = 0.0, res_last = 0.0;  // largest and last Res(k) seen in the FP32 phase
    double iterate_tol = 0.0;     // tolerance of the running swr_iterate (0 outside it)
    long long spin_limit = SPIN_LIMIT;
    int grid = 0;
    size_t win_smem = 0;
    std::vector<double> res_h, energy_h, norm2_h, cvtot_h;
    std::vector<int> win_h, win_prev_h;
    std::vector<int> win_pp_h;  // windows of the iteration before the last one
    // counters (see SWR_FIELD_COUNTERS)
    double counters[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaEvent_t evw0 = nullptr, evw1 = nullptr;
};

static std::string g_setup_err;

// Error text of calls without a context (swr_last_error(NULL)).
namespace swr {
void set_setup_error(const char* msg) { g_setup_err = msg; }
}  // namespace swr

// SWR_PREC_FP32_REFINED before its switch: the windows read only the hi plane
// of the step matrices (the FP32-rounded G).
static bool fp32_phase(const swr_ctx* c) { return c->prob.precision == SWR_PREC_FP32_REFINED && !c->refined; }

static swr_status fail(swr_ctx* c, swr_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_setup_err = buf;
    return s;
}

#define CU(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(c, SWR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                        __FILE__, __LINE__);                                                        \
    } while (0)

static long long align32(long long x) { return (x + 31) & ~31LL; }

// Bound of the contraction of the Crank-Nicolson fixed point x <- G0 (r - i theta Q' x):
// ||G0|| <= 1 and ||Q'|| <= max over the domain of |x_1 + ... + x_N|.
static double cn_contraction(const swr_instance& in) {
    double xm = fmax(fabs(in.box_lo - 0.5 * in.overlap), fabs(in.box_hi + 0.5 * in.overlap));
    return 0.5 * in.dt * fabs(in.field_E0) * in.n_elec * xm;
}

// Fixed-point iterations after x0 = G0 r so that rho^(m+1) <= 1e-15: the
// remainder then stays below the rounding of the double-single (and FP64)
// products of a sweep, ~2^-48 relative, and below 1e-12 over a 1000-step window.
static int cn_iterations_rho(double rho) {
    if (!(rho > 0.0)) return 0;
    int m = (int)ceil(log(1e-15) / log(rho)) - 1;
    return m < 0 ? 0 : m;
}
static int cn_iterations(const swr_instance& in) { return cn_iterations_rho(cn_contraction(in)); }

// Length-gauge field e(t) (Sec. 1.2), as the device evaluates it.
static double cn_field(const swr_instance& in, double t) {
    if (in.field_E0 == 0.0 || t < 0.0 || t > in.field_T) return 0.0;
    const double sn = sin(M_PI * t / in.field_T);
    return in.field_E0 * sn * sn * sin(in.field_omega * t + in.field_phase);
}

// Fixed-point iterations of step n in subdomain s: the contraction there is
// at most |theta_{n+1}| ||Q'_s|| (||G0|| <= 1) with theta = dt/2 e(t_{n+1}) and
// ||Q'_s|| <= max over the subdomain box of |x_1 + ... + x_N| (Q' is the
// Galerkin matrix of x_1 + ... + x_N in a basis orthonormal on the box), so
// the same rho^(m+1) <= 1e-15 holds with far fewer iterations where the pulse
// is weak or the subdomain lies near x_1 + ... + x_N = 0; capped by the
// a-priori count of the instance.
static void plan_cn_iterations(swr_ctx* c, int nmax) {
    const size_t ns = c->sub.size();
    c->cn_need.assign((size_t)nmax * ns, 0);
    c->cn_sweeps.assign(ns, 0.0);
    for (size_t sid = 0; sid < ns; ++sid) {
        const SubDev& sd = c->sub[sid];
        const swr_instance& in = c->inst_h[sd.inst];
        if (in.mode != SWR_MODE_TDSE) continue;
        double lo = 0, hi = 0;
        for (int e = 0; e < sd.N; ++e) {
            lo += sd.lo[e];
            hi += sd.hi[e];
        }
        const double qn = fmax(fabs(lo), fabs(hi));
        const int cap_m = cn_iterations(in);
        for (int n = 0; n < in.n_steps && n < nmax; ++n) {
            const double th = 0.5 * in.dt * fabs(cn_field(in, (n + 1) * in.dt));
            int m = cn_iterations_rho(th * qn);
            m = m > cap_m ? cap_m : m;
            c->cn_need[(size_t)n * ns + sid] = (unsigned char)m;
            c->cn_sweeps[sid] += 1.0 + m;
        }
    }
}

// ------------------------------------------------------------------ layout

static swr_status validate(swr_ctx* c, const swr_problem* p) {
    if (!p || p->n_instances < 1 || !p->instances) return fail(c, SWR_EINVAL, "empty problem");
    if (p->spin_limit < 0) return fail(c, SWR_EINVAL, "spin_limit must be >= 0 (0: default)");
    int mode0 = p->instances[0].mode;
    for (int i = 0; i < p->n_instances; ++i) {
        const swr_instance& in = p->instances[i];
        if (in.n_elec < 1 || in.n_elec > 2) return fail(c, SWR_EINVAL, "instance %d: n_elec must be 1 or 2", i);
        if (in.mode != mode0) return fail(c, SWR_EINVAL, "instance %d: all instances must share one mode", i);
        if (in.mode != SWR_MODE_TISE && in.mode != SWR_MODE_TDSE) return fail(c, SWR_EINVAL, "instance %d: bad mode", i);
        if (!(in.box_hi > in.box_lo)) return fail(c, SWR_EINVAL, "instance %d: empty box", i);
        if (in.L < 1 || in.L > 4096) return fail(c, SWR_EINVAL, "instance %d: L out of range", i);
        double H = (in.box_hi - in.box_lo) / in.L;
        if (!(in.overlap > 0) || (in.L > 1 && !(in.overlap < H)))
            return fail(c, SWR_EINVAL, "instance %d: need 0 < overlap < (b-a)/L", i);
        if (in.q_p < 1 || in.q_p > SWR_MAX_QP) return fail(c, SWR_EINVAL, "instance %d: q_p must be in [1,%d]", i, SWR_MAX_QP);
        if (in.n_mid < 1) return fail(c, SWR_EINVAL, "instance %d: n_mid must be >= 1", i);
        int q = (in.n_mid + 2) * in.q_p;
        if (q > 384) return fail(c, SWR_EINVAL, "instance %d: (n_mid+2)*q_p = %d exceeds 384", i, q);
        if (!(in.orth_tau >= 0.0 && in.orth_tau < 1.0))
            return fail(c, SWR_EINVAL, "instance %d: orth_tau must be in [0, 1)", i);
        if (in.tc != SWR_TC_ROBIN && in.tc != SWR_TC_DIRICHLET)
            return fail(c, SWR_EINVAL, "instance %d: unknown transmission condition", i);
        if (in.symmetry != SWR_SYM_NONE && in.symmetry != SWR_SYM_ANTISYMMETRIC)
            return fail(c, SWR_EINVAL, "instance %d: unknown symmetry", i);
        if (in.symmetry == SWR_SYM_ANTISYMMETRIC) {
            if (in.n_elec != 2)
                return fail(c, SWR_EINVAL, "instance %d: antisymmetric states need N = 2", i);
            for (int s = 0; s < in.L * in.L; ++s) {
                const int m = s / in.L + in.L * (s % in.L);
                const int ks = in.K_d_per_sub ? in.K_d_per_sub[s] : in.K_d, km = in.K_d_per_sub ? in.K_d_per_sub[m] : in.K_d;
                const double ds = in.delta_per_sub ? in.delta_per_sub[s] : in.delta;
                const double dm = in.delta_per_sub ? in.delta_per_sub[m] : in.delta;
                if (ks != km || ds != dm)
                    return fail(c, SWR_EINVAL, "instance %d: subdomains %d and %d (mirror images) differ in basis", i, s, m);
            }
            if (p->window_variant == SWR_WINDOW_FUSED)
                return fail(c, SWR_EINVAL, "instance %d: the fused window does not take antisymmetric states", i);
        }
        if (in.n_nuclei < 0 || in.n_nuclei > SWR_MAX_NUC) return fail(c, SWR_EINVAL, "instance %d: at most 3 nuclei", i);
        if (!(in.dt > 0)) return fail(c, SWR_EINVAL, "instance %d: dt must be > 0", i);
        if (in.mode == SWR_MODE_TDSE && in.n_steps < 1) return fail(c, SWR_EINVAL, "instance %d: TDSE needs n_steps >= 1", i);
        if (in.mode == SWR_MODE_TISE && in.ngf_tol <= 0 && in.n_steps < 1)
            return fail(c, SWR_EINVAL, "instance %d: TISE needs ngf_tol > 0 or n_steps >= 1", i);
        if (in.mode == SWR_MODE_TISE && in.ngf_tol > 0 && in.max_steps < 1)
            return fail(c, SWR_EINVAL, "instance %d: max_steps must be >= 1", i);
        if (in.mode == SWR_MODE_TISE && in.mu_im != 0.0)
            return fail(c, SWR_EINVAL, "instance %d: imaginary-time Robin constant must be real", i);
        if (in.mode == SWR_MODE_TDSE) {
            if (in.mu_im > 0.0)
                return fail(c, SWR_EINVAL, "instance %d: real-time Robin constant needs Im(mu) <= 0 (absorbing)", i);
            if (cn_contraction(in) >= 0.5)
                return fail(c, SWR_EINVAL, "instance %d: dt/2 * |E0| * max|x_1+..+x_N| = %g >= 0.5: field too "
                                           "strong for the fixed-point Crank-Nicolson solve", i, cn_contraction(in));
        }
        int nsub = 1;
        for (int e = 0; e < in.n_elec; ++e) nsub *= in.L;
        for (int s = 0; s < nsub; ++s) {
            int kd = in.K_d_per_sub ? in.K_d_per_sub[s] : in.K_d;
            double dl = in.delta_per_sub ? in.delta_per_sub[s] : in.delta;
            if (kd < 2) return fail(c, SWR_EINVAL, "instance %d sub %d: K_d must be >= 2", i, s);
            if (in.n_elec == 2 && kd > 32) return fail(c, SWR_EINVAL, "instance %d sub %d: K_d <= 32 for N = 2", i, s);
            if (in.n_elec == 1 && kd > 96) return fail(c, SWR_EINVAL, "instance %d sub %d: K_d <= 96 for N = 1", i, s);
            if (!(dl > 0)) return fail(c, SWR_EINVAL, "instance %d sub %d: delta must be > 0", i, s);
        }
    }
    if (p->precision != SWR_PREC_FP64 && p->precision != SWR_PREC_MIXED && p->precision != SWR_PREC_FP32_REFINED)
        return fail(c, SWR_EINVAL, "unknown precision");
    if (!(p->refine_res >= 0.0)) return fail(c, SWR_EINVAL, "refine_res must be >= 0 (0: default)");
    if (p->contraction_path < SWR_CONTRACT_AUTO || p->contraction_path > SWR_CONTRACT_TENSOR)
        return fail(c, SWR_EINVAL, "unknown contraction_path");
    if (p->window_variant < 0 || p->window_variant > SWR_WINDOW_CLUSTER)
        return fail(c, SWR_EINVAL, "unknown window variant");
    if (p->window_variant == SWR_WINDOW_CLUSTER && (p->precision == SWR_PREC_FP64 || mode0 != SWR_MODE_TISE))
        return fail(c, SWR_EINVAL, "the cluster window is a mixed-precision imaginary-time kernel");
    if (p->window_variant == SWR_WINDOW_RESIDENT && (p->precision == SWR_PREC_FP64 || mode0 != SWR_MODE_TISE))
        return fail(c, SWR_EINVAL, "the resident window is a mixed-precision imaginary-time kernel");
    if (p->window_variant == SWR_WINDOW_FUSED && (p->precision == SWR_PREC_FP64 || mode0 != SWR_MODE_TISE))
        return fail(c, SWR_EINVAL, "the fused window is the mixed-precision imaginary-time kernel");
    if (p->window_variant == SWR_WINDOW_SPLIT && (p->precision == SWR_PREC_FP64 || mode0 != SWR_MODE_TISE))
        return fail(c, SWR_EINVAL, "the split window is the mixed-precision imaginary-time kernel");
    if (p->window_variant == SWR_WINDOW_TWO_PHASE && p->precision == SWR_PREC_FP32_REFINED)
        return fail(c, SWR_EINVAL, "SWR_PREC_FP32_REFINED runs the fused or the split window");
    if (p->launch_mode != SWR_LAUNCH_GRAPH && p->launch_mode != SWR_LAUNCH_DIRECT)
        return fail(c, SWR_EINVAL, "unknown launch mode");
    if (p->rows_per_task != 0 && (p->rows_per_task < 8 || p->rows_per_task > 256))
        return fail(c, SWR_EINVAL, "rows_per_task must be 0 (automatic) or in [8, 256]");
    return SWR_OK;
}

static const int ROWS_MIN = 8;          // smallest row task
static const int ROWS_MANY_MAX = 256;    // largest row task (task state in global memory)
static const size_t WIN_SMEM_TASKS_MAX = 100 * 1024;  // dynamic shared memory for two CTAs per SM
static const int SPLIT_STAGES = 2;       // split window: stages of staged step-matrix rows in flight per CTA
static const int SPLIT_STAGE_ROWS = 4;   // split window: rows of the widest subdomain per stage (at most)

// Row tasks of the window kernel and their CTA ranges.  Every subdomain's rows
// are cut into equal blocks of about `target_rows` rows (0: total rows over the
// CTAs, at most 64); with `by_bytes`, that is the block of the widest
// subdomain and a narrower subdomain of K rows gets blocks of about
// target_rows x max_K / K rows, so that every task streams about the same bytes
// (the split window hands tasks out dynamically).  The tasks, in instance
// order, are dealt to `ctas` CTAs as contiguous ranges of about equal cost
// (rows x (K + 64) plus a fixed per-task overhead), so that uneven bases load
// the SMs evenly.
static void plan_tasks(swr_ctx* c, int target_rows, int ctas, bool by_bytes = false) {
    c->tasks.clear();
    c->inst_task0.clear();
    c->cta_task0.clear();
    long long rows = 0;
    for (const SubDev& s : c->sub) rows += s.K;
    long long target = target_rows;
    if (target <= 0) {
        target = (rows + ctas - 1) / ctas;
        if (target > window_rows_per_task_max()) target = window_rows_per_task_max();
    }
    if (target < ROWS_MIN) target = ROWS_MIN;
    if (target > ROWS_MANY_MAX) target = ROWS_MANY_MAX;
    c->rows_target = (int)target;
    c->max_rows = 0;
    long long own = 0;
    int cur_inst = -1;
    for (size_t sid = 0; sid < c->sub.size(); ++sid) {
        const SubDev& s = c->sub[sid];
        while (cur_inst < s.inst) {
            c->inst_task0.push_back((int)c->tasks.size());
            ++cur_inst;
        }
        // antisymmetric states: the lower subdomain (i1 > i2) of a mirror pair is
        // not solved, its iterates are the mirror images of the upper one's
        if (c->inst[s.inst].anti && s.N == 2 && s.idx[0] > s.idx[1]) continue;
        long long tgt = target;
        if (by_bytes) {
            tgt = (target * (long long)c->max_K + s.K / 2) / s.K;
            if (tgt > ROWS_MANY_MAX) tgt = ROWS_MANY_MAX;
        }
        int nt = (int)((s.K + tgt - 1) / tgt);
        int per = (s.K + nt - 1) / nt;
        for (int r0 = 0; r0 < s.K; r0 += per) {
            Task t;
            t.sid = (int)sid;
            t.r0 = r0;
            t.r1 = r0 + per < s.K ? r0 + per : s.K;
            t.inst = s.inst;
            t.own = own;
            own += 6LL * (t.r1 - t.r0);
            if (t.r1 - t.r0 > c->max_rows) c->max_rows = t.r1 - t.r0;
            c->tasks.push_back(t);
        }
    }
    while (cur_inst < (int)c->inst.size()) {
        c->inst_task0.push_back((int)c->tasks.size());
        ++cur_inst;
    }
    c->own_total = own;
    // deal the tasks, in instance order, each to the least-loaded CTA (ties: the
    // lowest index): loads end up balanced and every instance's rows spread
    // over the SMs, so the instances whose windows run longest still use the
    // whole GPU after the others have stopped
    const int nt = (int)c->tasks.size();
    const int g = nt < ctas ? nt : ctas;
    typedef std::pair<double, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < g; ++b) heap.push(Load(0.0, b));
    std::vector<std::vector<int>> per(g);
    for (int t = 0; t < nt; ++t) {
        const Task& tk = c->tasks[t];
        const double cost = (double)(tk.r1 - tk.r0) * (c->sub[tk.sid].K + 64) + 16384.0;
        Load l = heap.top();
        heap.pop();
        per[l.second].push_back(t);
        heap.push(Load(l.first + cost, l.second));
    }
    c->grid = g;
    c->cta_task0.assign(1, 0);
    c->cta_list.clear();
    c->tasks_per_cta = 1;
    for (int b = 0; b < g; ++b) {
        c->cta_list.insert(c->cta_list.end(), per[b].begin(), per[b].end());
        c->cta_task0.push_back((int)c->cta_list.size());
        if ((int)per[b].size() > c->tasks_per_cta) c->tasks_per_cta = (int)per[b].size();
    }
}

// Task capacity of the auxiliary arrays: the finest row target.
static long long task_capacity(const swr_ctx* c) {
    long long n = 0;
    for (const SubDev& s : c->sub) n += (s.K + ROWS_MIN - 1) / ROWS_MIN;
    return n;
}

// Window plan for a requested variant (0: automatic) and row target (0:
// automatic): the tasks, whether their state fits shared memory, the dynamic
// shared memory and the CTAs per SM.  Returns false when the request cannot be
// met (fused variant without W, or fused with task state in global memory).
// Cluster window plan: one cluster of cs CTAs (one CTA per SM) per subdomain,
// the rows of each subdomain split evenly over its cluster.  cs is the largest
// size with at most 16 CTAs, at least ROWS_MIN rows per CTA and ns * cs <= SMs
// whose rows fit shared and tensor memory and of which the device holds all ns
// clusters at once (a row request gives cs = ceil(max K / rows)).
static bool plan_cluster(swr_ctx* c, int rows_req, bool have_dev) {
    if (!c->df32 || c->tdse || c->any_anti || !c->robin_w) return false;
    const int nsm = c->nsm > 0 ? c->nsm : 152;
    const int ns = (int)c->sub.size();
    if (ns < 1 || ns > nsm) return false;
    if (nsm > 160) return false;  // the kernel polls at most 160 slots per instance
    int kmin = 1 << 30;
    for (const SubDev& s : c->sub) kmin = s.K < kmin ? s.K : kmin;
    int cs = nsm / ns;
    if (cs > 16) cs = 16;
    if (cs > kmin / ROWS_MIN) cs = kmin / ROWS_MIN;
    if (rows_req > 0) {
        const int want = (c->max_K + rows_req - 1) / rows_req;
        if (want > cs) return false;
        cs = want;
    }
    for (; cs >= 1; --cs) {
        const int rows = (c->max_K + cs - 1) / cs;
        const int hs = cluster_hi_smem(c->max_K, c->max_kd, rows);
        const int cols = cluster_tmem_cols(c->max_K, rows, hs);
        if (cols == 0) return false;  // fewer CTAs per cluster only lengthen the rows
        const size_t smem = window_smem_cluster(c->max_K, c->max_kd, rows, hs);
        if (have_dev) {
            int ncl = 0;
            if (cluster_occupancy(&ncl, rows, smem, cs, ns * cs) != cudaSuccess) {
                cudaGetLastError();
                ncl = 0;
            }
            if (ncl < ns) {
                if (rows_req > 0) return false;
                continue;
            }
        }
        c->tasks.clear();
        c->inst_task0.clear();
        c->cta_task0.assign(1, 0);
        c->cta_list.clear();
        c->max_rows = 0;
        long long own = 0;
        int cur_inst = -1;
        for (size_t sid = 0; sid < c->sub.size(); ++sid) {
            const SubDev& s = c->sub[sid];
            while (cur_inst < s.inst) {
                c->inst_task0.push_back((int)c->tasks.size());
                ++cur_inst;
            }
            for (int j = 0; j < cs; ++j) {
                Task t;
                t.sid = (int)sid;
                t.r0 = (int)((long long)j * s.K / cs);
                t.r1 = (int)((long long)(j + 1) * s.K / cs);
                t.inst = s.inst;
                t.own = own;
                own += 6LL * (t.r1 - t.r0);
                if (t.r1 - t.r0 > c->max_rows) c->max_rows = t.r1 - t.r0;
                c->cta_list.push_back((int)c->tasks.size());
                c->tasks.push_back(t);
                c->cta_task0.push_back((int)c->tasks.size());
            }
        }
        while (cur_inst < (int)c->inst.size()) {
            c->inst_task0.push_back((int)c->tasks.size());
            ++cur_inst;
        }
        c->own_total = own;
        c->grid = (int)c->tasks.size();
        c->tasks_per_cta = 1;
        c->rows_target = c->max_rows;
        c->variant = WIN_CLUSTER;
        c->many = 0;
        c->g_resident = false;
        c->cl_size = cs;
        c->cl_hs = cluster_hi_smem(c->max_K, c->max_kd, c->max_rows);
        c->tmem_cols = cluster_tmem_cols(c->max_K, c->max_rows, c->cl_hs);
        c->win_smem = window_smem_cluster(c->max_K, c->max_kd, c->max_rows, c->cl_hs);
        c->bps = 1;
        return true;
    }
    return false;
}

static bool plan_window(swr_ctx* c, int variant_req, int rows_req, bool have_dev) {
    const int nsm = c->nsm > 0 ? c->nsm : 152;
    if (variant_req == WIN_CLUSTER) return plan_cluster(c, rows_req, have_dev);
    // automatic plan: the cluster window wherever it fits (mixed precision,
    // imaginary time, every subdomain's rows on chip, one resident cluster per
    // subdomain), else the fused, split or two-phase window below
    if (variant_req == 0 && rows_req == 0 && plan_cluster(c, 0, have_dev)) return true;
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
        plan_tasks(c, rows_req, per_sm * nsm, variant_req == WIN_SPLIT);
        if (variant_req == 0 && c->df32 && !c->tdse && !c->has_w) plan_tasks(c, rows_req, per_sm * nsm, true);
        const bool fits = c->tasks_per_cta <= window_tasks_per_cta_max() && c->max_rows <= window_rows_per_task_max() &&
                          window_smem(c->max_K, c->max_kd, c->max_rows, c->tasks_per_cta, 0) <= WIN_SMEM_TASKS_MAX;
        int variant = variant_req;
        if (variant == 0)
            variant = (c->df32 && c->has_w && fits) ? WIN_FUSED : c->df32 && !c->tdse ? WIN_SPLIT : WIN_TWO_PHASE;
        if (variant == WIN_FUSED && (!c->df32 || !c->has_w || !fits)) return false;
        if (variant == WIN_SPLIT && !c->df32) return false;
        if (variant == WIN_RESIDENT && (!c->df32 || c->tdse || c->any_anti || !fits)) return false;
        c->variant = variant;
        c->many = (fits && variant != WIN_SPLIT) ? 0 : 1;  // the split kernel keeps task state in global memory
        const long long gres_floats = (long long)c->max_rows * df32_ld(c->max_K);
        c->g_resident = (variant == WIN_FUSED && c->tasks_per_cta == 1 &&
                         window_smem(c->max_K, c->max_kd, c->max_rows, 1, gres_floats) <= 110 * 1024) ||
                        (variant == WIN_RESIDENT && c->tasks_per_cta == 1 &&
                         window_smem_resident(c->max_K, c->max_kd, c->max_rows, 1, gres_floats) <= 110 * 1024);
        if (variant == WIN_SPLIT) {
            // stages of 4 rows of the widest subdomain (both planes), fewer rows when
            // the shared memory of per_sm CTAs per SM would not hold two of them
            const size_t budget = per_sm == 2 ? 112 * 1024 : 225 * 1024;
            c->n_stages = SPLIT_STAGES;
            for (int rs = SPLIT_STAGE_ROWS; rs >= 1; rs >>= 1) {
                c->stage_floats = 2 * rs * df32_ld(c->max_K);
                if (window_smem_split(c->max_K, c->max_kd, c->max_rows, c->stage_floats, c->n_stages) <= budget) break;
            }
            c->win_smem = window_smem_split(c->max_K, c->max_kd, c->max_rows, c->stage_floats, c->n_stages);
        } else if (variant == WIN_RESIDENT) {
            c->win_smem = window_smem_resident(c->max_K, c->max_kd, c->max_rows, c->tasks_per_cta,
                                               c->g_resident ? gres_floats : 0);
        } else {
            c->win_smem = window_smem(c->max_K, c->max_kd, c->max_rows, c->many ? 1 : c->tasks_per_cta,
                                      c->g_resident ? gres_floats : 0);
        }
        c->bps = per_sm;
        if (!have_dev) return true;
        int bps = 0;
        if (window_occupancy(&bps, c->win_smem, c->variant, c->df32) != cudaSuccess) {
            cudaGetLastError();
            bps = 0;
        }
        if (bps >= per_sm) return true;
        c->bps = bps;
    }
    return true;  // bps < 1 is reported by swr_setup
}

// Fill descriptors and offsets; returns arena size (doubles) and aux bytes.
static void plan(swr_ctx* c) {
    const swr_problem& p = c->prob;
    c->inst.clear();
    c->sub.clear();
    c->psi_off.clear();
    c->boff.clear();
    c->cn_iters = 0;
    for (int i = 0; i < p.n_instances; ++i) {
        int m = cn_iterations(c->inst_h[i]);
        if (c->inst_h[i].mode == SWR_MODE_TDSE && m > c->cn_iters) c->cn_iters = m;
    }
    c->tasks.clear();
    c->inst_task0.clear();
    long long off = 0, po = 0;
    c->cap = 0;
    c->tdse = p.instances[0].mode == SWR_MODE_TDSE;
    const int cx = c->tdse ? 2 : 1;
    for (int i = 0; i < p.n_instances; ++i) {
        const swr_instance& in = c->inst_h[i];
        int fixed = (in.mode == SWR_MODE_TDSE) ? in.n_steps : (in.ngf_tol > 0 ? 0 : in.n_steps);
        int cap = fixed > 0 ? fixed : in.max_steps;
        c->cap = cap > c->cap ? cap : c->cap;
    }
    for (int i = 0; i < p.n_instances; ++i) {
        const swr_instance& in = c->inst_h[i];
        InstDev d;
        memset(&d, 0, sizeof(d));
        d.N = in.n_elec;
        d.L = in.L;
        d.q_p = in.q_p;
        d.n_mid = in.n_mid;
        d.q = (in.n_mid + 2) * in.q_p;
        d.mode = in.mode;
        d.normalize = (in.mode == SWR_MODE_TISE) ? in.normalize : 0;
        d.n_nuc = in.n_nuclei;
        d.sub_base = (int)c->sub.size();
        d.n_sub = 1;
        for (int e = 0; e < in.n_elec; ++e) d.n_sub *= in.L;
        d.n_steps = in.n_steps;
        d.max_steps = in.max_steps;
        d.window_cap = (in.mode == SWR_MODE_TDSE) ? in.n_steps : (in.ngf_tol > 0 ? 0 : in.n_steps);
        d.a = in.box_lo;
        d.b = in.box_hi;
        d.H = (in.box_hi - in.box_lo) / in.L;
        d.eps = in.overlap;
        for (int A = 0; A < in.n_nuclei; ++A) {
            d.x_nuc[A] = in.x_nuc[A];
            d.Z_nuc[A] = in.Z_nuc[A];
        }
        d.eta_en = in.eta_en;
        d.eta_ee = in.eta_ee;
        d.ee_coef = (in.n_elec == 2) ? in.ee_coef : 0.0;
        d.harmonic = in.harmonic;
        d.kappa = in.kinetic;
        d.mu_re = in.mu_re;
        d.tc = in.tc;
        d.anti = in.symmetry == SWR_SYM_ANTISYMMETRIC;
        d.mu_im = in.mu_im;
        d.dt = in.dt;
        d.ngf_tol = in.ngf_tol;
        d.E0 = in.field_E0;
        d.T = in.field_T;
        d.omega = in.field_omega;
        d.phase = in.field_phase;
        d.gamma0 = in.phi0_gamma;
        d.x0[0] = in.phi0_center[0];
        d.x0[1] = in.phi0_center[1];
        d.orth_tau = in.orth_tau > 0.0 ? in.orth_tau : ORTH_TAU_DEFAULT;
        if (d.N == 2 && d.ee_coef != 0.0) c->any_ee = true;
        c->inst.push_back(d);
        c->inst_task0.push_back((int)c->tasks.size());
        for (int sidl = 0; sidl < d.n_sub; ++sidl) {
            SubDev s;
            memset(&s, 0, sizeof(s));
            s.inst = i;
            s.N = d.N;
            s.kd = c->kd_h[i][sidl];
            s.delta = c->delta_h[i][sidl];
            s.K = s.N == 2 ? s.kd * s.kd : s.kd;
            s.q = d.q;
            int rem = sidl;
            for (int e = 0; e < 2; ++e) {
                s.idx[e] = (e < d.N) ? rem % d.L : 0;
                if (e < d.N) rem /= d.L;
                s.lo[e] = d.a + s.idx[e] * d.H - 0.5 * d.eps;
                s.hi[e] = d.a + (s.idx[e] + 1) * d.H + 0.5 * d.eps;
            }
            s.edge_mask = 0;
            int ng = 0;
            for (int sl = 0; sl < 4; ++sl) s.gam_off[sl] = -1;
            for (int e = 0; e < d.N; ++e) {
                for (int side = 0; side < 2; ++side) {
                    bool interior = side == 0 ? s.idx[e] > 0 : s.idx[e] < d.L - 1;
                    if (!interior) continue;
                    s.edge_mask |= 1 << (2 * e + side);
                    s.gam_off[2 * e + side] = ng;
                    ng += (d.N == 2) ? d.q : 1;
                }
            }
            s.ngam = ng;
            s.nline = (d.N == 2) ? 16 * d.q : 8;
            const int K = s.K, q = d.q, kd = s.kd;
            T1Layout lay(q, kd);
            for (int e = 0; e < 2; ++e) {
                if (e < d.N) {
                    s.t1[e] = off;
                    off = align32(off + lay.size());
                } else {
                    s.t1[e] = s.t1[0];
                }
            }
            s.Hm = off; off = align32(off + (long long)K * K);
            s.Gm = off; off = align32(off + (long long)K * K * cx);
            s.c0 = off; off = align32(off + (long long)K * cx);
            s.hist = off; off = align32(off + (long long)(c->cap + 1) * K * cx);
            s.bvec = off; off = align32(off + (long long)(c->cap + 1) * K * cx);
            s.line = off; off = align32(off + (long long)(c->cap + 1) * s.nline * cx);
            s.u[0] = off; off = align32(off + (long long)(c->cap + 1) * (ng > 0 ? ng : 1) * cx);
            s.u[1] = off; off = align32(off + (long long)(c->cap + 1) * (ng > 0 ? ng : 1) * cx);
            s.g = off; off = align32(off + (long long)(c->cap + 1) * (ng > 0 ? ng : 1) * cx);
            long long ee = (d.N == 2) ? 3LL * q * kd * kd + (long long)q * q : 0;
            long long gj = ((long long)GJ_NB_HOST * GJ_NB_HOST + 2LL * GJ_NB_HOST * K) * cx;
            s.work = off; off = align32(off + (ee > gj ? ee : gj));
            if (c->tdse) {
                for (int b3 = 0; b3 < 3; ++b3) {
                    c->boff.push_back(off);
                    off = align32(off + 2LL * K);
                }
            }
            s.Gf = 0;
            s.Wf = 0;
            s.GE = s.Hr = s.Wr = 0;
            c->psi_off.push_back(po);
            po += (d.N == 2) ? (long long)q * q : q;
            if (K > c->max_K) c->max_K = K;
            if (kd > c->max_kd) c->max_kd = kd;
            if (q > c->max_q) c->max_q = q;
            if (ng > c->max_ngam) c->max_ngam = ng;
            c->sub.push_back(s);
        }
    }
    // Mixed precision: FP32 planes of the step matrix, and W = (Pp (x) Pp) G when
    // the fused single-barrier window can run (task state in shared memory).
    c->has_w = false;
    c->any_anti = false;  // antisymmetric states: no fused window
    for (const swr_instance& in : c->inst_h) c->any_anti = c->any_anti || in.symmetry == SWR_SYM_ANTISYMMETRIC;
    if (c->df32 && !c->tdse && !c->any_anti && (p.window_variant == 0 || p.window_variant == WIN_FUSED)) {
        plan_tasks(c, p.rows_per_task, 2 * (c->nsm > 0 ? c->nsm : 152));
        c->has_w = p.window_variant == WIN_FUSED ||
                   (c->tasks_per_cta <= window_tasks_per_cta_max() && c->max_rows <= window_rows_per_task_max() &&
                    window_smem(c->max_K, c->max_kd, c->max_rows, c->tasks_per_cta, 0) <= WIN_SMEM_TASKS_MAX);
    }
    // the Robin response w^n = kappa dt G b'^n of every step (swr_robin.cu),
    // read by the cluster and split windows: mixed precision, imaginary time,
    // no antisymmetric instance
    {
        // (the decomposition kernel stages edge vectors of at most 64 values)
        bool small_kd = true;
        for (const SubDev& s : c->sub) small_kd = small_kd && s.kd <= 64;
        c->robin_w = c->df32 && !c->tdse && !c->any_anti && small_kd && !c->sub.empty() &&
                     (p.window_variant == 0 || p.window_variant == WIN_CLUSTER || p.window_variant == WIN_SPLIT);
    }
    c->max_J = 0;
    for (SubDev& s : c->sub) {
        const long long K = s.K;
        if (c->robin_w) {
            const long long J = robin_columns(s);
            s.GE = off; off = align32(off + K * (J > 0 ? J : 1));
            s.Hr = off; off = align32(off + (long long)(c->cap + 1) * (J > 0 ? J : 1));
            s.Wr = off; off = align32(off + (long long)(c->cap + 1) * df32_ld((int)K));
            if (J > c->max_J) c->max_J = (int)J;
        }
        if (c->df32 && c->tdse) {
            s.Gf = off; off = align32(off + 2LL * K * df32_ld((int)K));  // four FP32 planes of the complex G0 [K][ld]
        } else if (c->df32) {
            s.Gf = off; off = align32(off + K * df32_ld((int)K));  // G_hi, G_lo planes [K][ldg]
            if (c->has_w) {
                s.Wf = off; off = align32(off + K * df32_ld((int)K));  // W_hi, W_lo planes [K][ld]
            }
        }
    }
    c->arena_doubles = (size_t)off;
    c->psi_total = po;
    int nmax = 0;
    for (const InstDev& d : c->inst) nmax = (d.mode == SWR_MODE_TDSE && d.window_cap > nmax) ? d.window_cap : nmax;
    plan_cn_iterations(c, nmax);
    c->energy_smem = 0;
    for (const SubDev& s : c->sub) c->energy_smem = energy_smem(s) > c->energy_smem ? energy_smem(s) : c->energy_smem;
}

// Auxiliary device arrays carved after the arena (bytes, 256-aligned).
struct AuxPlan {
    size_t inst, sub, err, jobs1, jobs2, norm_part, tasks, task0, part_s, part_d, cta0, tc, scal, alive, own,
        ctal, wfix, snorm, sums_s, sums_d,
        n_active, win, win_prev, bar, queue, qlist, clslots, cnneed, rtiles, res_part, res, cv_part, cvtot, epart, energy, norm2, dipole, boff,
        psi, psi_off, tg, total;
};
static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
static AuxPlan aux_plan(const swr_ctx* c) {
    AuxPlan a;
    size_t o = al256(c->arena_doubles * sizeof(double));
    const size_t ni = c->inst.size(), ns = c->sub.size(), nt = (size_t)c->tasks_cap;
    a.inst = o; o = al256(o + ni * sizeof(InstDev));
    a.sub = o; o = al256(o + ns * sizeof(SubDev));
    a.err = o; o = al256(o + sizeof(int) * 4);
    a.jobs1 = o; o = al256(o + ns * sizeof(GemmJob));
    a.jobs2 = o; o = al256(o + ns * sizeof(GemmJob));
    a.norm_part = o; o = al256(o + ns * sizeof(double));
    a.tasks = o; o = al256(o + nt * sizeof(Task));
    a.task0 = o; o = al256(o + (ni + 1) * sizeof(int));
    a.part_s = o; o = al256(o + 2 * nt * sizeof(double));
    a.part_d = o; o = al256(o + 2 * nt * sizeof(double));
    a.cta0 = o; o = al256(o + (2 * (size_t)(c->nsm > 0 ? c->nsm : 152) + 1) * sizeof(int));
    a.ctal = o; o = al256(o + nt * sizeof(int));
    a.wfix = o; o = al256(o + ni * sizeof(int));
    a.tc = o; o = al256(o + nt * sizeof(TaskCache));
    a.scal = o; o = al256(o + 4 * ni * sizeof(double));
    a.alive = o; o = al256(o + nt * sizeof(int));
    a.own = o; o = al256(o + (size_t)c->own_total * sizeof(double));
    a.snorm = o; o = al256(o + ni * (size_t)(c->cap + 1) * sizeof(double));
    a.sums_s = o; o = al256(o + ni * sizeof(double));
    a.sums_d = o; o = al256(o + ni * sizeof(double));
    a.n_active = o; o = al256(o + sizeof(int));
    a.win = o; o = al256(o + ni * sizeof(int));
    a.win_prev = o; o = al256(o + ni * sizeof(int));
    a.bar = o; o = al256(o + sizeof(GridBarrier));
    a.queue = o; o = al256(o + sizeof(SplitQueue));
    a.qlist = o; o = al256(o + 2 * nt * sizeof(int));
    a.clslots = o; o = al256(o + 8 * nt * sizeof(unsigned long long));
    a.res_part = o; o = al256(o + ns * RES_BLOCKS * sizeof(double));
    a.res = o; o = al256(o + ni * sizeof(double));
    a.cv_part = o; o = al256(o + cvtot_part_doubles((int)ni) * sizeof(double));
    a.cvtot = o; o = al256(o + ni * sizeof(double));
    a.epart = o; o = al256(o + 3 * ns * ENERGY_BLOCKS * sizeof(double));
    a.energy = o; o = al256(o + ni * sizeof(double));
    a.norm2 = o; o = al256(o + ni * sizeof(double));
    a.dipole = o; o = al256(o + ni * sizeof(double));
    a.boff = o; o = al256(o + (c->boff.size() + 1) * sizeof(long long));
    a.cnneed = o; o = al256(o + c->cn_need.size() + 1);
    a.rtiles = o; o = al256(o + (ns + 1) * sizeof(int));
    a.psi = o; o = al256(o + (size_t)c->psi_total * sizeof(double) * (c->tdse ? 2 : 1));
    a.psi_off = o; o = al256(o + ns * sizeof(long long));
    a.tg = o;
    if (c->use_tg) {
        std::vector<int> Ks(ns), qs(ns), kds(ns), nel(ns);
        for (size_t s = 0; s < ns; ++s) {
            Ks[s] = c->sub[s].K;
            qs[s] = c->sub[s].q;
            kds[s] = c->sub[s].kd;
            nel[s] = c->sub[s].N;
        }
        o = al256(o + tg_scratch_bytes(Ks.data(), qs.data(), kds.data(), nel.data(), (int)ns, c->tdse, c->any_ee));
    }
    a.total = o;
    return a;
}

// Layout for the current device: the row tasks depend on the SM count and on
// how many window CTAs fit per SM (two at most; 152 x 2 without a device).
static bool plan_for_device(swr_ctx* c, const swr_problem* p) {
    c->df32 = (p->precision != SWR_PREC_FP64);
    int dev = 0;
    bool have_dev = cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    if (!have_dev) {
        cudaGetLastError();
        c->nsm = 152;
    }
    plan(c);  // descriptors and arena
    // automatic: the tensor-core contractions where they measured faster, when
    // every subdomain has K >= 768 (K = 1024: 1.8x the FP64 assembly; K = 576: 0.8x)
    bool all_large = !c->sub.empty();
    for (const SubDev& sd : c->sub) all_large = all_large && sd.K >= 768;
    c->use_tg = p->contraction_path == SWR_CONTRACT_TENSOR || (p->contraction_path == SWR_CONTRACT_AUTO && all_large);
    c->tasks_cap = task_capacity(c);
    c->any_ngf_stop = false;
    for (const InstDev& d : c->inst)
        if (d.window_cap == 0 && d.ngf_tol > 0.0) c->any_ngf_stop = true;
    return plan_window(c, p->window_variant, p->rows_per_task, have_dev);
}

// The requested window plan cannot run the problem.
static swr_status plan_failure() {
    return fail(nullptr, SWR_EINVAL, "the requested window plan cannot run this problem (fused: mixed precision, at "
                "most %d row tasks of at most %d rows per CTA; cluster: mixed precision, no antisymmetric instance, "
                "every subdomain's rows on chip and one cluster per subdomain resident at once)",
                window_tasks_per_cta_max(), window_rows_per_task_max());
}

static swr_status copy_problem(swr_ctx* c, const swr_problem* p) {
    c->prob = *p;
    c->inst_h.assign(p->instances, p->instances + p->n_instances);
    c->kd_h.clear();
    c->delta_h.clear();
    for (int i = 0; i < p->n_instances; ++i) {
        const swr_instance& in = p->instances[i];
        int nsub = 1;
        for (int e = 0; e < in.n_elec; ++e) nsub *= in.L;
        std::vector<int> kd(nsub);
        std::vector<double> dl(nsub);
        for (int s = 0; s < nsub; ++s) {
            kd[s] = in.K_d_per_sub ? in.K_d_per_sub[s] : in.K_d;
            dl[s] = in.delta_per_sub ? in.delta_per_sub[s] : in.delta;
        }
        c->kd_h.push_back(kd);
        c->delta_h.push_back(dl);
        c->inst_h[i].K_d_per_sub = nullptr;
        c->inst_h[i].delta_per_sub = nullptr;
    }
    c->prob.instances = c->inst_h.data();
    return SWR_OK;
}

// Row tasks, instance and CTA ranges to the device (stream-ordered).
static cudaError_t upload_tasks(swr_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->d_tasks, c->tasks.data(), c->tasks.size() * sizeof(Task),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_inst_task0, c->inst_task0.data(), c->inst_task0.size() * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_cta_task0, c->cta_task0.data(), c->cta_task0.size() * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_cta_list, c->cta_list.data(), c->cta_list.size() * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream);
    c->counters[8] += (double)(c->tasks.size() * sizeof(Task) +
                               (c->inst_task0.size() + c->cta_task0.size() + c->cta_list.size()) * sizeof(int));
    return e;
}

extern "C" swr_status swr_workspace_size(const swr_problem* p, size_t* bytes) {
    if (!bytes) return fail(nullptr, SWR_EINVAL, "bytes is NULL");
    swr_status st = validate(nullptr, p);
    if (st != SWR_OK) return st;
    swr_ctx tmp;
    copy_problem(&tmp, p);
    if (!plan_for_device(&tmp, p))
        return plan_failure();
    *bytes = aux_plan(&tmp).total;
    return SWR_OK;
}

extern "C" swr_status swr_setup(const swr_problem* p, swr_ctx** out) {
    if (!out) return fail(nullptr, SWR_EINVAL, "out is NULL");
    *out = nullptr;
    swr_status st = validate(nullptr, p);
    if (st != SWR_OK) return st;
    swr_ctx* c = new swr_ctx();
    copy_problem(c, p);
    if (!plan_for_device(c, p)) {
        delete c;
        return plan_failure();
    }
    AuxPlan a = aux_plan(c);
    c->stream = (cudaStream_t)p->stream;
    if (p->workspace) {
        if (p->workspace_bytes < a.total) {
            swr_status s2 = fail(nullptr, SWR_ENOMEM, "workspace of %zu bytes < %zu needed", p->workspace_bytes, a.total);
            delete c;
            return s2;
        }
        if (((uintptr_t)p->workspace) & 255) {
            delete c;
            return fail(nullptr, SWR_EINVAL, "workspace must be 256-byte aligned");
        }
        c->base = p->workspace;
    } else {
        cudaError_t e = cudaMalloc(&c->base, a.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, SWR_ENOMEM, "cudaMalloc(%zu) failed: %s", a.total, cudaGetErrorString(e));
        }
        c->owns = true;
    }
    char* b = (char*)c->base;
    c->arena = (double*)b;
    c->d_inst = (InstDev*)(b + a.inst);
    c->d_sub = (SubDev*)(b + a.sub);
    c->d_err = (int*)(b + a.err);
    c->d_jobs1 = (GemmJob*)(b + a.jobs1);
    c->d_jobs2 = (GemmJob*)(b + a.jobs2);
    c->d_norm_part = (double*)(b + a.norm_part);
    c->d_tasks = (Task*)(b + a.tasks);
    c->d_inst_task0 = (int*)(b + a.task0);
    c->d_part_s = (double*)(b + a.part_s);
    c->d_part_d = (double*)(b + a.part_d);
    c->d_cta_task0 = (int*)(b + a.cta0);
    c->d_cta_list = (int*)(b + a.ctal);
    c->d_wfix = (int*)(b + a.wfix);
    c->d_tc = (TaskCache*)(b + a.tc);
    c->d_scal = (double*)(b + a.scal);
    c->d_alive = (int*)(b + a.alive);
    c->d_own = (double*)(b + a.own);
    c->d_snorm = (double*)(b + a.snorm);
    c->d_sums_s = (double*)(b + a.sums_s);
    c->d_sums_d = (double*)(b + a.sums_d);
    c->d_n_active = (int*)(b + a.n_active);
    c->d_win = (int*)(b + a.win);
    c->d_win_prev = (int*)(b + a.win_prev);
    c->d_bar = (GridBarrier*)(b + a.bar);
    c->d_clslots = (unsigned long long*)(b + a.clslots);
    c->d_queue = (SplitQueue*)(b + a.queue);
    c->d_qlist = (int*)(b + a.qlist);
    c->d_res_part = (double*)(b + a.res_part);
    c->d_res = (double*)(b + a.res);
    c->d_cv_part = (double*)(b + a.cv_part);
    c->d_cvtot = (double*)(b + a.cvtot);
    c->d_epart = (double*)(b + a.epart);
    c->d_energy = (double*)(b + a.energy);
    c->d_norm2 = (double*)(b + a.norm2);
    c->d_dipole = (double*)(b + a.dipole);
    c->d_boff = (long long*)(b + a.boff);
    c->d_cn_need = (unsigned char*)(b + a.cnneed);
    c->d_rtiles = (int*)(b + a.rtiles);
    c->d_psi = (double*)(b + a.psi);
    c->d_psi_off = (long long*)(b + a.psi_off);
    if (c->use_tg) {
        const size_t ns = c->sub.size();
        std::vector<int> Ks(ns), qs(ns), kds(ns), nel(ns);
        for (size_t s = 0; s < ns; ++s) {
            Ks[s] = c->sub[s].K;
            qs[s] = c->sub[s].q;
            kds[s] = c->sub[s].kd;
            nel[s] = c->sub[s].N;
        }
        c->d_tg = (void*)(b + a.tg);
        CU(tg_setup(&c->tg, c->d_tg, Ks.data(), qs.data(), kds.data(), nel.data(), (int)ns, c->tdse, c->any_ee,
                    c->stream));
    }
    // GEMM jobs of the sum-factorised e-e block
    std::vector<GemmJob> j1(c->sub.size()), j2(c->sub.size());
    for (size_t s = 0; s < c->sub.size(); ++s) {
        const SubDev& sd = c->sub[s];
        GemmJob z;
        memset(&z, 0, sizeof(z));
        j1[s] = z;
        j2[s] = z;
        if (sd.N != 2) continue;
        int q = sd.q, kd2 = sd.kd * sd.kd;
        long long P1 = sd.work, P2 = sd.work + (long long)q * kd2, Wv = sd.work + 2LL * q * kd2,
                  Mee = sd.work + 2LL * q * kd2 + (long long)q * q;
        j1[s].a = Wv; j1[s].b = P2; j1[s].c = Mee;
        j1[s].M = q; j1[s].N = kd2; j1[s].K = q;
        j1[s].lda = q; j1[s].ldb = kd2; j1[s].ldc = kd2;
        j2[s].a = P1; j2[s].b = Mee; j2[s].c = sd.Hm;
        j2[s].M = kd2; j2[s].N = kd2; j2[s].K = q;
        j2[s].lda = kd2; j2[s].ldb = kd2; j2[s].ldc = kd2;
        j2[s].transA = 1; j2[s].mode = 1; j2[s].kd = sd.kd;
    }
    CU(cudaMemcpyAsync(c->d_inst, c->inst.data(), c->inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_sub, c->sub.data(), c->sub.size() * sizeof(SubDev), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_jobs1, j1.data(), j1.size() * sizeof(GemmJob), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_jobs2, j2.data(), j2.size() * sizeof(GemmJob), cudaMemcpyHostToDevice, c->stream));
    CU(upload_tasks(c));
    std::vector<int> wfix(c->inst.size());
    for (size_t i = 0; i < c->inst.size(); ++i) wfix[i] = c->inst[i].window_cap;
    CU(cudaMemcpyAsync(c->d_wfix, wfix.data(), wfix.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_psi_off, c->psi_off.data(), c->psi_off.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    if (!c->boff.empty())
        CU(cudaMemcpyAsync(c->d_boff, c->boff.data(), c->boff.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
        if (!c->cn_need.empty())
            CU(cudaMemcpyAsync(c->d_cn_need, c->cn_need.data(), c->cn_need.size(), cudaMemcpyHostToDevice, c->stream));
    c->counters[8] += (double)(c->inst.size() * sizeof(InstDev) + c->sub.size() * (sizeof(SubDev) + 2 * sizeof(GemmJob) + sizeof(long long)));
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream));
    CU(cudaMemsetAsync(c->d_win_prev, 0, c->inst.size() * sizeof(int), c->stream));
    CU(cudaMemsetAsync(c->d_win, 0, c->inst.size() * sizeof(int), c->stream));
    CU(cudaEventCreate(&c->ev0));
    CU(cudaEventCreate(&c->ev1));
    CU(cudaEventCreate(&c->evw0));
    CU(cudaEventCreate(&c->evw1));
    // persistent grid for the window kernel: all CTAs must be co-resident
    if (c->bps < 1 || c->nsm < 1) return fail(c, SWR_EINVAL, "window kernel does not fit on an SM");
    if (c->energy_smem > 227 * 1024)
        return fail(c, SWR_EINVAL, "2-electron subdomain with K_d x q = %zu node values: the energy kernel's tables "
                    "exceed shared memory", c->energy_smem / (2 * sizeof(double)));
    if (c->grid > c->bps * c->nsm)
        return fail(c, SWR_EINVAL, "window grid of %d CTAs exceeds %d resident CTAs", c->grid, c->bps * c->nsm);
    c->res_h.assign(c->inst.size(), 0.0);
    c->cvtot_h.assign(c->inst.size(), 0.0);
    c->spin_limit = p->spin_limit > 0 ? p->spin_limit : SPIN_LIMIT;
    c->energy_h.assign(c->inst.size(), 0.0);
    c->norm2_h.assign(c->inst.size(), 0.0);
    c->win_h.assign(c->inst.size(), 0);
    c->win_prev_h.assign(c->inst.size(), 0);
    c->win_pp_h.assign(c->inst.size(), 0);
    c->dipole_h.assign(c->inst.size(), 0.0);
    *out = c;
    return SWR_OK;
}

static swr_status check_err(swr_ctx* c) {
    int e = 0;
    CU(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    c->counters[9] += sizeof(int);
    CU(cudaStreamSynchronize(c->stream));
    if (e & SWR_ERR_SINGULAR) return fail(c, SWR_ESINGULAR, "overlap or step matrix not positive definite (ill-conditioned basis)");
    if (e & SWR_ERR_TIMEOUT) return fail(c, SWR_ETIMEOUT, "a device-side grid barrier gave up waiting");
    if (e & SWR_ERR_NUMERIC) return fail(c, SWR_ENUMERIC, "non-finite normalisation");
    return SWR_OK;
}

static SwrDeviceView view(swr_ctx* c) {
    SwrDeviceView v;
    v.arena = c->arena;
    v.inst = c->d_inst;
    v.sub = c->d_sub;
    v.n_inst = (int)c->inst.size();
    v.n_sub = (int)c->sub.size();
    v.err = c->d_err;
    return v;
}

extern "C" swr_status swr_assemble(swr_ctx* c) {
    if (!c) return fail(nullptr, SWR_EINVAL, "ctx is NULL");
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream));
    CU(cudaEventRecord(c->ev0, c->stream));
    CU(launch_assemble(view(c), c->stream, c->max_q, c->max_kd, c->max_K, c->any_ee, c->tdse, !c->tdse,
                       c->d_jobs1, c->d_jobs2, c->d_norm_part, c->tg));
    if (c->df32 && !c->tdse) CU(launch_split_df32(view(c), c->stream, c->max_K, c->has_w));
    if (c->df32 && c->tdse) CU(launch_split_c_df32(view(c), c->stream, c->max_K));
    if (c->robin_w) CU(launch_robin_ge(view(c), c->stream, c->max_K, c->max_J));
    CU(cudaEventRecord(c->ev1, c->stream));
    swr_status st = check_err(c);
    if (st != SWR_OK) return st;
    float ams = 0;
    CU(cudaEventElapsedTime(&ams, c->ev0, c->ev1));
    c->counters[6] += ams;
    c->counters[2] += kAssembleLaunchesFixed + (c->any_ee ? (c->tg ? 7 : 3) : 0) +
                      (c->tg ? 4 : 2) * ((c->max_K + GJ_NB_HOST - 1) / GJ_NB_HOST) +
                      (c->df32 ? (c->tdse || !c->has_w ? 1 : 2) : 0) + (c->robin_w && c->max_J > 0 ? 1 : 0);
    c->assembled = true;
    c->k = 0;
    c->parity = 0;
    CU(cudaMemsetAsync(c->d_win_prev, 0, c->inst.size() * sizeof(int), c->stream));
    c->win_prev_h.assign(c->inst.size(), 0);
    c->win_pp_h.assign(c->inst.size(), 0);
    c->step_done = false;
    c->refined = false;
    c->res_peak = c->res_last = 0.0;
    return SWR_OK;
}

static SweepArgs sweep_args(swr_ctx* c) {
    SweepArgs a;
    a.v = view(c);
    a.tasks = c->d_tasks;
    a.cta_task0 = c->d_cta_task0;
    a.cta_list = c->d_cta_list;
    a.n_tasks = (int)c->tasks.size();
    a.tasks_per_cta = c->tasks_per_cta;
    a.kmax = c->max_K;
    a.kdmax = c->max_kd;
    a.rows_max = c->max_rows;
    a.many = c->many;
    a.tune_steps = 0;
    a.g_tc = c->d_tc;
    a.scal_inst = c->d_scal;
    a.g_alive = c->d_alive;
    a.g_own = c->d_own;
    a.g_resident = c->g_resident ? 1 : 0;
    a.any_ngf_stop = c->any_ngf_stop ? 1 : 0;
    a.inst_task0 = c->d_inst_task0;
    a.part_s = c->d_part_s;
    a.part_d = c->d_part_d;
    a.snorm = c->d_snorm;
    a.sums_s = c->d_sums_s;
    a.sums_d = c->d_sums_d;
    a.n_active = c->d_n_active;
    a.win = c->d_win;
    a.win_prev = c->d_win_prev;
    a.cap = c->cap;
    a.bar = c->d_bar;
    a.q = c->d_queue;
    a.q_list = c->d_qlist;
    a.spin_limit = c->spin_limit;
    a.stage_floats = c->stage_floats;
    a.n_stages = c->n_stages;
    a.cl_slots = c->variant == WIN_CLUSTER ? c->d_clslots : nullptr;  // zeroed by the reset before each window
    a.tmem_cols = c->tmem_cols;
    a.cl_size = c->cl_size;
    a.cl_hs = c->cl_hs;
    a.robin_w = c->robin_w && c->variant == WIN_SPLIT ? 1 : 0;
    return a;
}

// Every launch of one Schwarz iteration (Sec. 5.4 steps 1-5) on stream st:
// the time window, line traces, averaged Robin data, residual, energy.
static cudaError_t record_iteration(swr_ctx* c, cudaStream_t st, long long* win_launches) {
    cudaError_t e = cudaSuccess;
    *win_launches = 1;
    if (c->tdse) {
        // real time: fixed window of n_steps Crank-Nicolson steps
        int nmax = 0;
        for (size_t i = 0; i < c->inst.size(); ++i) nmax = c->inst[i].window_cap > nmax ? c->inst[i].window_cap : nmax;
        e = record_event(c->evw0, st);
        if (e == cudaSuccess)
            e = launch_tdse_window(view(c), st, c->d_boff, c->d_win_prev, nmax, c->cn_need.data(), c->d_cn_need,
                                   c->max_K, c->max_kd,
                                   c->df32, fp32_phase(c), win_launches);
        if (e == cudaSuccess) e = record_event(c->evw1, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_win, c->d_wfix, c->inst.size() * sizeof(int), cudaMemcpyDeviceToDevice, st);
    } else {
        SweepArgs a = sweep_args(c);
        // the cluster window takes the Robin response of every step from memory
        if (c->robin_w && (c->variant == WIN_CLUSTER || c->variant == WIN_SPLIT)) {
            int kd2 = 0;
            for (const SubDev& sd : c->sub) kd2 = (sd.N == 2 && sd.kd > kd2) ? sd.kd : kd2;
            e = launch_robin_w(view(c), st, c->d_win_prev, kd2, c->nsm > 0 ? c->nsm : 152, c->d_rtiles);
        }
        if (e == cudaSuccess)
            e = launch_window(a, c->grid, c->win_smem, st, (int)c->inst.size(), c->variant, c->df32, fp32_phase(c),
                              c->evw0, c->evw1);
    }
    if (e == cudaSuccess)
        e = launch_post(view(c), st, c->d_win, c->d_win_prev, c->d_snorm, c->cap, c->parity, c->k == 0 ? 1 : 0,
                        c->d_res_part, RES_BLOCKS, c->d_res, c->cap, c->max_K, c->max_kd, c->max_q, c->any_anti,
                        c->d_cv_part, c->d_cvtot, c->prob.cvtot_each_iteration != 0);
    if (e == cudaSuccess)
        e = launch_energy(view(c), st, c->d_win, c->d_snorm, c->cap, c->d_epart, c->d_energy, c->d_norm2,
                          c->d_dipole, c->d_psi, c->d_psi_off, c->energy_smem);
    return e;
}

static void drop_graphs(swr_ctx* c) {
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 2; ++f)
            for (int o = 0; o < 2; ++o)
                if (c->gexec[p][f][o]) {
                    cudaGraphExecDestroy(c->gexec[p][f][o]);
                    c->gexec[p][f][o] = nullptr;
                }
}

// Captures the iteration for the current (parity, first) once; later
// iterations of the same kind replay it with one cudaGraphLaunch.
static cudaError_t capture_iteration(swr_ctx* c, int p, int f, int o) {
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    long long wl = 1;
    cudaError_t er = record_iteration(c, c->cap_stream, &wl);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (er != cudaSuccess) e = er;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec[p][f][o], g, 0ULL);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[p][f][o] = nullptr;
        return e;
    }
    c->g_win_launches[p][f][o] = wl;
    return cudaSuccess;
}

extern "C" swr_status swr_step(swr_ctx* c, swr_iter_report* rep) {
    if (!c) return fail(nullptr, SWR_EINVAL, "ctx is NULL");
    if (!c->assembled) return fail(c, SWR_ESTATE, "swr_step before swr_assemble");
    c->step_done = false;  // set again once this iteration has completed without error
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream));
    const int gp = c->parity, gf = c->k == 0 ? 1 : 0, go = fp32_phase(c) ? 1 : 0;
    if (c->prob.launch_mode == SWR_LAUNCH_GRAPH && !c->graph_failed && !c->gexec[gp][gf][go]) {
        // a capture the CUDA driver refuses leaves the context on direct launches
        if (capture_iteration(c, gp, gf, go) != cudaSuccess) {
            cudaGetLastError();
            c->graph_failed = true;
        }
    }
    CU(cudaEventRecord(c->ev0, c->stream));
    long long win_launches = 1;
    if (c->gexec[gp][gf][go]) {
        CU(cudaGraphLaunch(c->gexec[gp][gf][go], c->stream));
        win_launches = c->g_win_launches[gp][gf][go];
    } else {
        CU(record_iteration(c, c->stream, &win_launches));
    }
    CU(cudaEventRecord(c->ev1, c->stream));
    const size_t ni = c->inst.size();
    CU(cudaMemcpyAsync(c->res_h.data(), c->d_res, ni * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->win_h.data(), c->d_win, ni * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->energy_h.data(), c->d_energy, ni * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->norm2_h.data(), c->d_norm2, ni * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->dipole_h.data(), c->d_dipole, ni * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (c->prob.cvtot_each_iteration)
        CU(cudaMemcpyAsync(c->cvtot_h.data(), c->d_cvtot, ni * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    c->counters[9] += (double)(ni * ((c->prob.cvtot_each_iteration ? 5 : 4) * sizeof(double) + sizeof(int)));
    swr_status st = check_err(c);
    if (st != SWR_OK) return st;
    c->cvtot_valid = c->prob.cvtot_each_iteration != 0;
    // the current window becomes the previous one for the next iteration
    CU(cudaMemcpyAsync(c->d_win_prev, c->d_win, ni * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
    c->win_pp_h = c->win_prev_h;
    c->win_prev_h = c->win_h;
    c->k += 1;
    c->parity ^= 1;
    double rmax = 0, cmax = 0;
    int wmax = 0;
    long long solves = 0;
    for (size_t i = 0; i < ni; ++i) {
        if (!isfinite(c->res_h[i])) return fail(c, SWR_ENUMERIC, "non-finite residual in instance %zu", i);
        rmax = c->res_h[i] > rmax ? c->res_h[i] : rmax;
        if (c->cvtot_valid) cmax = c->cvtot_h[i] > cmax ? c->cvtot_h[i] : cmax;
        wmax = c->win_h[i] > wmax ? c->win_h[i] : wmax;
        // antisymmetric states: the lower subdomain of a mirror pair is not solved
        const int solved = c->inst[i].anti ? c->inst[i].L * (c->inst[i].L + 1) / 2 : c->inst[i].n_sub;
        solves += (long long)c->win_h[i] * solved;
    }
    float ms = 0, wms = 0;
    CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    CU(cudaEventElapsedTime(&wms, c->evw0, c->evw1));
    double flops = 0, bytes = 0, bytes_alg = 0;
    {
        std::vector<int> nsolve(c->inst.size());
        for (size_t i = 0; i < ni; ++i) nsolve[i] = c->win_h[i];
        // bytes per matrix element: complex G0 16 (FP64 pair or four FP32 planes);
        // real G 8 (FP64 or FP32 hi/lo); the fused variant also streams W (16);
        // half of each with the FP32-rounded matrices (hi planes only)
        const double bel = (c->tdse ? 16.0 : (c->variant == WIN_FUSED ? 16.0 : 8.0)) * (go ? 0.5 : 1.0);
        for (size_t sid = 0; sid < c->sub.size(); ++sid) {
            const SubDev& sd = c->sub[sid];
            if (c->inst[sd.inst].anti && sd.N == 2 && sd.idx[0] > sd.idx[1]) continue;  // mirror image, not solved
            const double K2 = (double)sd.K * sd.K;
            // real time: (1 + fixed-point iterations) complex matvecs with G0 per step
            const double mv = c->tdse ? c->cn_sweeps[sid] : (double)nsolve[sd.inst];
            flops += (c->tdse ? 8.0 : 2.0) * K2 * mv;
            bytes += bel * K2 * mv;
            bytes_alg += (c->tdse ? 16.0 : 8.0) * (go ? 0.5 : 1.0) * K2 * mv;
        }
    }
    c->counters[0] += wms;
    c->counters[1] += 1;
    c->counters[2] += kStepLaunches - 1 + win_launches + (c->any_anti ? 1 : 0) + (c->prob.cvtot_each_iteration ? 2 : 0) +
                      (!c->tdse && c->robin_w && (c->variant == WIN_CLUSTER || c->variant == WIN_SPLIT) ? 3 : 0);
    c->counters[3] += flops;
    c->counters[4] += bytes;
    c->counters[5] += (double)solves;
    c->counters[7] += ms;
    c->counters[10] += bytes_alg;
    if (rep) {
        rep->k = c->k;
        rep->res = rmax;
        rep->window_max = wmax;
        rep->subdomain_solves = solves;
        rep->seconds = ms * 1e-3;
        rep->cvtot = c->cvtot_valid ? cmax : -1.0;
        rep->fp32_matrices = go;
    }
    if (go) {
        // the FP32 phase ends once Res(k) reaches the switch level, or when it has
        // fallen far below its peak and stopped falling
        c->res_peak = rmax > c->res_peak ? rmax : c->res_peak;
        // default: ten times the tolerance of the running swr_iterate (iterations of the
        // FP32-rounded problem below that only approach its own fixed point), else
        // 1e-7 of the largest residual so far
        const double thr = c->prob.refine_res > 0.0 ? c->prob.refine_res
                           : c->iterate_tol > 0.0   ? 10.0 * c->iterate_tol
                                                    : 1e-7 * c->res_peak;
        const bool stalled = c->k >= 3 && rmax < 1e-3 * c->res_peak && rmax > 0.9 * c->res_last;
        if (rmax <= thr || stalled) c->refined = true;  // graphs are kept per phase
        c->res_last = rmax;
    }
    c->step_done = true;
    return SWR_OK;
}

// Times the current window plan on a fixed window of `steps` steps (best of two).
static swr_status time_window_plan(swr_ctx* c, int steps, double* sec_per_step) {
    CU(upload_tasks(c));
    SweepArgs a = sweep_args(c);
    a.tune_steps = steps;
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        CU(cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream));
        CU(launch_window(a, c->grid, c->win_smem, c->stream, (int)c->inst.size(), c->variant, c->df32, fp32_phase(c),
                         c->evw0,
                         c->evw1));
        c->counters[2] += 2;
        swr_status st = check_err(c);
        if (st != SWR_OK) return st;
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, c->evw0, c->evw1));
        best = ms < best ? ms : best;
    }
    *sec_per_step = 1e-3 * best / steps;
    return SWR_OK;
}

extern "C" swr_status swr_window_plan(const swr_ctx* c, swr_tune_report* out) {
    if (!c || !out) return fail(nullptr, SWR_EINVAL, "ctx or out is NULL");
    memset(out, 0, sizeof(*out));
    out->variant = c->tdse ? 0 : c->variant;
    out->rows_per_task = c->rows_target;
    out->tasks = (int)c->tasks.size();
    out->ctas = c->grid;
    out->task_state_global = c->many;
    out->graph = (c->prob.launch_mode == SWR_LAUNCH_GRAPH && !c->graph_failed) ? 1 : 0;
    out->tensor_contractions = c->use_tg ? 1 : 0;
    return SWR_OK;
}

extern "C" swr_status swr_autotune(swr_ctx* c, int steps, swr_tune_report* out) {
    if (!c) return fail(nullptr, SWR_EINVAL, "ctx is NULL");
    if (c->tdse) return fail(c, SWR_EINVAL, "real-time problems have no window kernel to tune");
    if (!c->assembled || c->k != 0) return fail(c, SWR_ESTATE, "swr_autotune needs swr_assemble and no swr_step yet");
    if (steps < 2 || steps > c->cap) return fail(c, SWR_EINVAL, "steps must be in [2, %d]", c->cap);
    struct Cand {
        int variant, rows;
    };
    std::vector<Cand> cands;
    cands.push_back({c->prob.window_variant, c->prob.rows_per_task});  // the plan before tuning
    const int rows_list[] = {0, 16, 32, 64, 128, 256};
    const int variants[] = {WIN_TWO_PHASE, WIN_FUSED, WIN_SPLIT, WIN_RESIDENT, WIN_CLUSTER};
    for (int v : variants) {
        if (v == WIN_FUSED && !(c->df32 && c->has_w)) continue;
        if ((v == WIN_SPLIT || v == WIN_RESIDENT || v == WIN_CLUSTER) && !c->df32) continue;
        if (v == WIN_CLUSTER && (c->any_anti || !c->robin_w)) continue;
        if (v == WIN_TWO_PHASE && c->prob.precision == SWR_PREC_FP32_REFINED) continue;  // reads both planes
        for (int r : rows_list) cands.push_back({v, r});
    }
    std::vector<std::vector<int>> seen;  // (variant, tasks, grid, rows target) of the plans timed
    double best_t = 1e30, t_default = 0;
    Cand best = cands[0];
    int timed = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (!plan_window(c, cands[i].variant, cands[i].rows, true)) continue;
        if (c->bps < 1 || c->grid > c->bps * c->nsm) continue;
        std::vector<int> sig = {c->variant, (int)c->tasks.size(), c->grid, c->rows_target};
        bool dup = false;
        for (const auto& x : seen) dup = dup || x == sig;
        if (dup) continue;
        seen.push_back(sig);
        double t = 0;
        swr_status st = time_window_plan(c, steps, &t);
        if (st != SWR_OK) return st;
        ++timed;
        if (i == 0) t_default = t;
        if (t < best_t) {
            best_t = t;
            best = {c->variant, c->rows_target};
        }
    }
    drop_graphs(c);  // captured with the old plan's launch configuration
    if (!plan_window(c, best.variant, best.rows, true) || c->bps < 1 || c->grid > c->bps * c->nsm)
        return fail(c, SWR_EINVAL, "autotune: the chosen plan no longer fits");
    CU(upload_tasks(c));
    c->prob.window_variant = best.variant;
    c->prob.rows_per_task = best.rows;
    if (out) {
        out->variant = c->variant;
        out->rows_per_task = c->rows_target;
        out->tasks = (int)c->tasks.size();
        out->ctas = c->grid;
        out->task_state_global = c->many;
        out->candidates = timed;
        out->graph = (c->prob.launch_mode == SWR_LAUNCH_GRAPH && !c->graph_failed) ? 1 : 0;
        out->seconds_per_step = best_t;
        out->seconds_default = t_default;
    }
    return check_err(c);
}

extern "C" swr_status swr_iterate(swr_ctx* c, double tol, int kmax, swr_report* rep, double* hist) {
    if (!c) return fail(nullptr, SWR_EINVAL, "ctx is NULL");
    if (kmax < 1) return fail(c, SWR_EINVAL, "kmax must be >= 1");
    swr_report r;
    memset(&r, 0, sizeof(r));
    for (int it = 0; it < kmax; ++it) {
        swr_iter_report ir;
        c->iterate_tol = tol;
        swr_status st = swr_step(c, &ir);
        c->iterate_tol = 0.0;
        if (st != SWR_OK) return st;
        if (hist) hist[it] = ir.res;
        r.iterations = it + 1;
        r.res_last = ir.res;
        r.subdomain_solves += ir.subdomain_solves;
        r.seconds += ir.seconds;
        r.fp32_iterations += ir.fp32_matrices;
        if (ir.res <= tol && ir.fp32_matrices && !c->refined) {
            c->refined = true;  // tolerance met with the FP32-rounded matrices: refine from here
            continue;
        }
        if (ir.res <= tol && !ir.fp32_matrices) {
            r.converged = 1;
            break;
        }
    }
    if (rep) *rep = r;
    return r.converged ? SWR_OK : fail(c, SWR_ENOTCONV, "Res(k) = %g > tol = %g after %d iterations", r.res_last, tol, kmax);
}

static size_t trace_bytes(const swr_ctx* c) {
    // [win per instance as int64] + per subdomain: own traces u and Robin source b' for steps 0..cap
    size_t b = c->inst.size() * sizeof(long long);
    const int cx = c->tdse ? 2 : 1;
    for (const SubDev& s : c->sub)
        b += (size_t)(c->cap + 1) * ((size_t)(s.ngam > 0 ? s.ngam : 1) + s.K) * cx * sizeof(double);
    return b;
}

extern "C" swr_status swr_field_bytes(swr_ctx* c, int field, size_t* bytes) {
    if (!c || !bytes) return fail(c, SWR_EINVAL, "NULL argument");
    const size_t ni = c->inst.size(), ns = c->sub.size();
    const int cx = c->tdse ? 2 : 1;
    switch (field) {
        case SWR_FIELD_ENERGY: case SWR_FIELD_NORM2: case SWR_FIELD_DIPOLE: case SWR_FIELD_RES: case SWR_FIELD_CVTOT:
            *bytes = ni * sizeof(double); return SWR_OK;
        case SWR_FIELD_WINDOW: *bytes = ni * sizeof(int); return SWR_OK;
        case SWR_FIELD_PSI_NODES: *bytes = (size_t)c->psi_total * cx * sizeof(double); return SWR_OK;
        case SWR_FIELD_OWN_TRACES: case SWR_FIELD_ROBIN: {
            size_t b = 0;
            for (size_t s = 0; s < ns; ++s)
                b += (size_t)(c->win_h[c->sub[s].inst] + 1) * c->sub[s].ngam * cx * sizeof(double);
            *bytes = b;
            return SWR_OK;
        }
        case SWR_FIELD_TRACE_BYTES: *bytes = sizeof(size_t); return SWR_OK;
        case SWR_FIELD_NODE_COUNTS: *bytes = 3 * ns * sizeof(int); return SWR_OK;
        case SWR_FIELD_K_MAX: *bytes = sizeof(int); return SWR_OK;
        case SWR_FIELD_COUNTERS: *bytes = 11 * sizeof(double); return SWR_OK;
    }
    return fail(c, SWR_EINVAL, "unknown field %d", field);
}

extern "C" swr_status swr_get(swr_ctx* c, int field, void* host, size_t bytes) {
    if (!c || !host) return fail(c, SWR_EINVAL, "NULL argument");
    size_t need = 0;
    swr_status st = swr_field_bytes(c, field, &need);
    if (st != SWR_OK) return st;
    if (bytes != need) return fail(c, SWR_EINVAL, "field %d needs exactly %zu bytes, got %zu", field, need, bytes);
    const size_t ni = c->inst.size();
    const int cx = c->tdse ? 2 : 1;
    switch (field) {
        case SWR_FIELD_ENERGY: memcpy(host, c->energy_h.data(), need); return SWR_OK;
        case SWR_FIELD_NORM2: memcpy(host, c->norm2_h.data(), need); return SWR_OK;
        case SWR_FIELD_RES: memcpy(host, c->res_h.data(), need); return SWR_OK;
        case SWR_FIELD_CVTOT:
            if (c->k == 0) return fail(c, SWR_ESTATE, "no iteration done yet");
            if (!c->cvtot_valid) {
                CU(launch_cvtot(view(c), c->stream, c->d_win, c->d_snorm, c->cap, c->d_cv_part, c->d_cvtot));
                CU(cudaMemcpyAsync(c->cvtot_h.data(), c->d_cvtot, need, cudaMemcpyDeviceToHost, c->stream));
                CU(cudaStreamSynchronize(c->stream));
                c->counters[2] += 2;
                c->counters[9] += (double)need;
                c->cvtot_valid = true;
            }
            memcpy(host, c->cvtot_h.data(), need);
            return SWR_OK;
        case SWR_FIELD_WINDOW: memcpy(host, c->win_h.data(), need); return SWR_OK;
        case SWR_FIELD_DIPOLE: memcpy(host, c->dipole_h.data(), need); return SWR_OK;
        case SWR_FIELD_K_MAX: memcpy(host, &c->k, sizeof(int)); return SWR_OK;
        case SWR_FIELD_COUNTERS: memcpy(host, c->counters, sizeof(c->counters)); return SWR_OK;
        case SWR_FIELD_TRACE_BYTES: { size_t tb = trace_bytes(c); memcpy(host, &tb, sizeof(size_t)); return SWR_OK; }
        case SWR_FIELD_NODE_COUNTS: {
            int* o = (int*)host;
            for (size_t s = 0; s < c->sub.size(); ++s) {
                o[3 * s] = c->sub[s].q;
                o[3 * s + 1] = c->sub[s].ngam;
                o[3 * s + 2] = c->sub[s].K;
            }
            return SWR_OK;
        }
        case SWR_FIELD_PSI_NODES:
            c->counters[9] += (double)need;
            CU(cudaMemcpyAsync(host, c->d_psi, need, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            return SWR_OK;
        case SWR_FIELD_OWN_TRACES: case SWR_FIELD_ROBIN: {
            if (c->k == 0) return fail(c, SWR_ESTATE, "no iteration done yet");
            char* h = (char*)host;
            const int par = c->parity ^ 1;  // buffer written by the last iteration
            for (size_t s = 0; s < c->sub.size(); ++s) {
                const SubDev& sd = c->sub[s];
                size_t nb = (size_t)(c->win_h[sd.inst] + 1) * sd.ngam * cx * sizeof(double);
                long long off = (field == SWR_FIELD_OWN_TRACES) ? sd.u[par] : sd.g;
                if (nb) CU(cudaMemcpyAsync(h, c->arena + off, nb, cudaMemcpyDeviceToHost, c->stream));
                h += nb;
            }
            CU(cudaStreamSynchronize(c->stream));
            (void)ni;
            return SWR_OK;
        }
    }
    return fail(c, SWR_EINVAL, "unknown field %d", field);
}

extern "C" swr_status swr_traces(swr_ctx* c, int dir, swr_trace_view* view_) {
    if (!c || !view_ || !view_->host) return fail(c, SWR_EINVAL, "NULL argument");
    if (!c->assembled) return fail(c, SWR_ESTATE, "swr_traces before swr_assemble");
    const size_t need = trace_bytes(c);
    if (view_->bytes != need) return fail(c, SWR_EINVAL, "trace window needs %zu bytes, got %zu", need, view_->bytes);
    const int cx = c->tdse ? 2 : 1;
    char* h = (char*)view_->host;
    const size_t ni = c->inst.size();
    const int par = c->parity ^ 1;  // u buffer of the last iteration
    if (dir == SWR_GET) {
        long long* w = (long long*)h;
        for (size_t i = 0; i < ni; ++i) w[i] = c->win_prev_h[i];
        h += ni * sizeof(long long);
        for (const SubDev& s : c->sub) {
            size_t nu = (size_t)(c->cap + 1) * (s.ngam > 0 ? s.ngam : 1) * cx * sizeof(double);
            size_t nbv = (size_t)(c->cap + 1) * s.K * cx * sizeof(double);
            CU(cudaMemcpyAsync(h, c->arena + s.u[par], nu, cudaMemcpyDeviceToHost, c->stream));
            h += nu;
            CU(cudaMemcpyAsync(h, c->arena + s.bvec, nbv, cudaMemcpyDeviceToHost, c->stream));
            h += nbv;
        }
        CU(cudaStreamSynchronize(c->stream));
        return SWR_OK;
    }
    if (dir != SWR_SET) return fail(c, SWR_EINVAL, "dir must be SWR_GET or SWR_SET");
    const long long* w = (const long long*)h;
    for (size_t i = 0; i < ni; ++i) {
        if (w[i] < 0 || w[i] > c->cap) return fail(c, SWR_EINVAL, "window %lld out of range", w[i]);
        c->win_prev_h[i] = (int)w[i];
        c->win_h[i] = (int)w[i];
    }
    h += ni * sizeof(long long);
    // the restored u goes to the buffer the next iteration compares against
    const int tgt = c->parity ^ 1;
    for (const SubDev& s : c->sub) {
        size_t nu = (size_t)(c->cap + 1) * (s.ngam > 0 ? s.ngam : 1) * cx * sizeof(double);
        size_t nbv = (size_t)(c->cap + 1) * s.K * cx * sizeof(double);
        CU(cudaMemcpyAsync(c->arena + s.u[tgt], h, nu, cudaMemcpyHostToDevice, c->stream));
        h += nu;
        CU(cudaMemcpyAsync(c->arena + s.bvec, h, nbv, cudaMemcpyHostToDevice, c->stream));
        h += nbv;
    }
    CU(cudaMemcpyAsync(c->d_win_prev, c->win_prev_h.data(), ni * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (c->k == 0) c->k = 1;  // the next residual compares against the restored traces
    c->step_done = false;     // the restored state has no residual of its own until the next swr_step
    return SWR_OK;
}

extern "C" swr_status swr_set_spin_limit(swr_ctx* c, long long polls) {
    if (!c) return fail(nullptr, SWR_EINVAL, "ctx is NULL");
    if (polls < 0) return fail(c, SWR_EINVAL, "polls must be >= 0 (0: default)");
    c->spin_limit = polls > 0 ? polls : SPIN_LIMIT;
    drop_graphs(c);  // captured iterations carry the old limit in their kernel arguments
    return SWR_OK;
}

// Internal accessor for the allocation-free residual entry point (swr_noalloc.cu).
namespace swr {
bool residual_inputs(swr_ctx* c, ResidualInputs* r) {
    if (!c || !c->assembled || c->k < 1 || !c->step_done) return false;
    r->v = view(c);
    r->stream = c->stream;
    r->k = c->k;
    r->parity_last = c->parity ^ 1;
    r->n_inst = (int)c->inst.size();
    r->n_sub = (int)c->sub.size();
    r->win_last = c->win_prev_h.data();
    r->win_before = c->win_pp_h.data();
    return true;
}
void set_error(swr_ctx* c, const char* msg) {
    if (c) c->err = msg;
}
struct CodecInputs {
    SwrDeviceView v;
    cudaStream_t stream;
    int n_sub, n_inst, window, nch, max_q;
    int* d_win_prev;
    std::vector<int>* win_prev_h;
    std::vector<int>* win_h;
    bool* codec_ready;
};
bool codec_inputs(swr_ctx* c, CodecInputs* r) {
    if (!c || !c->assembled) return false;
    r->v = view(c);
    r->stream = c->stream;
    r->n_sub = (int)c->sub.size();
    r->n_inst = (int)c->inst.size();
    int w = c->inst[0].window_cap;
    for (const InstDev& d : c->inst)
        if (d.window_cap != w) w = 0;  // the code needs one fixed window for all instances
    r->window = w;
    r->nch = c->tdse ? 2 : 1;
    r->max_q = c->max_q;
    r->d_win_prev = c->d_win_prev;
    r->win_prev_h = &c->win_prev_h;
    r->win_h = &c->win_h;
    r->codec_ready = nullptr;
    return true;
}
void codec_release(const swr_ctx* c);
}  // namespace swr

extern "C" void swr_destroy(swr_ctx* c) {
    if (!c) return;
    codec_release(c);
    if (c->tg) tg_release(c->tg);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->evw0) cudaEventDestroy(c->evw0);
    if (c->evw1) cudaEventDestroy(c->evw1);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->owns && c->base) cudaFree(c->base);
    delete c;
}

extern "C" const char* swr_last_error(const swr_ctx* c) {
    if (!c) return g_setup_err.c_str();
    return c->err.c_str();
}
