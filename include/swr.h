/*
 * swr.h -- C ABI of the GB300 (sm_103a) Schwarz Waveform Relaxation (SWR)
 * Galerkin sweep for the N-body Schroedinger equation.
 *
 * The method (E. Lorin, "Domain Decomposition Method for the N-body
 * Time-Independent and Time-Dependent Schroedinger Equation"):
 *   - the configuration space [a,b]^N (d = 1, N = 1 or 2 electrons) is cut into
 *     L^N overlapping hypercubes Omega_{i1 + L*i2}, overlap bands of width eps
 *     (opening of Sec. 6);
 *   - on each subdomain the wavefunction is expanded in tensor products of 1-D
 *     Gaussians exp(-delta (x - alpha)^2) (Sec. 2, Eq. gauss1d), giving local
 *     Galerkin systems A_i, H~_i (with the Robin term R_i) and Q_i
 *     (Sec. 5.1, "Construction of the local approximate solutions");
 *   - imaginary time: implicit Euler + global normalisation (NGF, Sec. 5.2 and
 *     Sec. 5.4 step 2/4); real time: Crank-Nicolson under the dipole field
 *     (Sec. 1.2, Sec. 5.4 step 2);
 *   - subdomains exchange Robin data (d_n + mu) psi_j, averaged over all
 *     overlapping neighbours (Sec. 5.1, Eq. RTC and the multi-subdomain rule);
 *   - convergence is measured by the residual Res(k) of Eq. residueRT / residueIT
 *     (Sec. 6.2, 6.3).
 *
 * Every entry point returns a swr_status; no C++ exception crosses the ABI.
 * swr_last_error(ctx) returns a human-readable detail string for the last
 * failing call on that context (or a setup failure when ctx is NULL).
 * A context is not thread-safe; distinct contexts are independent.
 * All device work is ordered on the CUDA stream given in swr_problem.stream
 * (NULL = the legacy default stream).  Host buffers are owned by the caller.
 */
#ifndef SWR_H
#define SWR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum swr_status {
    SWR_OK = 0,
    SWR_EINVAL = 1,      /* invalid argument or problem description            */
    SWR_ENOMEM = 2,      /* device allocation failed / workspace too small      */
    SWR_ECUDA = 3,       /* CUDA runtime error (detail in swr_last_error)       */
    SWR_ESINGULAR = 4,   /* overlap matrix not positive definite (basis too
                            ill-conditioned for the Cholesky orthogonalisation) */
    SWR_ENUMERIC = 5,    /* NaN / Inf met in a solve or a trace                 */
    SWR_ENOTCONV = 6,    /* swr_iterate reached kmax above tol (report filled)  */
    SWR_ETIMEOUT = 7,    /* a bounded device-side wait gave up                  */
    SWR_ESTATE = 8       /* call out of order (e.g. swr_step before assemble)  */
} swr_status;

typedef enum swr_mode {
    SWR_MODE_TISE = 0,   /* imaginary time: implicit Euler (+ normalisation)    */
    SWR_MODE_TDSE = 1    /* real time: Crank-Nicolson with the dipole field     */
} swr_mode;

typedef enum swr_precision {
    SWR_PREC_FP64 = 0,   /* plain FP64 everywhere                                */
    SWR_PREC_MIXED = 1,  /* step matrices stored as FP32 hi/lo pairs (four planes for
                            the complex real-time G0) with error-free FP32
                            accumulation: FP64-level accuracy on the FP32 pipes;
                            FP64 reductions, norms, orthogonalisation, inversion  */
    SWR_PREC_FP32_REFINED = 2 /* the Schwarz iterations first run with the step
                            matrices rounded to FP32 (only the hi plane of
                            SWR_PREC_MIXED is read: 4 bytes per real element, 8
                            per complex one; the products of the rounded matrix
                            are still formed in double-single arithmetic, so each
                            iteration is the FP64 iteration of a matrix perturbed
                            by at most 2^-24 relative), then, once Res(k) <=
                            swr_problem.refine_res or Res(k) stops falling, with
                            the double-single matrices: the remaining iterations
                            are the outer refinement that carries the iterate to
                            the fixed point of the exact discrete problem.
                            swr_iterate stops only on a refined iteration.      */
} swr_precision;

/* How swr_step launches the kernels of one Schwarz iteration.  Both run the
 * same kernels with the same arguments (bit-identical results).             */
typedef enum swr_launch_mode {
    SWR_LAUNCH_GRAPH = 0,      /* capture the iteration into a CUDA graph once
                                  per kind (parity of the trace buffers, first
                                  iteration) and replay it: one host launch per
                                  iteration (if the CUDA driver refuses the
                                  capture, it launches directly; swr_window_plan
                                  reports which)                                */
    SWR_LAUNCH_DIRECT = 1      /* launch every kernel from the host             */
} swr_launch_mode;

/* Kernel that runs the imaginary-time window (Sec. 5.2, system SIT).  Both
 * compute the same step; they differ in how the per-step normalisation is
 * synchronised, and so in summation order (results agree to rounding).      */
typedef enum swr_window_variant {
    SWR_WINDOW_AUTO = 0,       /* mixed precision: cluster when it fits (and no
                                  row target is given), else fused when it fits,
                                  else split; FP64: two-phase                    */
    SWR_WINDOW_TWO_PHASE = 1,  /* y = G v, grid barrier, z = (Pp (x) Pp) y, grid
                                  barrier: G read once per step (8 bytes per
                                  element in both precisions); any batch size
                                  (task state in global memory when a CTA holds
                                  more tasks than its shared memory)             */
    SWR_WINDOW_FUSED = 2,      /* mixed precision only: y = G v and z = W v with
                                  W = (Pp (x) Pp) G precomputed, one grid barrier
                                  per step (16 bytes per element); at most 4 row
                                  tasks of at most 64 rows per CTA               */
    SWR_WINDOW_SPLIT = 3,      /* mixed precision only: u = G y^n in one pass
                                  over G before s_n is known, y^{n+1} = u / s_n
                                  + w formed after the next barrier, with
                                  w = kappa dt G b' read from the Robin response
                                  formed before the window for every step (with
                                  antisymmetric instances: formed in the same
                                  pass over G); one grid barrier per step,
                                  8 bytes per element, any batch size (task state
                                  in global memory); the stop on the NGF
                                  tolerance is decided one step later and the
                                  extra step dropped                             */
    SWR_WINDOW_RESIDENT = 4,   /* mixed precision only, no antisymmetric
                                  instances: the split recursion with static
                                  tasks (at most 4 of at most 64 rows per CTA)
                                  whose G_hi rows stay in shared memory for the
                                  whole window: a step reads only G_lo from L2
                                  (nothing with the FP32-rounded matrices), no W;
                                  one grid barrier per step                      */
    SWR_WINDOW_CLUSTER = 5     /* mixed precision only, no antisymmetric
                                  instances, K <= 768: one thread-block cluster
                                  (one CTA per SM) per subdomain; each CTA keeps
                                  its rows of G on chip for the whole window
                                  (G_hi in shared memory, G_lo in tensor memory),
                                  y^n moves between the CTAs of a cluster through
                                  distributed shared memory, one cluster barrier
                                  per step and one arrival counter per instance
                                  for s_n (no grid barrier), the product G y^n
                                  formed while s_n is reduced and w = kappa dt
                                  G b' read from the Robin response formed before
                                  the window; needs every subdomain's cluster
                                  resident at once                              */
} swr_window_variant;

/* Where swr_assemble runs its two dense contractions: the e-e block of the
 * local Hamiltonians (Sec. 5.1: B^T diag(w V_ee) B, sum-factorised into two
 * products per subdomain) and the rank-32 trailing updates of the blocked
 * Gauss-Jordan inversion of the step matrices (Sec. 5.4 step 2: the local
 * systems I + dt H' and I + i dt/2 H').  Either in FP64 on the FP64 pipe, or
 * on the 5th-generation tensor cores with FP64 emulated by exact BF16 slices:
 * every operand row / column scaled by a power of two and cut into integer
 * slices that BF16 holds exactly (9 slices of 7 bits for the inversion's
 * 32-long inner products, 11 of 6 bits for the e-e products' inner length up
 * to 384), one FP32 tensor-memory accumulator per slice level (exact sums),
 * levels combined in FP64: the dropped terms stay below 2^-63 (inversion) or
 * 2^-66 (e-e) of the largest operand products times the inner length.     */
typedef enum swr_contraction {
    SWR_CONTRACT_AUTO = 0,     /* tensor cores when every subdomain has K >= 768
                                  (measured: 1.8x the FP64 assembly at K = 1024,
                                  0.8x at K = 576), else FP64                     */
    SWR_CONTRACT_FP64 = 1,     /* FP64 products                                   */
    SWR_CONTRACT_TENSOR = 2    /* tensor-core products                            */
} swr_contraction;

/* Transmission condition (Sec. 4, "Selection of the transmission
 * conditions"): the data g_i each subdomain takes from its covering
 * neighbours j at its interface nodes, averaged over them.  Both enter the
 * local problem through the same boundary term (mu/2 R, kappa = 1/2) and the
 * source of g_i.                                                            */
typedef enum swr_tc {
    SWR_TC_ROBIN = 0,      /* g_i = (n_i . grad + mu) psi_j  (Eq. RTC)            */
    SWR_TC_DIRICHLET = 1   /* g_i = mu psi_j: the classical SWR (Dirichlet
                              condition psi_i = psi_j) imposed by penalty with
                              constant mu; consistent up to O(1/mu)               */
} swr_tc;

/* Exchange symmetry of the state (Appendix A).  With SWR_SYM_ANTISYMMETRIC
 * (N = 2) the initial data is the antisymmetric part of the projected
 * Gaussian and psi_sigma(i)(x2, x1) = -psi_i(x1, x2) holds at every step,
 * sigma(i) the subdomain (i2, i1) of subdomain (i1, i2): only one subdomain
 * of each mirror pair is stepped, the other filled in as its mirror image
 * (swap: coefficient (a, b) -> (b, a), sign flipped).  In imaginary time the
 * diagonal subdomains also act on the antisymmetric part of each step's
 * input, (v - swap(v)) / 2, so the iteration reaches the lowest
 * antisymmetric (triplet) state.  Needs mirror subdomains with the same K_d
 * and delta, and an initial Gaussian whose antisymmetric part is not zero
 * (phi0_center off the diagonal); the fused window variant is not available
 * for such instances.                                                       */
typedef enum swr_symmetry {
    SWR_SYM_NONE = 0,
    SWR_SYM_ANTISYMMETRIC = 1
} swr_symmetry;

/* One SWR problem: global box [box_lo, box_hi]^n_elec cut into L^n_elec
 * subdomains.  Subdomain sid = i1 + L*i2 covers, in coordinate e,
 * [a + i_e H - overlap/2, a + (i_e+1) H + overlap/2], H = (b-a)/L.          */
typedef struct swr_instance {
    int    n_elec;          /* N = 1 or 2 (d = 1)                                 */
    double box_lo, box_hi;  /* a, b                                               */
    int    L;               /* subdomains per coordinate (>= 1)                   */
    double overlap;         /* eps, 0 < eps < H (any eps > 0 when L == 1)         */
    int    K_d;             /* Gaussians per coordinate, used when K_d_per_sub is NULL */
    const int*    K_d_per_sub;   /* optional [L^N] Gaussians per coordinate per subdomain */
    double delta;           /* Gaussian exponent, used when delta_per_sub is NULL */
    const double* delta_per_sub; /* optional [L^N]                                */
    int    q_p;             /* Gauss-Legendre nodes per panel (1..64)             */
    int    n_mid;           /* equal panels of the middle zone [lo+eps, hi-eps]   */
    int    n_nuclei;        /* P <= 3                                              */
    double x_nuc[3], Z_nuc[3];
    double eta_en, eta_ee;  /* soft-Coulomb parameters (Eq. pseudo)               */
    double ee_coef;         /* e-e prefactor (1: physical, 0: none)               */
    double harmonic;        /* + harmonic * x_e^2 / 2 per electron                 */
    double kinetic;         /* kappa in -kappa * Laplacian (1/2 for H0)           */
    double mu_re, mu_im;    /* Robin constant mu (Eq. RTC)                         */
    int    mode;            /* swr_mode                                            */
    int    normalize;       /* TISE: renormalise every step (NGF)                 */
    double dt;
    int    n_steps;         /* fixed window (TDSE; TISE when ngf_tol <= 0)        */
    double ngf_tol;         /* TISE inner stop ||phi^{n+1} - phi^n|| <= ngf_tol   */
    int    max_steps;       /* TISE window cap                                    */
    double field_E0, field_T, field_omega, field_phase; /* e(t) = E0 sin^2(pi t/T) sin(omega t + phase), 0 <= t <= T */
    double phi0_gamma;      /* phi0 = exp(-gamma |x - x0|^2)                       */
    double phi0_center[2];
    double orth_tau;        /* basis reduction (Sec. 2's Gaussian overlaps are ill-
                               conditioned): per coordinate, Cholesky of the 1-D
                               overlap S when every pivot >= orth_tau * max diag,
                               else canonical orthogonalisation, keeping the
                               eigenvectors with lambda > orth_tau * lambda_max
                               (X = U_r lambda_r^-1/2, the other columns zero).
                               0 selects 1e-12; must be < 1                      */
    int    tc;              /* swr_tc: transmission condition of the Schwarz data  */
    int    symmetry;        /* swr_symmetry                                        */
} swr_instance;

typedef struct swr_problem {
    int                 n_instances;  /* independent problems batched together */
    const swr_instance* instances;    /* [n_instances], copied by swr_setup     */
    int                 precision;    /* swr_precision                          */
    void*               stream;       /* cudaStream_t (NULL: default stream)    */
    void*               workspace;    /* optional caller-owned device buffer    */
    size_t              workspace_bytes; /* >= swr_workspace_size() when given   */
    int                 window_variant;  /* swr_window_variant (0: automatic)    */
    int                 rows_per_task;   /* window row-task size: 0 (automatic) or
                                            8..256; swr_autotune may change it   */
    int                 launch_mode;     /* swr_launch_mode                        */
    double              refine_res;      /* SWR_PREC_FP32_REFINED: Res(k) at or below which
                                            the iteration switches to the double-single
                                            step matrices; 0 selects 10 x the tolerance
                                            inside swr_iterate, else 1e-7 x the largest
                                            Res(k) so far                             */
    long long           spin_limit;      /* polls (about 64 ns each) before a device-side
                                            wait of the window kernels gives up and
                                            swr_step returns SWR_ETIMEOUT; 0 selects
                                            the default 2^24 (about one second);
                                            swr_set_spin_limit changes it later      */
    int                 contraction_path; /* swr_contraction                       */
    int                 cvtot_each_iteration; /* 1: every swr_step computes CVTOT
                                            (SWR_FIELD_CVTOT) and reports it in
                                            swr_iter_report.cvtot; 0: swr_get computes
                                            it for the last iteration on request   */
} swr_problem;

typedef struct swr_ctx swr_ctx;

/* Per Schwarz iteration (one call of swr_step). */
typedef struct swr_iter_report {
    int       k;                 /* Schwarz iteration index (1-based)              */
    double    res;               /* max over instances of Res(k)                   */
    int       window_max;        /* longest time window of this iteration          */
    long long subdomain_solves;  /* local step solves done in this iteration       */
    double    seconds;           /* device time of the iteration (CUDA events)     */
    double    cvtot;             /* max over instances of CVTOT(k) (SWR_FIELD_CVTOT)
                                    with cvtot_each_iteration, else -1            */
    int       fp32_matrices;     /* 1: this iteration used the FP32-rounded step
                                    matrices (SWR_PREC_FP32_REFINED before the switch) */
} swr_iter_report;

typedef struct swr_report {
    int       iterations;
    int       converged;         /* 1 when max_instance Res(k) <= tol              */
    double    res_last;
    long long subdomain_solves;
    double    seconds;
    int       fp32_iterations;   /* iterations run with the FP32-rounded step matrices
                                    (SWR_PREC_FP32_REFINED)                          */
} swr_report;

/* Device bytes the context needs (so the caller can pass them in as
 * swr_problem.workspace).  Fails with SWR_EINVAL on an invalid problem. */
swr_status swr_workspace_size(const swr_problem* p, size_t* bytes);

/* Validates and copies the problem, lays out device memory (the caller's
 * workspace when given, else cudaMalloc'ed and owned by the context), and
 * uploads the subdomain descriptors.  *out is NULL on failure. */
swr_status swr_setup(const swr_problem* p, swr_ctx** out);

/* Sec. 5.1: quadrature tables, local Galerkin matrices, orthonormalisation of
 * the local bases, step matrices (TISE: (I + dt H'), TDSE: I + i dt/2 H')
 * and their inverses, projection of phi0 (Sec. 6.1).  Once per problem.
 * SWR_ESINGULAR when an overlap matrix fails the Cholesky factorisation. */
swr_status swr_assemble(swr_ctx* ctx);

/* Exactly one Schwarz iteration over all subdomains of all instances:
 * time window of local solves (Sec. 5.4 step 2, 4), interface traces,
 * averaged Robin data for the next iteration, Res(k).  rep may be NULL. */
swr_status swr_step(swr_ctx* ctx, swr_iter_report* rep);

/* swr_step until max_instance Res(k) <= tol or kmax iterations.
 * res_history (nullable) receives up to kmax residuals.
 * Returns SWR_ENOTCONV (report filled) when tol is not reached. */
swr_status swr_iterate(swr_ctx* ctx, double tol, int kmax, swr_report* rep, double* res_history);

/* Changes the number of polls after which a device-side wait of the window
 * kernels gives up (swr_problem.spin_limit; 0 restores the default).  A step
 * that gives up returns SWR_ETIMEOUT and leaves the Robin data of that
 * iteration unusable: restore a checkpoint (swr_traces SET) before the next
 * swr_step to continue from a known state.                                  */
swr_status swr_set_spin_limit(swr_ctx* ctx, long long polls);

/* Interface-trace window of the last iteration (checkpoint / warm start). */
typedef enum swr_dir { SWR_GET = 0, SWR_SET = 1 } swr_dir;
typedef struct swr_trace_view {
    void*  host;      /* host buffer of `bytes` bytes                               */
    size_t bytes;     /* must equal swr_get(ctx, SWR_FIELD_TRACE_BYTES) on SET      */
} swr_trace_view;
swr_status swr_traces(swr_ctx* ctx, int dir, swr_trace_view* view);

/* Read-back of results into a HOST buffer of exactly the stated size. */
typedef enum swr_field {
    SWR_FIELD_ENERGY = 0,       /* double[n_instances]: PoU Rayleigh quotient (TISE)   */
    SWR_FIELD_NORM2 = 1,        /* double[n_instances]: PoU norm^2 of the last state   */
    SWR_FIELD_DIPOLE = 2,       /* double[n_instances]: <x_1 + ... + x_N> (TDSE)        */
    SWR_FIELD_RES = 3,          /* double[n_instances]: Res(k) of the last iteration   */
    SWR_FIELD_WINDOW = 4,       /* int[n_instances]: window length of the last iteration */
    SWR_FIELD_PSI_NODES = 5,    /* double (TISE) or double2 (TDSE) per volume node of
                                   every subdomain, subdomains in order, node
                                   p = q1 + q*q2 (q nodes per coordinate)            */
    SWR_FIELD_OWN_TRACES = 6,   /* u_i at the interface nodes for steps 0..window of
                                   the last iteration, layout [sub][step][node]       */
    SWR_FIELD_ROBIN = 7,        /* averaged Robin data g_i, same layout                */
    SWR_FIELD_TRACE_BYTES = 8,  /* size_t: bytes of the swr_traces window              */
    SWR_FIELD_NODE_COUNTS = 9,  /* int[3 * n_sub_total]: per subdomain (q, n_gamma, K) */
    SWR_FIELD_K_MAX = 10,       /* int: Schwarz iterations done so far                 */
    SWR_FIELD_COUNTERS = 11,    /* double[11], cumulative since swr_setup:
                                   [0] ms inside the time-window kernel (CUDA events on
                                       the context stream, one pair per launch),
                                   [1] launches of the time-window kernel,
                                   [2] kernel launches of the library (all kernels),
                                   [3] algorithmic flops of the window kernels
                                       (2 K^2 per local step solve in imaginary time;
                                       8 K^2 per matrix sweep, 1 + m sweeps per step,
                                       in real time),
                                   [4] algorithmic bytes of the window kernels
                                       (step-matrix bytes read per local step solve),
                                   [5] local step solves,
                                   [6] ms of swr_assemble (events), [7] ms of swr_step,
                                   [8] host->device bytes copied, [9] device->host bytes,
                                   [10] algorithmic step-matrix bytes of the window
                                       kernels: per real matrix element 8 (the FP64
                                       value or its FP32 hi/lo pair) or 4 (FP32-rounded
                                       matrix), per complex one 16 or 8; K^2 elements
                                       per local step solve (imaginary time) or per
                                       matrix sweep (real time)                     */
    SWR_FIELD_CVTOT = 12        /* double[n_instances]: interface mismatch of the last
                                   iteration, Eq. CVTOT (Sec. 4.1) / Eq. CVTOT2 (Sec. 4.2):
                                   the L2 norm in time (rectangle rule, weight dt at
                                   t_1..t_W) of the sum over ordered subdomain pairs (i, j)
                                   of ||psi_i - psi_j||_{L2(Gamma_ij)}, Gamma_ij the
                                   interface nodes of Omega_i inside closure(Omega_j), psi
                                   the normalised state.  Unlike Res(k) it does not tend to
                                   0: at the converged iterate it is the discretisation
                                   mismatch of neighbouring local solutions.  Computed
                                   on this request from the last iteration's line traces
                                   (they stay until the next swr_step), or in every
                                   iteration with swr_problem.cvtot_each_iteration      */
} swr_field;
swr_status swr_get(swr_ctx* ctx, int field, void* host, size_t bytes);

/* Bytes that swr_get needs for `field` (for the sized fields). */
swr_status swr_field_bytes(swr_ctx* ctx, int field, size_t* bytes);

/* ---- learned initial traces (not part of the paper's method) ---------------
 * The paper starts the Schwarz iteration from g^(0) = 0.  These entry points
 * let a caller start it from predicted Robin data instead.  A trace code is
 * the projection of each interior edge's Robin data onto discrete
 * orthonormal polynomials of degree < S along the edge (S = 1 for the point
 * edges of 1-electron problems) times degree < Tm in the step index; per
 * subdomain the code has 4 x 2 x S x Tm floats ([edge slot 2d+side][re, im]
 * [s][t], zero for absent edges and for the imaginary plane in imaginary
 * time).  Needs one fixed time window for all instances. */

/* Builds the bases for this context (after swr_assemble).  *floats_per_sub
 * receives 8*S*Tm.  1 <= S <= 16, 1 <= Tm <= 32. */
swr_status swr_trace_codec(swr_ctx* ctx, int S, int Tm, size_t* floats_per_sub);
/* Code of the Robin data of the last iteration into code_dev, a DEVICE array
 * of n_sub_total * floats_per_sub floats, subdomains in order. */
swr_status swr_trace_encode(swr_ctx* ctx, float* code_dev);
/* Decodes code_dev (device, same layout) into Robin data and the Robin
 * source b' that the next swr_step starts from (instead of zero traces). */
swr_status swr_trace_decode_set(swr_ctx* ctx, const float* code_dev);

/* Small BF16 multilayer perceptron trained with its own kernels (tanh hidden
 * layers, identity output, mean squared error, Adam); products on the
 * 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands staged in
 * shared memory, FP32 accumulator in tensor memory read back by tcgen05.ld),
 * FP32 master weights.  Parameters: for each layer l, W_l [d_l x d_{l+1}] row-major then
 * b_l [d_{l+1}], d = (n_in, width x n_hidden, n_out).  x, y, t are DEVICE
 * arrays [batch x dim] row-major FP32.  Not part of the paper. */
typedef struct swr_mlp swr_mlp;
swr_status  swr_mlp_create(int n_in, int width, int n_hidden, int n_out, void* stream, swr_mlp** out);
swr_status  swr_mlp_param_count(swr_mlp* mlp, size_t* n);
swr_status  swr_mlp_set_params(swr_mlp* mlp, const float* host, size_t n);  /* also resets Adam */
swr_status  swr_mlp_get_params(swr_mlp* mlp, float* host, size_t n);
swr_status  swr_mlp_forward(swr_mlp* mlp, const float* x_dev, int batch, float* y_dev);
/* One Adam step (lr > 0) or only gradients (lr == 0); loss_host / grad_host nullable. */
swr_status  swr_mlp_train_step(swr_mlp* mlp, const float* x_dev, const float* t_dev, int batch, float lr,
                               float* loss_host, float* grad_host);
void        swr_mlp_destroy(swr_mlp* mlp);
const char* swr_mlp_last_error(const swr_mlp* mlp);

/* Allocation-free recomputation of Res(k) of the last completed Schwarz
 * iteration, one value per instance into res_host[0..n) (n = n_instances).
 * No counterpart in the paper: this is a service for callers that may not
 * allocate device memory when they call it (for example code that runs under
 * a framework owning all device memory, or a real-time loop that forbids
 * allocation after start-up).  It calls no cudaMalloc/cudaFree and no
 * allocating library routine; its scratch (partial sums, window lengths,
 * result) lives in one file-scope __device__ array of 2 MiB, held by every
 * GPU that loads the library until the process exits, which limits it to
 * about 32,000 subdomains (SWR_EINVAL beyond that).  The first call on a
 * device resolves the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the array: calls
 * that overlap on the GPU (other streams, other contexts) race and must be
 * serialised by the caller.  Nothing in the array needs clearing: every call
 * overwrites all of the scratch it reads.  The device address is cached per
 * CUDA context: after cudaDeviceReset (or any other teardown of a device's
 * primary context) the next call resolves it again in the new context.
 * Synchronises the context stream.  Returns SWR_ESTATE unless a swr_step has
 * completed since the last swr_assemble or swr_traces(SET) (a restored state
 * has no residual of its own), or after a swr_step that failed; SWR_EINVAL
 * when n differs from the number of instances.  The result equals
 * swr_get(SWR_FIELD_RES) of the same iteration. */
swr_status swr_residual_noalloc(swr_ctx* ctx, double* res_host, size_t n);

/* ----------------------------------------------------------------------------
 * Window autotuner (no counterpart in the paper: a launch-configuration
 * choice).  Times every candidate (window variant x row-task size:
 * automatic, 16, 32, 64, 128, 256 rows; the fused variant only where its W was
 * allocated, i.e. when the problem was set up with window_variant 0 or 2) on
 * a fixed window of `steps` imaginary-time steps from the projected initial
 * data, twice each, and keeps the fastest for all later swr_step calls.
 * Call after swr_assemble and before the first swr_step (SWR_ESTATE
 * otherwise); real-time problems have no window kernel (SWR_EINVAL).  The
 * window state it writes is re-initialised by the first swr_step.  `out`
 * (may be NULL) receives the choice.                                         */
typedef struct swr_tune_report {
    int    variant;          /* swr_window_variant chosen                       */
    int    rows_per_task;    /* row-task target chosen                          */
    int    tasks;            /* row tasks of the chosen plan                    */
    int    ctas;             /* CTAs of the persistent launch                   */
    int    task_state_global;/* 1: per-task state in global memory             */
    int    candidates;       /* plans timed                                     */
    int    graph;            /* 1: iterations replay a captured CUDA graph      */
    double seconds_per_step; /* best time per window step                       */
    double seconds_default;  /* time per step of the plan before tuning         */
    int    tensor_contractions; /* 1: assembly runs the Gauss-Jordan updates and
                                   e-e products on the tensor cores             */
} swr_tune_report;
swr_status swr_autotune(swr_ctx* ctx, int steps, swr_tune_report* out);

/* The window plan in use (variant, rows_per_task, tasks, ctas,
 * task_state_global, graph, tensor_contractions; the timing fields are zero).  variant is 0 for
 * real-time problems, whose steps are launched from the host.               */
swr_status swr_window_plan(const swr_ctx* ctx, swr_tune_report* out);

/* ------------------------------------------------------------------------
 * Local orbitals and local Slater determinants: the paper's second basis
 * family (Sec. 3.2 "Local orbital construction" with the barrier potential
 * of Eq. BARPOT; Eq. LSD; Appendix A "Discrete local Hamiltonian
 * construction with local Slater's determinants"; Sec. 7 Test 1, Table 1).
 *
 * The line [box_lo, box_hi] is cut into L subdomains D_i of width
 * H + overlap (H = (box_hi - box_lo) / L, centre x_ci = box_lo + (i + 1/2) H).
 * In each D_i the M lowest eigenpairs of
 *   1/2 int a phi' psi' + int (V_en + V_b) phi psi = lambda int phi psi,
 *   V_b = v_inf s(|x - x_ci| - x_b),  a = 1 - s,  x_b = xb_factor (H + overlap),
 * s the C^2 step rising over [x_b - eps_b/2, x_b + eps_b/2], V_en soft-Coulomb
 * nuclei (-Z / sqrt((x - x_A)^2 + eta_en^2)) plus harmonic x^2 / 2, are
 * computed in a basis of kd Gaussians exp(-delta (x - alpha_k)^2), alpha_k
 * equally spaced on [x_ci - x_b, x_ci + x_b] (delta = 0: 1 / (2 h^2), h their
 * spacing), with composite Gauss-Legendre rules (q_p nodes per panel of width
 * <= panel).  Each orbital's sign makes int phi exp(0.37 (x - x_ci)) dx > 0.
 * The 2-D subdomain Omega_{i,j} (x1 in D_i, x2 in D_j, index i + L j) takes
 * the K determinants
 *   v = (phi_l^i(x1) phi_p^j(x2) - phi_l^i(x2) phi_p^j(x1)) / sqrt(2)
 * of lowest lambda_l^i + lambda_p^j (l < p when i = j; sums within 1e-9
 * relative are ties, broken by (l, p)).  All integrals run over the whole
 * line; the e-e interaction is ee_coef / sqrt((x1 - x2)^2 + eta_ee^2).
 * Everything is computed on the device in FP64 (one call; the device memory
 * it needs is allocated and freed inside).                                  */
typedef struct swr_lsd_problem {
    double box_lo, box_hi;
    int    L;                  /* 1-D subdomains, 1..16                         */
    double overlap;            /* overlap width of neighbouring D_i, >= 0       */
    int    n_nuclei;           /* 0..3                                          */
    double x_nuc[3], Z_nuc[3];
    double eta_en, eta_ee;     /* soft-Coulomb parameters (> 0)                 */
    double ee_coef;            /* e-e strength                                  */
    double harmonic;           /* harmonic term in V_en                         */
    int    M;                  /* orbitals per subdomain, 1..kd                 */
    int    K;                  /* determinants per Omega, 1..M (M - 1) / 2      */
    int    kd;                 /* Gaussians per orbital basis, 2..64            */
    double delta;              /* Gaussian exponent, 0: 1 / (2 h^2)             */
    double xb_factor;          /* x_b = xb_factor |D_i|, > 0                    */
    double eps_b;              /* width of the barrier's rise, > 0              */
    double v_inf;              /* barrier height, >= 0                          */
    int    q_p;                /* Gauss-Legendre nodes per panel, 2..16         */
    double panel;              /* panel width, > 0                              */
} swr_lsd_problem;

/* Caller-owned host buffers, row-major; orbital a = i M + l.                */
typedef struct swr_lsd_result {
    double* lam;               /* [L][M] lambda_l^i, ascending per subdomain    */
    double* coef;              /* [L][kd][M] Gaussian coefficients of phi_l^i    */
    double* S1;                /* [L M][L M] <phi_a, phi_b>                      */
    double* h1;                /* [L M][L M] 1/2 <phi_a', phi_b'> + <phi_a|V_en|phi_b> */
    double* J1;                /* [L M][L M] <phi_a|x|phi_b>                     */
    int*    pairs;             /* [L L][K][2] (l, p) of every determinant        */
    double* S_lsd;             /* [L L][K][K] Gram of the determinants of Omega  */
    double* H_lsd;             /* [L L][K][K] H0 between them                    */
    double* G_next;            /* [L L][K][K] <v of Omega_{i,j}, v of Omega_{i+1,j}>
                                  (zero for i = L - 1)                          */
} swr_lsd_result;

/* Builds everything above.  SWR_EINVAL for an invalid problem or a NULL
 * buffer, SWR_ENOMEM when the device memory cannot be had, SWR_ESINGULAR when
 * an orbital basis overlap is not positive definite, SWR_ECUDA on a runtime
 * error; details in swr_last_error(NULL).                                   */
swr_status swr_lsd_build(const swr_lsd_problem* p, swr_lsd_result* out);

void        swr_destroy(swr_ctx* ctx);
const char* swr_last_error(const swr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SWR_H */
