// swr_tdse.cu -- real-time time window (Crank-Nicolson under the dipole field).
//
// Sec. 5.4 step 2 (real time) with the Robin data of Sec. 5.1 and the
// length-gauge field of Sec. 1.2, in the orthonormal local basis (A' = I):
//   (I + i dt/2 (H' + e_{n+1} Q')) c^{n+1}
//       = (I - i dt/2 (H' + e_n Q')) c^n + i dt/2 kappa (b'^{n+1} + b'^n),
// H' = kappa (Kf' + mu R') + V' (complex through mu = mu_re + i mu_im),
// Q' = Xp' (+) Xp' (position in each coordinate, Kronecker sum).
// With M0 = I + i dt/2 H' inverted once at assembly (G0 = M0^{-1}) and
// theta_m = dt/2 e(t_m), a step is
//   r = 2 c^n + i (theta_{n+1} - theta_n) Q' c^n + i dt/2 kappa (b'^{n+1} + b'^n),
//   solve (M0 + i theta_{n+1} Q') x = r  by  x <- G0 (r - i theta_{n+1} Q' x),
//   c^{n+1} = x - c^n.
// The Hermitian part of M0 is I - (dt/2) kappa mu_im R' >= I for mu_im <= 0,
// so ||G0|| <= 1 and the fixed point contracts with
// rho <= (dt/2) max|e| max_{Omega_i}|x_1 + ... + x_N|; the host chooses the
// iteration count from rho so that rho^(m+1) <= 1e-15.
//
// Complex vectors are planar: [re block K][im block K].  G0 is interleaved
// (re, im) per element as the Gauss-Jordan inversion leaves it.
#include <math.h>

#include "swr_internal.cuh"

namespace swr {

#define CN_THREADS 256
#define CN_ROWS 256  // rows per CTA of the element-wise kernels (one per thread)
#define MV_ROWS 32   // rows per CTA of the complex matvec

__device__ inline double field_e(const InstDev& in, double t) {
    if (in.E0 == 0.0 || t < 0.0 || t > in.T) return 0.0;
    double s = sin(M_PI * t / in.T);
    return in.E0 * s * s * sin(in.omega * t + in.phase);
}

// (Q' x)[r] for rows r of one subdomain, x planar channel in shared memory,
// the first coordinate's factor transposed (X1t[c kd + a] = Xp1[a][c]: the
// lanes of a warp, consecutive rows, read consecutive words): FP64 for the
// plain FP64 path; for the mixed path factors and x as double-single pairs
// (the products on the FP32 pipes: this part's FP64 unit spends tens of
// microseconds per launch on them).
__device__ inline double qx_row(const SubDev& s, const double* X1t, const double* Xp2, const double* x, int r) {
    const int kd = s.kd;
    if (s.N == 1) {
        double acc = 0;
        for (int c = 0; c < kd; ++c) acc += X1t[c * kd + r] * x[c];
        return acc;
    }
    const int a = r % kd, b = r / kd;
    double acc = 0;
    for (int c = 0; c < kd; ++c) acc += X1t[c * kd + a] * x[c + kd * b];
    for (int e = 0; e < kd; ++e) acc += Xp2[b * kd + e] * x[a + kd * e];
    return acc;
}
__device__ inline double qx_row(const SubDev& s, const float2* X1t, const float2* Xp2, const float2* x, int r) {
    const int kd = s.kd;
    float h = 0.f, l = 0.f;
    if (s.N == 1) {
        for (int c = 0; c < kd; ++c) ds_fma(h, l, X1t[c * kd + r], x[c]);
        return dsp_to_double(dsp_norm(h, l));
    }
    const int a = r % kd, b = r / kd;
    for (int c = 0; c < kd; ++c) ds_fma(h, l, X1t[c * kd + a], x[c + kd * b]);
    for (int e = 0; e < kd; ++e) ds_fma(h, l, Xp2[b * kd + e], x[a + kd * e]);
    return dsp_to_double(dsp_norm(h, l));
}

// Antisymmetric states: the lower subdomain (i1 > i2) of a mirror pair is not
// stepped; its iterates are filled in as the mirror images of the upper one's
// after the window.
__device__ inline bool cn_mirror_skip(const SwrDeviceView& v, const SubDev& s) {
    const InstDev& in = v.inst[s.inst];
    return in.anti && s.N == 2 && s.idx[0] > s.idx[1];
}

struct CnBufs {
    long long r, u, x;   // per-subdomain planar vectors (offsets in doubles, 2K each)
};

// Shared-memory element of the element-wise kernels: FP64, or a double-single
// pair on the mixed path.
template <bool DS> struct CnElem { typedef double T; };
template <> struct CnElem<true> { typedef float2 T; };
template <bool DS> __device__ inline typename CnElem<DS>::T cn_elem(double x);
template <> __device__ inline double cn_elem<false>(double x) { return x; }
template <> __device__ inline float2 cn_elem<true>(double x) { return dsp_split_int(x); }

// dst[e] (TR: dst[(e % kd) kd + e / kd]) = src[e] for e < n, by the whole
// CTA: eight loads per thread in flight before the first store.
template <bool DS, bool TR>
__device__ inline void cn_stage(typename CnElem<DS>::T* dst, const double* src, int n, int kd) {
    for (int base = threadIdx.x; base < n; base += 8 * CN_THREADS) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = base + u * CN_THREADS;
            t[u] = e < n ? src[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = base + u * CN_THREADS;
            if (e < n) dst[TR ? (e % kd) * kd + e / kd : e] = cn_elem<DS>(t[u]);
        }
    }
}

// r = 2c^n + i dth Q' c^n + i hk (b^{n+1} + b^n);  u = r
template <bool DS>
__global__ void k_cn_rhs(SwrDeviceView v, const long long* boff, const int* win_prev, int n) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int K = s.K, kd = s.kd;
    const int r0 = blockIdx.x * CN_ROWS;
    if (r0 >= K || cn_mirror_skip(v, s)) return;
    typedef typename CnElem<DS>::T E;
    extern __shared__ double sm_raw[];
    E* c = reinterpret_cast<E*>(sm_raw);  // 2K
    E* X1 = c + 2 * K;                     // kd^2, transposed
    E* X2 = X1 + kd * kd;                  // kd^2
    T1Layout lay(s.q, kd);
    const double* cn = v.arena + s.hist + (long long)n * 2 * K;
    cn_stage<DS, false>(c, cn, 2 * K, kd);
    cn_stage<DS, true>(X1, v.arena + s.t1[0] + lay.mat(M_XP), kd * kd, kd);
    cn_stage<DS, false>(X2, v.arena + s.t1[s.N == 2 ? 1 : 0] + lay.mat(M_XP), kd * kd, kd);
    // the field at t_n and t_{n+1}: once per CTA (the FP64 sines of every
    // thread would take most of the launch on this part's FP64 unit)
    __shared__ double s_th[2];
    if (threadIdx.x == 0) {
        s_th[0] = 0.5 * in.dt * field_e(in, n * in.dt);
        s_th[1] = 0.5 * in.dt * field_e(in, (n + 1) * in.dt);
    }
    __syncthreads();
    const double th0 = s_th[0], th1 = s_th[1];
    const double dth = th1 - th0, hk = 0.5 * in.dt * in.kappa;
    const int wp = win_prev[s.inst];
    const double* b1 = (wp > 0) ? v.arena + s.bvec + (long long)min(n + 1, wp) * 2 * K : nullptr;
    const double* b0 = (wp > 0) ? v.arena + s.bvec + (long long)min(n, wp) * 2 * K : nullptr;
    double* R = v.arena + boff[3 * sid + 0];
    double* U = v.arena + boff[3 * sid + 1];
    for (int r = r0 + threadIdx.x; r < min(K, r0 + CN_ROWS); r += CN_THREADS) {
        const double qre = qx_row(s, X1, X2, c, r), qim = qx_row(s, X1, X2, c + K, r);
        double bre = 0, bim = 0;
        if (b1) {
            bre = b1[r] + b0[r];
            bim = b1[K + r] + b0[K + r];
        }
        const double rre = 2.0 * cn[r] - dth * qim - hk * bim;
        const double rim = 2.0 * cn[K + r] + dth * qre + hk * bre;
        R[r] = rre;
        R[K + r] = rim;
        U[r] = rre;
        U[K + r] = rim;
    }
}

// x = G0 u  (complex, FP64); one warp per row, lanes over the columns.
// need (nullable): fixed-point iterations of this step per subdomain; the
// launch of iteration m skips the subdomains that need no more than m.
__global__ void __launch_bounds__(256) k_cmv(SwrDeviceView v, const long long* boff, const unsigned char* need,
                                             int m) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K;
    const int r0 = blockIdx.x * MV_ROWS;
    if (r0 >= K || (need && m >= need[sid]) || cn_mirror_skip(v, s)) return;
    extern __shared__ double sm[];
    const double* U = v.arena + boff[3 * sid + 1];
    for (int e = threadIdx.x; e < 2 * K; e += blockDim.x) sm[e] = U[e];
    __syncthreads();
    const double2* G = (const double2*)(v.arena + s.Gm);
    double* X = v.arena + boff[3 * sid + 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = r0 + warp; r < min(K, r0 + MV_ROWS); r += nw) {
        const double2* g = G + (long long)r * K;
        double are = 0, aim = 0;
        for (int c = lane; c < K; c += 32) {
            const double2 gg = g[c];
            const double ur = sm[c], ui = sm[K + c];
            are = fma(gg.x, ur, fma(-gg.y, ui, are));
            aim = fma(gg.x, ui, fma(gg.y, ur, aim));
        }
        are = warp_sum(are);
        aim = warp_sum(aim);
        if (lane == 0) {
            X[r] = are;
            X[K + r] = aim;
        }
    }
}

// u = r - i theta_{n+1} Q' x  (fixed-point iteration m; the subdomains that
// need no more than m iterations at this step are skipped)
template <bool DS>
__global__ void k_cn_update(SwrDeviceView v, const long long* boff, int n, const unsigned char* need, int m) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int K = s.K, kd = s.kd;
    const int r0 = blockIdx.x * CN_ROWS;
    if (r0 >= K || m >= need[sid] || cn_mirror_skip(v, s)) return;
    typedef typename CnElem<DS>::T E;
    extern __shared__ double sm_raw[];
    E* x = reinterpret_cast<E*>(sm_raw);
    E* X1 = x + 2 * K;
    E* X2 = X1 + kd * kd;
    T1Layout lay(s.q, kd);
    const double* Xg = v.arena + boff[3 * sid + 2];
    cn_stage<DS, false>(x, Xg, 2 * K, kd);
    cn_stage<DS, true>(X1, v.arena + s.t1[0] + lay.mat(M_XP), kd * kd, kd);
    cn_stage<DS, false>(X2, v.arena + s.t1[s.N == 2 ? 1 : 0] + lay.mat(M_XP), kd * kd, kd);
    __shared__ double s_th1;
    if (threadIdx.x == 0) s_th1 = 0.5 * in.dt * field_e(in, (n + 1) * in.dt);  // once per CTA
    __syncthreads();
    const double th1 = s_th1;
    const double* R = v.arena + boff[3 * sid + 0];
    double* U = v.arena + boff[3 * sid + 1];
    for (int r = r0 + threadIdx.x; r < min(K, r0 + CN_ROWS); r += CN_THREADS) {
        const double qre = qx_row(s, X1, X2, x, r), qim = qx_row(s, X1, X2, x + K, r);
        U[r] = R[r] + th1 * qim;
        U[K + r] = R[K + r] - th1 * qre;
    }
}

__device__ inline void ds_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Double-single accumulation acc += g * x, g = (gh + gl), x = (xh + xl),
// products and sums error-free on the FP32 pipes.
__device__ inline void ds_mac(float& ah, float& al, float gh, float gl, float xh, float xl) {
    float p = gh * xh, e = fmaf(gh, xh, -p), s, q;
    ds_two_sum(ah, p, s, q);
    ah = s;
    al += (q + e) + fmaf(gh, xl, gl * xh);
}

// x = G0 u with G0 stored as four FP32 planes (re_hi, re_lo, im_hi, im_lo),
// rows of ld = df32_ld(K) columns (zero-padded, 16-byte aligned): complex
// double-single matvec, FP64-level accuracy on the FP32 pipes.  Each warp
// takes two rows at a time with 16-byte loads of every plane, so that eight
// independent 512-byte requests per warp are in flight.  ONEP: only the hi
// planes are read (the FP32-rounded G0 of SWR_PREC_FP32_REFINED before its
// switch, 8 bytes per complex element), their lo terms taken as 0.
template <bool ONEP>
__global__ void __launch_bounds__(256) k_cmv_df32(SwrDeviceView v, const long long* boff, const unsigned char* need,
                                                  int m) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, ld = df32_ld(K);
    const int r0 = blockIdx.x * MV_ROWS;
    if (r0 >= K || (need && m >= need[sid]) || cn_mirror_skip(v, s)) return;
    extern __shared__ float smf[];
    float* urh = smf;           // ld each
    float* url = smf + ld;
    float* uih = smf + 2 * ld;
    float* uil = smf + 3 * ld;
    const double* U = v.arena + boff[3 * sid + 1];
    for (int e = threadIdx.x; e < ld; e += blockDim.x) {
        const double a = e < K ? U[e] : 0.0, b = e < K ? U[K + e] : 0.0;
        const float ah = (float)a, bh = (float)b;
        urh[e] = ah;
        url[e] = (float)(a - (double)ah);
        uih[e] = bh;
        uil[e] = (float)(b - (double)bh);
    }
    __syncthreads();
    const long long KL = (long long)K * ld;
    const float* Grh = (const float*)(v.arena + s.Gf);
    const float* Grl = Grh + KL;
    const float* Gih = Grh + 2 * KL;
    const float* Gil = Grh + 3 * KL;
    double* X = v.arena + boff[3 * sid + 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int r1 = min(K, r0 + MV_ROWS);
    for (int rb = r0 + 2 * warp; rb < r1; rb += 2 * nw) {
        const int nrow = min(2, r1 - rb);
        // re = Gr ur - Gi ui ; im = Gr ui + Gi ur
        float reh[2] = {0.f, 0.f}, rel[2] = {0.f, 0.f}, imh[2] = {0.f, 0.f}, iml[2] = {0.f, 0.f};
        for (int c = lane * 4; c < ld; c += 128) {
            const float4 xrh = *reinterpret_cast<const float4*>(urh + c), xrl = *reinterpret_cast<const float4*>(url + c);
            const float4 xih = *reinterpret_cast<const float4*>(uih + c), xil = *reinterpret_cast<const float4*>(uil + c);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i < nrow) {
                    const long long o = (long long)(rb + i) * ld + c;
                    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 grh = *reinterpret_cast<const float4*>(Grh + o);
                    const float4 grl = ONEP ? zero4 : *reinterpret_cast<const float4*>(Grl + o);
                    const float4 gih = *reinterpret_cast<const float4*>(Gih + o);
                    const float4 gil = ONEP ? zero4 : *reinterpret_cast<const float4*>(Gil + o);
#define CMV_TERM(f)                                                   \
    ds_mac(reh[i], rel[i], grh.f, grl.f, xrh.f, xrl.f);               \
    ds_mac(reh[i], rel[i], -gih.f, -gil.f, xih.f, xil.f);             \
    ds_mac(imh[i], iml[i], grh.f, grl.f, xih.f, xil.f);               \
    ds_mac(imh[i], iml[i], gih.f, gil.f, xrh.f, xrl.f);
                    CMV_TERM(x)
                    CMV_TERM(y)
                    CMV_TERM(z)
                    CMV_TERM(w)
#undef CMV_TERM
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float sh, eh;
                float oh = __shfl_xor_sync(0xffffffffu, reh[i], o), ol = __shfl_xor_sync(0xffffffffu, rel[i], o);
                ds_two_sum(reh[i], oh, sh, eh);
                reh[i] = sh;
                rel[i] = rel[i] + ol + eh;
                oh = __shfl_xor_sync(0xffffffffu, imh[i], o);
                ol = __shfl_xor_sync(0xffffffffu, iml[i], o);
                ds_two_sum(imh[i], oh, sh, eh);
                imh[i] = sh;
                iml[i] = iml[i] + ol + eh;
            }
            if (lane == 0 && i < nrow) {
                X[rb + i] = (double)reh[i] + (double)rel[i];
                X[K + rb + i] = (double)imh[i] + (double)iml[i];
            }
        }
    }
}

// Complex G0 (interleaved doubles) -> four FP32 planes for the double-single matvec.
__global__ void k_split_c_df32(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, ld = df32_ld(K);
    const long long KL = (long long)K * ld;
    const double* G = v.arena + s.Gm;
    float* P = (float*)(v.arena + s.Gf);
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < KL; e += (long long)blockDim.x * gridDim.x) {
        const long long r = e / ld;
        const int c = (int)(e - r * ld);
        const double a = c < K ? G[2 * (r * K + c)] : 0.0, b = c < K ? G[2 * (r * K + c) + 1] : 0.0;
        const float ah = (float)a, bh = (float)b;
        P[e] = ah;
        P[KL + e] = (float)(a - (double)ah);
        P[2 * KL + e] = bh;
        P[3 * KL + e] = (float)(b - (double)bh);
    }
}

// c^{n+1} = x - c^n
__global__ void k_cn_finish(SwrDeviceView v, const long long* boff, int n) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    if (cn_mirror_skip(v, s)) return;
    const int K = s.K;
    const double* X = v.arena + boff[3 * sid + 2];
    const double* cn = v.arena + s.hist + (long long)n * 2 * K;
    double* cn1 = v.arena + s.hist + (long long)(n + 1) * 2 * K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * K; e += gridDim.x * blockDim.x) cn1[e] = X[e] - cn[e];
}

// c^0 into hist[0] (planar)
__global__ void k_cn_init(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K;
    const double* c0 = v.arena + s.c0;
    double* h0 = v.arena + s.hist;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * K; e += gridDim.x * blockDim.x) h0[e] = c0[e];
}

static inline unsigned div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Launches of one real-time window: n_steps steps, step n with as many
// fixed-point iterations as its neediest subdomain (h_need / d_need:
// [n_steps][n_sub] iteration counts, host and device copies); returns the
// number of kernel launches.
cudaError_t launch_split_c_df32(const SwrDeviceView& v, cudaStream_t st, int max_K) {
    long long kk = (long long)max_K * df32_ld(max_K);
    k_split_c_df32<<<dim3((unsigned)((kk + 2047) / 2048), v.n_sub), 256, 0, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_tdse_window(const SwrDeviceView& v, cudaStream_t st, const long long* d_boff, const int* d_win_prev,
                               int n_steps, const unsigned char* h_need, const unsigned char* d_need, int max_K,
                               int max_kd, bool df32, bool onep, long long* launches) {
    const size_t sm_el = (2 * (size_t)max_K + 2 * (size_t)max_kd * max_kd) * sizeof(double);
    const size_t sm_mv = 2 * (size_t)df32_ld(max_K) * sizeof(double);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_cn_rhs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cn_rhs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cn_update<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cn_update<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cmv, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cmv_df32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_cmv_df32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_done = true;
    }
    const dim3 ge(div_up(max_K, CN_ROWS), v.n_sub), gm(div_up(max_K, MV_ROWS), v.n_sub), gf(div_up(2 * max_K, 256), v.n_sub);
    long long nl = 0;
    k_cn_init<<<gf, 256, 0, st>>>(v);
    ++nl;
    for (int n = 0; n < n_steps; ++n) {
        const unsigned char* nd = d_need + (size_t)n * v.n_sub;
        int iters = 0;
        for (int s = 0; s < v.n_sub; ++s) iters = h_need[(size_t)n * v.n_sub + s] > iters ? h_need[(size_t)n * v.n_sub + s] : iters;
        if (df32) k_cn_rhs<true><<<ge, CN_THREADS, sm_el, st>>>(v, d_boff, d_win_prev, n);
        else k_cn_rhs<false><<<ge, CN_THREADS, sm_el, st>>>(v, d_boff, d_win_prev, n);
        if (df32 && onep) k_cmv_df32<true><<<gm, 256, sm_mv, st>>>(v, d_boff, nullptr, 0);
        else if (df32) k_cmv_df32<false><<<gm, 256, sm_mv, st>>>(v, d_boff, nullptr, 0);
        else k_cmv<<<gm, 256, sm_mv, st>>>(v, d_boff, nullptr, 0);
        for (int m = 0; m < iters; ++m) {
            if (df32) k_cn_update<true><<<ge, CN_THREADS, sm_el, st>>>(v, d_boff, n, nd, m);
            else k_cn_update<false><<<ge, CN_THREADS, sm_el, st>>>(v, d_boff, n, nd, m);
            if (df32 && onep) k_cmv_df32<true><<<gm, 256, sm_mv, st>>>(v, d_boff, nd, m);
            else if (df32) k_cmv_df32<false><<<gm, 256, sm_mv, st>>>(v, d_boff, nd, m);
            else k_cmv<<<gm, 256, sm_mv, st>>>(v, d_boff, nd, m);
        }
        k_cn_finish<<<gf, 256, 0, st>>>(v, d_boff, n);
        nl += 3 + 2 * iters;
    }
    *launches = nl;
    return cudaGetLastError();
}

}  // namespace swr
