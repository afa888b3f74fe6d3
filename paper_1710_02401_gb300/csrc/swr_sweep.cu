// swr_sweep.cu -- one Schwarz iteration over all subdomains on sm_103a.
//
// The time window itself runs in swr_window.cu.  After the window: line traces (psi and d psi at the 4 line positions of
// every subdomain coordinate), the averaged Robin data of Sec. 5.1 for every
// interface node, the Robin source b' of the next iteration, the own interface
// traces and Res(k) (Eq. residueIT), and the energy.
#include <math.h>
#include <stdio.h>

#include "swr_internal.cuh"

namespace swr {

#define WARPS_MAX 32

__device__ inline double block_sum(double x, double* red) {
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = x;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Deterministic sum of the partials of one instance (fixed task order).
__device__ inline double inst_sum(const double* part, int t0, int t1, double* red) {
    double x = 0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) x += __ldcg(part + t);
    // fixed reduction tree: thread order is deterministic for a fixed blockDim
    return block_sum(x, red);
}

// ---------------------------------------------------------------- traces
//
// Per-step vectors are planar over nch channels: nch = 1 (imaginary time,
// real) or 2 (real time: real plane then imaginary plane).  Everything below
// is linear in the coefficients, so the complex case runs the real arithmetic
// on each plane and combines the planes only where mu is complex.

__device__ inline int n_channels(const InstDev& in) { return in.mode == SWR_MODE_TDSE ? 2 : 1; }

// Line traces of subdomain j at step n from the un-normalised iterate y^n:
// N = 2: [d][l][kind][q] with psi (kind 0) and d_{x_d} psi (kind 1) on the line
// x_d = pos_l, sampled at the nodes of the other coordinate.  N = 1: [l][kind].
// The two contractions (line values of one coordinate against Y, then the
// other coordinate's node values) run in double-single on the FP32 pipes; the
// subdomain's line and node tables are staged once per CTA as FP32 pairs
// (from global memory when they do not fit, `staged` = 0).  Shared-memory
// layouts avoid bank conflicts: Y with an odd column stride (kd + 1), the node
// tables transposed (node index fastest).
// Dynamic shared memory (float2): ys[kmax + kdmax] | r[16 kdmax] | Lt[2][8][kdmax] | Bt[2][kdmax][qmax] (staged)
__global__ void k_line_traces(SwrDeviceView v, const int* win, int cap, int kmax, int kdmax, int qmax, int staged) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int W = win[s.inst], nch = n_channels(in);
    const int kd = s.kd, q = s.q, K = s.K;
    T1Layout lay(q, kd);
    extern __shared__ float2 ls[];
    float2* ys = ls;
    float2* r = ys + kmax + kdmax;
    float2* Lt = r + 16 * kdmax;
    float2* Bt = Lt + 2 * 8 * kdmax;
    if (s.N == 2) {
        for (int e = threadIdx.x; e < 2 * 8 * kd; e += blockDim.x) {  // Lt[d][2 l + kind][a]
            const int d = e / (8 * kd), rest = e % (8 * kd), lk = rest / kd, a = rest % kd;
            const double* T = v.arena + s.t1[d];
            Lt[e] = ds_split(T[((lk & 1) ? lay.Ld() : lay.Lv()) + (lk >> 1) * kd + a]);
        }
        if (staged)
            for (int e = threadIdx.x; e < 2 * q * kd; e += blockDim.x) {  // Bt[d][m][node] = B_d[node][m]
                const int d = e / (q * kd), rest = e % (q * kd), node = rest / kd, m = rest % kd;
                Bt[(d * kd + m) * q + node] = ds_split(v.arena[s.t1[d] + lay.B() + rest]);
            }
    }
    __syncthreads();
    for (int item = blockIdx.x; item <= W * nch + nch - 1; item += gridDim.x) {
        const int n = item / nch, ch = item % nch;
        const double* y = v.arena + s.hist + ((long long)n * nch + ch) * K;
        double* out = v.arena + s.line + ((long long)n * nch + ch) * s.nline;
        if (s.N == 1) {
            const double* T = v.arena + s.t1[0];
            for (int e = threadIdx.x; e < 8; e += blockDim.x) {
                int l = e / 2, kind = e % 2;
                const double* Lr = T + (kind ? lay.Ld() : lay.Lv()) + l * kd;
                double acc = 0;
                for (int a = 0; a < kd; ++a) acc += Lr[a] * y[a];
                out[l * 2 + kind] = acc;
            }
            continue;
        }
        for (int c = threadIdx.x; c < K; c += blockDim.x) ys[c + c / kd] = dsp_split_int(y[c]);  // (a, b) at a + (kd+1) b
        __syncthreads();
        // two combinations (lines 2p and 2p+1 of one coordinate) per thread: the
        // Y element loaded once for both, two independent chains
        for (int e = threadIdx.x; e < 8 * kd; e += blockDim.x) {
            const int pc = e / kd, m = e - pc * kd;
            const int d = pc / 4;
            const float2* L0 = Lt + (2 * pc) * kd;
            const float2* L1 = L0 + kd;
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
            if (d == 0) {  // r[b] = sum_a L1[a] Y[a][b]
#pragma unroll 4
                for (int a = 0; a < kd; ++a) {
                    const float2 yv = ys[a + (kd + 1) * m];
                    ds_fma(h0, l0, L0[a], yv);
                    ds_fma(h1, l1, L1[a], yv);
                }
            } else {       // r[a] = sum_b Y[a][b] L2[b]
#pragma unroll 4
                for (int b = 0; b < kd; ++b) {
                    const float2 yv = ys[m + (kd + 1) * b];
                    ds_fma(h0, l0, L0[b], yv);
                    ds_fma(h1, l1, L1[b], yv);
                }
            }
            float hs = h0 + l0;  // renormalised pairs
            r[(2 * pc) * kd + m] = make_float2(hs, l0 - (hs - h0));
            hs = h1 + l1;
            r[(2 * pc + 1) * kd + m] = make_float2(hs, l1 - (hs - h1));
        }
        __syncthreads();
        // two combinations of one coordinate per thread against one node row
        for (int e = threadIdx.x; e < 8 * q; e += blockDim.x) {
            const int pc = e / q, node = e - pc * q;
            const int d = pc / 4;
            const float2* rc0 = r + (2 * pc) * kd;
            const float2* rc1 = rc0 + kd;
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
            if (staged) {
                const float2* Bo = Bt + (1 - d) * kd * q + node;
#pragma unroll 4
                for (int m = 0; m < kd; ++m) {
                    const float2 bv = Bo[m * q];
                    ds_fma(h0, l0, bv, rc0[m]);
                    ds_fma(h1, l1, bv, rc1[m]);
                }
            } else {
                const double* Bo = v.arena + s.t1[1 - d] + lay.B() + (long long)node * kd;
                for (int m = 0; m < kd; ++m) {
                    const float2 bv = ds_split(Bo[m]);
                    ds_fma(h0, l0, bv, rc0[m]);
                    ds_fma(h1, l1, bv, rc1[m]);
                }
            }
            out[(2 * pc) * q + node] = (double)h0 + (double)l0;
            out[(2 * pc + 1) * q + node] = (double)h1 + (double)l1;
        }
        __syncthreads();
    }
}

// Edge slot (2*d + side) and tangential node of interface node `node`.
__device__ inline void gamma_slot(const SubDev& s, int node, int& slot, int& nt) {
    slot = -1;
    nt = 0;
    for (int sl = 3; sl >= 0; --sl)
        if (s.gam_off[sl] >= 0 && node >= s.gam_off[sl]) {
            slot = sl;
            nt = node - s.gam_off[sl];
            return;
        }
}

// Averaged Robin data g_i and own traces u_i at the interface nodes of every
// subdomain for steps 0..W, and the Robin source b'_i of the next iteration.
// The tangential sums of b' run in double-single on the FP32 pipes over the
// weighted node tables WB_d[t][m] = w_t B_d[t][m], staged once per CTA in
// shared memory as pairs when they fit (`staged`), each sum split into
// GATHER_SPLIT chunks added in a fixed order; b' is written in FP64.
#define GATHER_SPLIT 4
__global__ void k_gather(SwrDeviceView v, const int* win, const double* snorm, int cap, int parity, int staged,
                         int gsz) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int W = win[s.inst], nch = n_channels(in);
    const int kd = s.kd, q = s.q, K = s.K, L = in.L, qp = in.q_p;
    T1Layout lay(q, kd);
    __shared__ float2 hsum[4][64];
    __shared__ float2 hpart[GATHER_SPLIT][4][64];
    __shared__ float2 lvt[2][2][64];     // Lv rows l = 0, 3 of both coordinates as pairs
    // dynamic: the step's Robin data as pairs for the b' sums [2][gsz] (gsz >= the
    // interface nodes of any subdomain), then the staged tables [2][q][kd]; sized
    // to the problem so that several CTAs share an SM
    extern __shared__ float2 gdyn[];
    float2* gs2 = gdyn;
    float2* wbs = gdyn + 2 * gsz;
    if (s.N == 2) {
        if (staged)
            for (int e = threadIdx.x; e < 2 * q * kd; e += blockDim.x) {
                const int d = e / (q * kd), rest = e % (q * kd), t = rest / kd;
                const double* To = v.arena + s.t1[d];
                wbs[e] = dsp_split_int(To[lay.w() + t] * To[lay.B() + rest]);
            }
        for (int e = threadIdx.x; e < 2 * 2 * kd; e += blockDim.x) {
            const int d = e / (2 * kd), li = (e / kd) & 1, a = e % kd;
            lvt[d][li][a] = dsp_split_int(v.arena[s.t1[d] + lay.Lv() + (li ? 3 : 0) * kd + a]);
        }
        __syncthreads();
    }
    for (int n = blockIdx.x; n <= W; n += gridDim.x) {
        // one FP64 division per step and CTA (per thread it would keep this
        // part's FP64 unit busy for a good share of the kernel)
        __shared__ double s_isn;
        if (threadIdx.x == 0) s_isn = 1.0 / (in.normalize ? snorm[(long long)s.inst * (cap + 1) + n] : 1.0);
        __syncthreads();
        const double isn = s_isn;
        for (int node = threadIdx.x; node < s.ngam; node += blockDim.x) {
            int slot, nt;
            gamma_slot(s, node, slot, nt);
            const int d = slot / 2, side = slot % 2;
            const double sig = side ? 1.0 : -1.0;
            const int lown = side ? 3 : 0;
            double val[2] = {0, 0}, der[2] = {0, 0}, own[2] = {0, 0};
            int cnt = 0;
            for (int ch = 0; ch < nch; ++ch) {
                const double* lo = v.arena + s.line + ((long long)n * nch + ch) * s.nline;
                own[ch] = (s.N == 1) ? lo[lown * 2 + 0] : lo[((d * 4 + lown) * 2 + 0) * q + nt];
            }
            // contributors: the neighbour across the edge and the same column, times
            // the tangential set (own index, plus the overlap neighbour in the bands)
            const int kdn = s.idx[d];
            const int across = kdn + (side ? 1 : -1);
            if (s.N == 1) {
                const int j = in.sub_base + across;
                const int l = side ? 1 : 2;
                for (int ch = 0; ch < nch; ++ch) {
                    const double* lj = v.arena + v.sub[j].line + ((long long)n * nch + ch) * v.sub[j].nline;
                    val[ch] += lj[l * 2 + 0];
                    der[ch] += lj[l * 2 + 1];
                }
                cnt = 1;
            } else {
                const int o = 1 - d;
                const int ko = s.idx[o];
                const int pt = nt / qp, npan = in.n_mid + 2;
                int jo_list[3], shift[3], njo = 0;
                jo_list[njo] = ko; shift[njo++] = 0;
                if (pt == 0 && ko > 0) { jo_list[njo] = ko - 1; shift[njo++] = q - qp; }
                if (pt == npan - 1 && ko < L - 1) { jo_list[njo] = ko + 1; shift[njo++] = -(q - qp); }
                for (int jd_i = 0; jd_i < 2; ++jd_i) {
                    const int jd = jd_i ? across : kdn;
                    for (int t = 0; t < njo; ++t) {
                        const int jo = jo_list[t];
                        if (jd == kdn && jo == ko) continue;
                        int j1 = d == 0 ? jd : jo, j2 = d == 0 ? jo : jd;
                        const int j = in.sub_base + j1 + L * j2;
                        const int l = (jd == kdn) ? lown : (side ? 1 : 2);
                        const int nj = nt + shift[t];
                        for (int ch = 0; ch < nch; ++ch) {
                            const double* lj = v.arena + v.sub[j].line + ((long long)n * nch + ch) * v.sub[j].nline;
                            val[ch] += lj[((d * 4 + l) * 2 + 0) * q + nj];
                            der[ch] += lj[((d * 4 + l) * 2 + 1) * q + nj];
                        }
                        ++cnt;
                    }
                }
            }
            // 1/cnt for the contributor counts that occur (1 to 3: constants)
            const double inv = cnt == 1 ? 1.0 : cnt == 2 ? 0.5 : cnt == 3 ? 1.0 / 3.0 : 1.0 / (double)cnt;
            // g = (n.grad + mu) psi_j averaged (Robin), or mu psi_j (classical SWR by
            // penalty); complex mu mixes the planes
            const double sd = in.tc == SWR_TC_DIRICHLET ? 0.0 : sig;
            double gre = (sd * der[0] + in.mu_re * val[0] - in.mu_im * val[1]) * inv;
            double gim = (sd * der[1] + in.mu_re * val[1] + in.mu_im * val[0]) * inv;
            for (int ch = 0; ch < nch; ++ch) {
                const double gv = ch ? gim : gre;
                v.arena[s.u[parity] + ((long long)n * nch + ch) * s.ngam + node] = own[ch] * isn;
                v.arena[s.g + ((long long)n * nch + ch) * s.ngam + node] = gv;
                gs2[ch * gsz + node] = dsp_split_int(gv);
            }
        }
        __syncthreads();
        // b'[a + kd b] for this step, one plane per channel
        for (int ch = 0; ch < nch; ++ch) {
            double* bdst = v.arena + s.bvec + ((long long)n * nch + ch) * K;
            if (s.N == 1) {
                const double* T = v.arena + s.t1[0];
                for (int a = threadIdx.x; a < kd; a += blockDim.x) {
                    double acc = 0;
                    for (int sl = 0; sl < 2; ++sl) {
                        if (s.gam_off[sl] < 0) continue;
                        int l = sl ? 3 : 0;
                        acc += v.arena[s.g + ((long long)n * nch + ch) * s.ngam + s.gam_off[sl]] *
                               T[lay.Lv() + l * kd + a];
                    }
                    bdst[a] = acc;
                }
            } else {
                const int chunk = (q + GATHER_SPLIT - 1) / GATHER_SPLIT;
                for (int e = threadIdx.x; e < GATHER_SPLIT * 4 * kd; e += blockDim.x) {
                    const int part = e / (4 * kd), rest = e % (4 * kd), sl = rest / kd, m = rest % kd;
                    float2 acc = make_float2(0.f, 0.f);
                    if (s.gam_off[sl] >= 0) {
                        const int d = sl / 2, t0 = part * chunk, t1 = min(q, t0 + chunk);
                        const float2* gv = gs2 + ch * gsz + s.gam_off[sl];
                        if (staged) {
                            const float2* wb = wbs + (long long)(1 - d) * q * kd;
                            for (int t = t0; t < t1; ++t) ds_fma(acc.x, acc.y, gv[t], wb[t * kd + m]);
                        } else {
                            const double* To = v.arena + s.t1[1 - d];
                            for (int t = t0; t < t1; ++t)
                                ds_fma(acc.x, acc.y, gv[t], dsp_split_int(To[lay.w() + t] * To[lay.B() + t * kd + m]));
                        }
                    }
                    hpart[part][sl][m] = dsp_norm(acc.x, acc.y);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < 4 * kd; e += blockDim.x) {
                    const int sl = e / kd, m = e % kd;
                    float2 acc = make_float2(0.f, 0.f);
                    for (int part = 0; part < GATHER_SPLIT; ++part) acc = dsp_add(acc, hpart[part][sl][m]);
                    hsum[sl][m] = acc;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < K; e += blockDim.x) {
                    int a = e % kd, b = e / kd;
                    float2 acc = make_float2(0.f, 0.f);
                    for (int sl = 0; sl < 4; ++sl) {
                        if (s.gam_off[sl] < 0) continue;
                        const int d = sl / 2, li = sl % 2;
                        if (d == 0) ds_fma(acc.x, acc.y, lvt[0][li][a], hsum[sl][b]);
                        else ds_fma(acc.x, acc.y, hsum[sl][a], lvt[1][li][b]);
                    }
                    bdst[e] = dsp_to_double(acc);
                }
            }
            __syncthreads();
        }
    }
}

// Res(k)^2 partials: sum_{n=1}^{max(W, Wp)} dt sum_nodes w |u^(k) - u^(k-1)|^2 with
// hold-last indexing; u^(0) = 0.  One partial per (subdomain, block).
__global__ void k_residual(SwrDeviceView v, const int* win, const int* win_prev, int parity, int first_iter,
                           double* part) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int nch = n_channels(in);
    const int W = win[s.inst], Wp = first_iter ? 0 : win_prev[s.inst];
    const int Nn = max(W, Wp);
    const int q = s.q, kd = s.kd;
    T1Layout lay(q, kd);
    __shared__ double red[33];
    double acc = 0;
    // 32-bit indices (Nn * ngam stays far below 2^31: windows of at most a few
    // thousand steps, at most 4 q interface nodes)
    const int total = Nn * s.ngam, ng = s.ngam;
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < total; e += blockDim.x * gridDim.x) {
        const int n = 1 + e / ng, node = e - (n - 1) * ng;
        double w = 1.0;
        if (s.N == 2) {
            int slot, nt;
            gamma_slot(s, node, slot, nt);
            const double* To = v.arena + s.t1[1 - slot / 2];
            w = To[lay.w() + nt];
        }
        for (int ch = 0; ch < nch; ++ch) {
            double a = v.arena[s.u[parity] + ((long long)min(n, W) * nch + ch) * s.ngam + node];
            double b = first_iter ? 0.0
                                  : v.arena[s.u[parity ^ 1] + ((long long)min(n, Wp) * nch + ch) * s.ngam + node];
            acc += in.dt * w * (a - b) * (a - b);
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[sid * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_residual_reduce(SwrDeviceView v, const double* part, int nblk, double* res) {
    const int i = blockIdx.x;
    const InstDev& in = v.inst[i];
    __shared__ double red[33];
    double acc = 0;
    for (int e = threadIdx.x; e < in.n_sub * nblk; e += blockDim.x) acc += part[(long long)in.sub_base * nblk + e];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) res[i] = sqrt(acc);
}

// CVTOT (Eq. CVTOT, Sec. 4.1; Eq. CVTOT2, Sec. 4.2) of one instance:
// CVTOT^2 = sum_{n=1}^{W} dt C_n^2, C_n = sum over ordered pairs (i, j) of
// ||psi_i - psi_j||_{L2(Gamma_{i;j})} at t_n, Gamma_{i;j} = the interface
// nodes of Omega_i that lie in closure(Omega_j) (the contributors of the
// averaged Robin data), psi the normalised state (y^n / s_n).  The pair
// (i, j) is identified by the offset of j in the 3 x 3 block around i
// (slot (j1 - i1 + 1) + 3 (j2 - i2 + 1)).  Grid (CV_BLOCKS, n_inst): block b
// takes steps n = 1 + b, 1 + b + CV_BLOCKS, ...; within a step, warp w takes
// the subdomains w, w + 8, ... (lanes over interface nodes, one register
// accumulator per slot, shuffle sums), and the warps' sums of C_i are added
// in warp order: a fixed order, so the result is deterministic.  The block's
// partial of sum_n dt C_n^2 goes to part[inst * CV_BLOCKS + b].
#define CV_BLOCKS 512
__global__ void __launch_bounds__(256) k_cvtot(SwrDeviceView v, const int* win, const double* snorm, int cap,
                                               double* part) {
    const int ii = blockIdx.y;
    const InstDev& in = v.inst[ii];
    const int W = win[ii], nch = n_channels(in), L = in.L, qp = in.q_p;
    __shared__ double wsum[WARPS_MAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double acc_t = 0;  // thread 0: sum over this block's steps of dt C_n^2
    for (int n = 1 + blockIdx.x; n <= W; n += gridDim.x) {
        double c_w = 0;  // this warp's sum of C_i over its subdomains
        for (int loc = wid; loc < in.n_sub; loc += nw) {
            const SubDev& s = v.sub[in.sub_base + loc];
            const int q = s.q, kd = s.kd;
            T1Layout lay(q, kd);
            double a[9];
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) a[sl] = 0.0;
            for (int node = lane; node < s.ngam; node += 32) {
                int slot, nt;
                gamma_slot(s, node, slot, nt);
                const int d = slot / 2, side = slot % 2;
                const int lown = side ? 3 : 0;
                double own[2] = {0, 0};
                for (int ch = 0; ch < nch; ++ch) {
                    const double* lo = v.arena + s.line + ((long long)n * nch + ch) * s.nline;
                    own[ch] = (s.N == 1) ? lo[lown * 2 + 0] : lo[((d * 4 + lown) * 2 + 0) * q + nt];
                }
                const int kdn = s.idx[d];
                const int across = kdn + (side ? 1 : -1);
                if (s.N == 1) {
                    const int j = in.sub_base + across;
                    const int l = side ? 1 : 2;
                    double e2 = 0;
                    for (int ch = 0; ch < nch; ++ch) {
                        const double* lj = v.arena + v.sub[j].line + ((long long)n * nch + ch) * v.sub[j].nline;
                        const double df = own[ch] - lj[l * 2 + 0];
                        e2 += df * df;
                    }
                    const int sl = across - kdn + 1;
#pragma unroll
                    for (int t = 0; t < 9; ++t) a[t] += (t == sl) ? e2 : 0.0;
                } else {
                    const int o = 1 - d;
                    const int ko = s.idx[o];
                    const double w = v.arena[s.t1[o] + lay.w() + nt];
                    const int pt = nt / qp, npan = in.n_mid + 2;
                    int jo_list[3], shift[3], njo = 0;
                    jo_list[njo] = ko; shift[njo++] = 0;
                    if (pt == 0 && ko > 0) { jo_list[njo] = ko - 1; shift[njo++] = q - qp; }
                    if (pt == npan - 1 && ko < L - 1) { jo_list[njo] = ko + 1; shift[njo++] = -(q - qp); }
                    for (int jd_i = 0; jd_i < 2; ++jd_i) {
                        const int jd = jd_i ? across : kdn;
                        for (int t = 0; t < njo; ++t) {
                            const int jo = jo_list[t];
                            if (jd == kdn && jo == ko) continue;
                            const int j1 = d == 0 ? jd : jo, j2 = d == 0 ? jo : jd;
                            const int j = in.sub_base + j1 + L * j2;
                            const int l = (jd == kdn) ? lown : (side ? 1 : 2);
                            const int nj = nt + shift[t];
                            double e2 = 0;
                            for (int ch = 0; ch < nch; ++ch) {
                                const double* lj = v.arena + v.sub[j].line + ((long long)n * nch + ch) * v.sub[j].nline;
                                const double df = own[ch] - lj[((d * 4 + l) * 2 + 0) * q + nj];
                                e2 += df * df;
                            }
                            const int sl = (j1 - s.idx[0] + 1) + 3 * (j2 - s.idx[1] + 1);
#pragma unroll
                            for (int u = 0; u < 9; ++u) a[u] += (u == sl) ? w * e2 : 0.0;
                        }
                    }
                }
            }
            double c_i = 0;
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) c_i += sqrt(warp_sum(a[sl]));
            c_w += c_i;
        }
        if (lane == 0) wsum[wid] = c_w;
        __syncthreads();
        if (threadIdx.x == 0) {
            double c_n = 0;
            for (int u = 0; u < nw; ++u) c_n += wsum[u];
            const double cs = c_n / (in.normalize ? snorm[(long long)ii * (cap + 1) + n] : 1.0);
            acc_t += in.dt * cs * cs;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)ii * gridDim.x + blockIdx.x] = acc_t;
}

__global__ void k_cvtot_reduce(int n_inst, const double* part, int nblk, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    double acc = 0;
    for (int b = 0; b < nblk; ++b) acc += part[(long long)i * nblk + b];
    out[i] = sqrt(acc);
}

// Per subdomain at step W (normalised state): sums over the volume nodes of
// w chi (kappa |grad psi|^2 + V |psi|^2), w chi |psi|^2 and w chi (x_1+..+x_N)|psi|^2,
// and psi at the nodes (node p = q1 + q*q2; re, im interleaved in real time).
// Energy partials of one subdomain split over ENERGY_BLOCKS blocks: block b
// takes the quadrature nodes of the last coordinate in
// [b q / ENERGY_BLOCKS, (b+1) q / ENERGY_BLOCKS) (and, N = 2, only the columns
// of the first contraction those nodes need); partial (sid, b) at
// part[3 (sid ENERGY_BLOCKS + b)].
__global__ void k_energy(SwrDeviceView v, const int* win, const double* snorm, int cap, double* part,
                         double* psi_out, const long long* psi_off) {
    const int sid = blockIdx.y, blk = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int W = win[s.inst], nch = n_channels(in);
    const int kd = s.kd, q = s.q, K = s.K;
    T1Layout lay(q, kd);
    const double sn = in.normalize ? snorm[(long long)s.inst * (cap + 1) + W] : 1.0;
    extern __shared__ double sm[];
    double* ys = sm;               // K
    double* G1 = sm + K;           // kd * q
    double* G1d = G1 + kd * q;     // kd * q
    __shared__ double red[33];
    const double* T0 = v.arena + s.t1[0];
    double num = 0, den = 0, dip = 0;
    for (int ch = 0; ch < nch; ++ch) {
        const double* y = v.arena + s.hist + ((long long)W * nch + ch) * K;
        for (int c = threadIdx.x; c < K; c += blockDim.x) ys[c] = y[c] / sn;
        __syncthreads();
        if (s.N == 1) {
            const int n_lo = blk * q / ENERGY_BLOCKS, n_hi = (blk + 1) * q / ENERGY_BLOCKS;
            for (int n = n_lo + threadIdx.x; n < n_hi; n += blockDim.x) {
                double p = 0, dp = 0;
                for (int a = 0; a < kd; ++a) {
                    p += T0[lay.B() + n * kd + a] * ys[a];
                    dp += T0[lay.D() + n * kd + a] * ys[a];
                }
                double wc = T0[lay.w() + n] * T0[lay.chi() + n];
                num += wc * (in.kappa * dp * dp + T0[lay.v1() + n] * p * p);
                den += wc * p * p;
                dip += wc * T0[lay.x() + n] * p * p;
                if (psi_out) psi_out[(psi_off[sid] + n) * nch + ch] = p;
            }
        } else {
            const double* T1 = v.arena + s.t1[1];
            const int n2_lo = blk * q / ENERGY_BLOCKS, n2_hi = (blk + 1) * q / ENERGY_BLOCKS, nw = n2_hi - n2_lo;
            for (int e = threadIdx.x; e < kd * nw; e += blockDim.x) {
                int a = e / nw, n2 = n2_lo + e % nw;
                double acc = 0, accd = 0;
                for (int b = 0; b < kd; ++b) {
                    double c = ys[a + kd * b];
                    acc += c * T1[lay.B() + n2 * kd + b];
                    accd += c * T1[lay.D() + n2 * kd + b];
                }
                G1[e] = acc;
                G1d[e] = accd;
            }
            __syncthreads();
            for (int e = n2_lo * q + threadIdx.x; e < n2_hi * q; e += blockDim.x) {
                int n2 = e / q, n1 = e % q;
                double p = 0, d1 = 0, d2 = 0;
                for (int a = 0; a < kd; ++a) {
                    double b1 = T0[lay.B() + n1 * kd + a];
                    p += b1 * G1[a * nw + (n2 - n2_lo)];
                    d1 += T0[lay.D() + n1 * kd + a] * G1[a * nw + (n2 - n2_lo)];
                    d2 += b1 * G1d[a * nw + (n2 - n2_lo)];
                }
                double x1 = T0[lay.x() + n1], x2 = T1[lay.x() + n2];
                double r = x1 - x2;
                double V = T0[lay.v1() + n1] + T1[lay.v1() + n2] + in.ee_coef / sqrt(r * r + in.eta_ee * in.eta_ee);
                double wc = T0[lay.w() + n1] * T1[lay.w() + n2] * T0[lay.chi() + n1] * T1[lay.chi() + n2];
                num += wc * (in.kappa * (d1 * d1 + d2 * d2) + V * p * p);
                den += wc * p * p;
                dip += wc * (x1 + x2) * p * p;
                if (psi_out) psi_out[(psi_off[sid] + e) * nch + ch] = p;
            }
        }
        __syncthreads();
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    dip = block_sum(dip, red);
    if (threadIdx.x == 0) {
        const long long o = 3LL * ((long long)sid * ENERGY_BLOCKS + blk);
        part[o] = num;
        part[o + 1] = den;
        part[o + 2] = dip;
    }
}

__global__ void k_energy_reduce(SwrDeviceView v, const double* part, double* energy, double* norm2, double* dipole) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_inst) return;
    const InstDev& in = v.inst[i];
    double num = 0, den = 0, dip = 0;
    for (int j = 0; j < in.n_sub; ++j)
        for (int b = 0; b < ENERGY_BLOCKS; ++b) {
            const long long o = 3LL * ((long long)(in.sub_base + j) * ENERGY_BLOCKS + b);
            num += part[o];
            den += part[o + 1];
            dip += part[o + 2];
        }
    energy[i] = num / den;
    norm2[i] = den;
    dipole[i] = dip / den;
}

// Antisymmetric states (Appendix A): the lower subdomain (i1 > i2) of each
// mirror pair is not solved; its iterates of the window are the mirror images
// of the upper one's, y_sigma(i)^n = -swap(y_i^n) for n = 0..window (swap:
// coefficient (a, b) -> (b, a); both planes of complex iterates), filled
// before the traces, the exchange and the energies read them.
__global__ void k_anti_fill(SwrDeviceView v, const int* win) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    if (!in.anti || s.N != 2) return;
    const int loc = sid - in.sub_base, i1 = loc % in.L, i2 = loc / in.L;
    if (i1 <= i2) return;
    const SubDev& ms = v.sub[in.sub_base + i2 + in.L * i1];
    const int K = s.K, kd = s.kd, nch = in.mode == SWR_MODE_TDSE ? 2 : 1;
    const long long total = (long long)(win[s.inst] + 1) * nch * K;
    double* h = v.arena + s.hist;
    const double* hm = v.arena + ms.hist;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / K;  // (step, plane)
        const int c = (int)(e - row * K);
        h[e] = -hm[row * K + c / kd + kd * (c % kd)];
    }
}

// ------------------------------------------------------------- host driver

static inline unsigned div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Kernel launches per swr_step besides the window (reset, window, line traces,
// gather, residual, residual reduce, energy, energy reduce; two more with
// CVTOT in every iteration, one more with antisymmetric instances: the mirror
// fill).
extern const int kStepLaunches = 8;

cudaError_t launch_post(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const int* d_win_prev,
                        const double* d_snorm, int cap, int parity, int first_iter, double* d_res_part,
                        int res_blocks, double* d_res, int max_cap_hint, int lt_kmax, int lt_kdmax, int lt_qmax,
                        bool any_anti, double* d_cv_part, double* d_cvtot, bool with_cvtot) {
    int nb = 64;
    if (any_anti) k_anti_fill<<<dim3(nb, v.n_sub), 256, 0, st>>>(v, d_win);
    {
        const size_t base = ((size_t)lt_kmax + (size_t)lt_kdmax + 32 * (size_t)lt_kdmax) * sizeof(float2);
        const size_t tab = 2 * (size_t)lt_qmax * lt_kdmax * sizeof(float2);
        const int staged = base + tab <= 96 * 1024;
        const size_t sm = base + (staged ? tab : 0);
        if (sm > 48 * 1024) cudaFuncSetAttribute(k_line_traces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_line_traces, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        k_line_traces<<<dim3(nb, v.n_sub), 256, sm, st>>>(v, d_win, cap, lt_kmax, lt_kdmax, lt_qmax, staged);
    }
    {
        const int gsz = 4 * lt_qmax;  // interface nodes of a subdomain: at most 4 edges of q
        const size_t gbytes = 2 * (size_t)gsz * sizeof(float2);
        const size_t tab = 2 * (size_t)lt_qmax * lt_kdmax * sizeof(float2);
        const int staged = tab <= 96 * 1024;
        const size_t sm = gbytes + (staged ? tab : 0);
        if (sm > 48 * 1024) cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_gather, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        k_gather<<<dim3(nb, v.n_sub), 256, sm, st>>>(v, d_win, d_snorm, cap, parity, staged, gsz);
    }
    k_residual<<<dim3(res_blocks, v.n_sub), 256, 0, st>>>(v, d_win, d_win_prev, parity, first_iter, d_res_part);
    k_residual_reduce<<<v.n_inst, 256, 0, st>>>(v, d_res_part, res_blocks, d_res);
    if (with_cvtot) {
        k_cvtot<<<dim3(CV_BLOCKS, v.n_inst), 256, 0, st>>>(v, d_win, d_snorm, cap, d_cv_part);
        k_cvtot_reduce<<<div_up(v.n_inst, 128), 128, 0, st>>>(v.n_inst, d_cv_part, CV_BLOCKS, d_cvtot);
    }
    return cudaGetLastError();
}

// CVTOT of the last iteration on request (its line traces, windows and
// normalisations are still in place until the next swr_step).
cudaError_t launch_cvtot(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const double* d_snorm, int cap,
                         double* d_cv_part, double* d_cvtot) {
    k_cvtot<<<dim3(CV_BLOCKS, v.n_inst), 256, 0, st>>>(v, d_win, d_snorm, cap, d_cv_part);
    k_cvtot_reduce<<<div_up(v.n_inst, 128), 128, 0, st>>>(v.n_inst, d_cv_part, CV_BLOCKS, d_cvtot);
    return cudaGetLastError();
}

// Partials of the CVTOT reduction per instance (doubles).
size_t cvtot_part_doubles(int n_inst) { return (size_t)n_inst * CV_BLOCKS; }

// Residual of one iteration into caller-chosen scratch (partials) and output.
cudaError_t launch_residual(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const int* d_win_prev,
                            int parity, int first_iter, double* d_part, int res_blocks, double* d_res) {
    k_residual<<<dim3(res_blocks, v.n_sub), 256, 0, st>>>(v, d_win, d_win_prev, parity, first_iter, d_part);
    k_residual_reduce<<<v.n_inst, 256, 0, st>>>(v, d_part, res_blocks, d_res);
    return cudaGetLastError();
}

// Dynamic shared memory of k_energy for one subdomain: the scaled iterate (K)
// and, with two electrons, the two half-contracted node tables (2 K_d q).
size_t energy_smem(const SubDev& s) {
    return ((size_t)s.K + (s.N == 2 ? 2 * (size_t)s.kd * s.q : 0)) * sizeof(double);
}

cudaError_t launch_energy(const SwrDeviceView& v, cudaStream_t st, const int* d_win, const double* d_snorm,
                          int cap, double* d_part, double* d_energy, double* d_norm2, double* d_dipole,
                          double* psi_out, const long long* psi_off, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_energy<<<dim3(ENERGY_BLOCKS, v.n_sub), 256, smem, st>>>(v, d_win, d_snorm, cap, d_part, psi_out, psi_off);
    k_energy_reduce<<<div_up(v.n_inst, 128), 128, 0, st>>>(v, d_part, d_energy, d_norm2, d_dipole);
    return cudaGetLastError();
}

}  // namespace swr
