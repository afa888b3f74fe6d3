// swr_lsd.cu -- local orbitals (LOs) and local Slater determinants (LSDs).
//
// The paper's second basis family (Sec. 3.2 "Local orbital construction",
// Eq. BARPOT, Eq. LSD; Appendix A "Discrete local Hamiltonian construction
// with local Slater's determinants"; Sec. 7 Test 1 and its Table 1):
//
//   1. in every 1-D subdomain D_i the one-electron eigenproblem
//        1/2 int a phi' psi' + int (V_en + V_b) phi psi = lambda int phi psi,
//      V_b = V_inf s(|x - x_ci| - x_b), a = 1 - s, s the C^2 step rising over
//      [x_b - eps_b/2, x_b + eps_b/2], in a Gaussian basis of kd functions:
//      quadrature of the overlap and Hamiltonian matrices, Cholesky of the
//      overlap, parallel cyclic Jacobi of L^-1 H L^-T in shared memory, back
//      substitution, the M lowest orbitals, each with the sign that makes
//      int phi(x) exp(0.37 (x - x_ci)) dx positive (one CTA per subdomain);
//   2. every orbital at the nodes of one composite Gauss-Legendre rule over
//      the line, and the one-electron integrals between all orbitals:
//      <phi_a, phi_b>, 1/2 <phi_a', phi_b'> + <phi_a|V_en|phi_b>, <phi_a|x|phi_b>
//      (Appendix A's I and J);
//   3. the pair densities w phi_a phi_c of orbitals whose supports
//      [x_ci - x_b - m, x_ci + x_b + m] meet (m past the Gaussian tails; the
//      same or neighbouring subdomains for x_b near |D_i| / 2), T = P W with the soft-Coulomb
//      kernel W(x, s), so that the two-electron integral (ac|bd) of
//      Appendix A is the dot product of T_ac and P_bd;
//   4. per 2-D subdomain Omega_{i,j} (x1 in D_i, x2 in D_j) the K
//      determinants of lowest lambda_l^i + lambda_p^j (l < p when i = j; sums
//      within 1e-9 relative are ties broken by (l, p)), their Gram matrix
//      <a,c><b,d> - <a,d><b,c>, the matrix of H0 = h(1) + h(2) + W(x1 - x2):
//      h_ac S_bd + S_ac h_bd - h_ad S_bc - S_ad h_bc + (ac|bd) - (ad|bc), and
//      their Gram against the determinants of Omega_{i+1,j} (Table 1's w).
//
// Nuclear and electron-electron interactions are soft-Coulomb (the 1-D
// mollified Coulomb of Eq. GEPS diverges).  All arithmetic is FP64; every
// reduction has a fixed order.  The host only lays out the quadrature panels
// and the index tables.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "swr_internal.cuh"

namespace swr {

#define LSD_KD_MAX 64
#define LSD_Q_MAX 16
#define LSD_TIE 1e-9

struct LsdDev {
    double a, H, eps, xb, eps_b, v_inf, delta, eta_en, eta_ee, ee_coef, harmonic;
    double xn[3], zn[3];
    int L, M, K, kd, q, n_nuc, ng, n_pairs;
};

__device__ inline double lsd_centre(const LsdDev& d, int i) { return d.a + (i + 0.5) * d.H; }

// C^2 step: 0 for u <= 0, 1 for u >= 1, 6u^5 - 15u^4 + 10u^3 between.
__device__ inline double lsd_step(double u) {
    u = fmin(fmax(u, 0.0), 1.0);
    return u * u * u * (u * (6.0 * u - 15.0) + 10.0);
}
__device__ inline double lsd_switch(const LsdDev& d, double x, double xc) {
    const double t = fabs(x - xc) - d.xb;
    return lsd_step((t + 0.5 * d.eps_b) / d.eps_b);
}
__device__ inline double lsd_ven(const LsdDev& d, double x) {
    double v = 0.5 * d.harmonic * x * x;
    for (int A = 0; A < d.n_nuc; ++A) v -= d.zn[A] / sqrt((x - d.xn[A]) * (x - d.xn[A]) + d.eta_en * d.eta_en);
    return v;
}

// Gauss-Legendre nodes and weights of order q on [-1, 1]: Newton's method on
// the three-term recurrence of P_q, from the Chebyshev-like initial guess.
__global__ void k_lsd_gl(int q, double* t, double* w) {
    const int k = threadIdx.x;
    if (k >= q) return;
    double x = cos(3.14159265358979323846 * (k + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int j = 2; j <= q; ++j) {
            const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
    }
    t[q - 1 - k] = x;  // ascending
    w[q - 1 - k] = 2.0 / ((1.0 - x * x) * dp * dp);
}

// Nodes of composite rules: panel p of [edges[p], edges[p+1]] gives nodes
// p q .. p q + q - 1 (panels of all rules concatenated, edge index base[p]).
__global__ void k_lsd_nodes(const double* edges, const int* ebase, int n_panels, const double* t, const double* w, int q,
                            double* x, double* wx) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_panels * q) return;
    const int p = n / q, k = n - p * q;
    const double e0 = edges[ebase[p]], e1 = edges[ebase[p] + 1];
    x[n] = 0.5 * (e1 - e0) * t[k] + 0.5 * (e1 + e0);
    wx[n] = 0.5 * (e1 - e0) * w[k];
}

// ------------------------------------------------------ 1. local orbitals
//
// One CTA per subdomain.  Shared memory: A (overlap, then its Cholesky factor
// in the lower triangle) | B (Hamiltonian, then L^-1 H L^-T, then its
// eigenvalues on the diagonal) | V (eigenvectors) | scratch, each n x n with
// n = kd rounded up to even (a padded row is decoupled with a large diagonal).
__device__ void lsd_jacobi(double* B, double* V, int n, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x, half = n / 2;
    __shared__ int s_pair[LSD_KD_MAX][2];
    __shared__ double s_cs[LSD_KD_MAX / 2][2];
    __shared__ int s_go;
    for (int sweep = 0; sweep < 60; ++sweep) {
        for (int r = 0; r < n - 1; ++r) {
            if (tid < half) {
                // circle method: player 0 against 1 + r mod (n-1), then symmetric pairs
                int p, qq;
                if (tid == 0) {
                    p = 0;
                    qq = 1 + (r % (n - 1));
                } else {
                    p = 1 + ((r + tid) % (n - 1));
                    qq = 1 + ((r + n - 1 - tid) % (n - 1));
                }
                if (p > qq) {
                    const int tmp = p;
                    p = qq;
                    qq = tmp;
                }
                s_pair[tid][0] = p;
                s_pair[tid][1] = qq;
                const double app = B[p * n + p], aqq = B[qq * n + qq], apq = B[p * n + qq];
                double c = 1.0, s = 0.0;
                if (fabs(apq) > 1e-300) {
                    const double th = (aqq - app) / (2.0 * apq);
                    const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    c = 1.0 / sqrt(tt * tt + 1.0);
                    s = tt * c;
                }
                s_cs[tid][0] = c;
                s_cs[tid][1] = s;
            }
            __syncthreads();
            // rows p, q of B <- J^T B
            for (int e = tid; e < half * n; e += nt) {
                const int k = e / n, col = e - k * n;
                const int p = s_pair[k][0], qq = s_pair[k][1];
                const double c = s_cs[k][0], s = s_cs[k][1];
                const double bp = B[p * n + col], bq = B[qq * n + col];
                B[p * n + col] = c * bp - s * bq;
                B[qq * n + col] = s * bp + c * bq;
            }
            __syncthreads();
            // columns p, q of B <- B J, and of V
            for (int e = tid; e < half * n; e += nt) {
                const int k = e / n, row = e - k * n;
                const int p = s_pair[k][0], qq = s_pair[k][1];
                const double c = s_cs[k][0], s = s_cs[k][1];
                const double bp = B[row * n + p], bq = B[row * n + qq];
                B[row * n + p] = c * bp - s * bq;
                B[row * n + qq] = s * bp + c * bq;
                const double vp = V[row * n + p], vq = V[row * n + qq];
                V[row * n + p] = c * vp - s * vq;
                V[row * n + qq] = s * vp + c * vq;
            }
            __syncthreads();
        }
        // off-diagonal mass against the diagonal (fixed-order reduction)
        double off = 0.0, dia = 0.0;
        for (int e = tid; e < n * n; e += nt) {
            const int rr = e / n, cc = e - rr * n;
            if (rr == cc) dia += B[e] * B[e];
            else off += B[e] * B[e];
        }
        red[tid] = off;
        red[nt + tid] = dia;
        __syncthreads();
        if (tid == 0) {
            double o = 0.0, d = 0.0;
            for (int k = 0; k < nt; ++k) {
                o += red[k];
                d += red[nt + k];
            }
            s_go = o > 1e-32 * d;
        }
        __syncthreads();
        if (!s_go) break;
    }
}

__global__ void k_lsd_local(LsdDev d, const double* xl, const double* wl, const int* nbase, double* gtab, double* lam_out,
                            double* coef_out, int* err) {
    extern __shared__ double lsm[];
    const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int kd = d.kd, n = (kd + 1) & ~1;
    double* A = lsm;
    double* B = A + n * n;
    double* V = B + n * n;
    double* W = V + n * n;  // scratch n x n
    double* red = W + n * n;  // 2 nt
    __shared__ int s_ord[LSD_KD_MAX];
    __shared__ double s_sign[LSD_KD_MAX];
    const int n0 = nbase[i], nn = nbase[i + 1] - n0;
    const double* x = xl + n0;
    const double* w = wl + n0;
    const double xc = lsd_centre(d, i);
    const double h = 2.0 * d.xb / (kd - 1);
    double* g = gtab + (size_t)n0 * 2 * LSD_KD_MAX;  // [nn][kd] values then [nn][kd] derivatives
    double* dg = g + (size_t)nn * LSD_KD_MAX;
    for (int e = tid; e < nn * kd; e += nt) {
        const int m = e / kd, k = e - m * kd;
        const double al = (k == kd - 1) ? xc + d.xb : (double)k * h + (xc - d.xb);
        const double u = x[m] - al, gv = exp(-d.delta * u * u);
        g[(size_t)m * LSD_KD_MAX + k] = gv;
        dg[(size_t)m * LSD_KD_MAX + k] = -2.0 * d.delta * u * gv;
    }
    __syncthreads();
    // overlap and Hamiltonian (upper triangle computed, both filled)
    for (int e = tid; e < n * n; e += nt) {
        const int r = e / n, c = e - r * n;
        if (r >= kd || c >= kd) {
            A[e] = (r == c) ? 1.0 : 0.0;
            B[e] = (r == c) ? 1e30 : 0.0;
            continue;
        }
        if (c < r) continue;
        double s = 0.0, hh = 0.0;
        for (int m = 0; m < nn; ++m) {
            const double sw = lsd_switch(d, x[m], xc);
            const double gr = g[(size_t)m * LSD_KD_MAX + r], gc = g[(size_t)m * LSD_KD_MAX + c];
            const double dr = dg[(size_t)m * LSD_KD_MAX + r], dc = dg[(size_t)m * LSD_KD_MAX + c];
            s += w[m] * gr * gc;
            hh += w[m] * (0.5 * (1.0 - sw) * dr * dc + (lsd_ven(d, x[m]) + d.v_inf * sw) * gr * gc);
        }
        A[r * n + c] = A[c * n + r] = s;
        B[r * n + c] = B[c * n + r] = hh;
    }
    __syncthreads();
    // Cholesky A = L L^T (lower triangle of A)
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            double s = A[j * n + j];
            for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
            if (!(s > 0.0)) {
                atomicOr(err, 1);
                s = 1e-300;
            }
            A[j * n + j] = sqrt(s);
        }
        __syncthreads();
        for (int r = j + 1 + tid; r < n; r += nt) {
            double s = A[r * n + j];
            for (int k = 0; k < j; ++k) s -= A[r * n + k] * A[j * n + k];
            A[r * n + j] = s / A[j * n + j];
        }
        __syncthreads();
    }
    // W = L^-1 B (forward substitution per column), then B = L^-1 W^T
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = tid; c < n; c += nt) {
            for (int r = 0; r < n; ++r) {
                double s = pass == 0 ? B[r * n + c] : W[c * n + r];
                for (int k = 0; k < r; ++k) s -= A[r * n + k] * (pass == 0 ? W[k * n + c] : V[k * n + c]);
                if (pass == 0) W[r * n + c] = s / A[r * n + r];
                else V[r * n + c] = s / A[r * n + r];
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) {
        const int r = e / n, c = e - r * n;
        B[e] = 0.5 * (V[r * n + c] + V[c * n + r]);
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) V[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    lsd_jacobi(B, V, n, red);
    // ascending order of the eigenvalues (ties by index)
    if (tid < n) {
        const double lv = B[tid * n + tid];
        int rank = 0;
        for (int k = 0; k < n; ++k) {
            const double lk = B[k * n + k];
            rank += (lk < lv || (lk == lv && k < tid)) ? 1 : 0;
        }
        s_ord[rank] = tid;
    }
    __syncthreads();
    // X = L^-T V[:, ord] for the M lowest (back substitution), into W's columns
    for (int l = tid; l < d.M; l += nt) {
        const int col = s_ord[l];
        for (int r = n - 1; r >= 0; --r) {
            double s = V[r * n + col];
            for (int k = r + 1; k < n; ++k) s -= A[k * n + r] * W[k * n + l];
            W[r * n + l] = s / A[r * n + r];
        }
    }
    __syncthreads();
    // sign: int phi exp(0.37 (x - xc)) dx > 0
    for (int l = tid; l < d.M; l += nt) {
        double pr = 0.0;
        for (int m = 0; m < nn; ++m) {
            double v = 0.0;
            for (int k = 0; k < kd; ++k) v += W[k * n + l] * g[(size_t)m * LSD_KD_MAX + k];
            pr += w[m] * exp(0.37 * (x[m] - xc)) * v;
        }
        s_sign[l] = pr < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (int e = tid; e < kd * d.M; e += nt) {
        const int k = e / d.M, l = e - k * d.M;
        coef_out[((size_t)i * kd + k) * d.M + l] = s_sign[l] * W[k * n + l];
    }
    for (int l = tid; l < d.M; l += nt) lam_out[i * d.M + l] = B[s_ord[l] * n + s_ord[l]];
}

// ------------------------------------------- 2. orbitals on the global rule
__global__ void k_lsd_table(LsdDev d, const double* xg, const double* coef, double* F, double* dF) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x, o = blockIdx.y;
    if (m >= d.ng) return;
    const int i = o / d.M, l = o - i * d.M, kd = d.kd;
    const double xc = lsd_centre(d, i), h = 2.0 * d.xb / (kd - 1), x = xg[m];
    double v = 0.0, dv = 0.0;
    for (int k = 0; k < kd; ++k) {
        const double al = (k == kd - 1) ? xc + d.xb : (double)k * h + (xc - d.xb);
        const double u = x - al, gv = exp(-d.delta * u * u), c = coef[((size_t)i * kd + k) * d.M + l];
        v += c * gv;
        dv += c * (-2.0 * d.delta * u * gv);
    }
    F[(size_t)o * d.ng + m] = v;
    dF[(size_t)o * d.ng + m] = dv;
}

// One warp per orbital pair (a, b): overlap, one-electron Hamiltonian, position.
__global__ void k_lsd_one(LsdDev d, const double* xg, const double* wg, const double* F, const double* dF, double* S1,
                          double* h1, double* J1) {
    const int LM = d.L * d.M;
    const int pr = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (pr >= LM * LM) return;
    const int a = pr / LM, b = pr - a * LM;
    const double* fa = F + (size_t)a * d.ng;
    const double* fb = F + (size_t)b * d.ng;
    const double* da = dF + (size_t)a * d.ng;
    const double* db = dF + (size_t)b * d.ng;
    double s = 0.0, hh = 0.0, jj = 0.0;
    for (int m = lane; m < d.ng; m += 32) {
        const double ff = wg[m] * fa[m] * fb[m];
        s += ff;
        hh += 0.5 * wg[m] * da[m] * db[m] + lsd_ven(d, xg[m]) * ff;
        jj += xg[m] * ff;
    }
    s = warp_sum(s);
    hh = warp_sum(hh);
    jj = warp_sum(jj);
    if (lane == 0) {
        S1[pr] = s;
        h1[pr] = hh;
        J1[pr] = jj;
    }
}

// ------------------------------------------------- 3. two-electron integrals
// Pair densities P[k][m] = w_m phi_a(x_m) phi_c(x_m) of the listed pairs.
__global__ void k_lsd_pairs(LsdDev d, const double* wg, const double* F, const int* pa, const int* pc, double* P) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (m >= d.ng) return;
    P[(size_t)k * d.ng + m] = wg[m] * F[(size_t)pa[k] * d.ng + m] * F[(size_t)pc[k] * d.ng + m];
}

// The soft-Coulomb kernel on the global nodes, W[m][s] = c / sqrt((x_m - x_s)^2 + eta^2).
__global__ void k_lsd_w(LsdDev d, const double* xg, double* Wm) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
    if (s >= d.ng) return;
    const double u = xg[m] - xg[s];
    Wm[(size_t)m * d.ng + s] = d.ee_coef / sqrt(u * u + d.eta_ee * d.eta_ee);
}

// T[k][s] = sum_m P[k][m] W[m][s] over the pair's support nodes [lo, hi)
// (rows of W read along s: coalesced; P staged in shared memory).
__global__ void k_lsd_pw(LsdDev d, const double* Wm, const double* P, const int* lo, const int* hi, double* T) {
    __shared__ double sp[256];
    const int k = blockIdx.y, s = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int m0 = lo[k]; m0 < hi[k]; m0 += 256) {
        const int m = m0 + threadIdx.x;
        sp[threadIdx.x] = m < hi[k] ? P[(size_t)k * d.ng + m] : 0.0;
        __syncthreads();
        const int cnt = min(256, hi[k] - m0);
        if (s < d.ng)
            for (int j = 0; j < cnt; ++j) acc += sp[j] * Wm[(size_t)(m0 + j) * d.ng + s];
        __syncthreads();
    }
    if (s < d.ng) T[(size_t)k * d.ng + s] = acc;
}

// ----------------------------------------------- 4. determinants per Omega
// Rank of every candidate (l, p) of Omega_{i,j} (i = om mod L, j = om / L) by
// lambda_l^i + lambda_p^j with the tie rule; the first K kept.
__global__ void k_lsd_select(LsdDev d, const double* lam, int* pairs, int* err) {
    const int om = blockIdx.x, i = om % d.L, j = om / d.L, M = d.M;
    const int nc = (i == j) ? M * (M - 1) / 2 : M * M;
    for (int u = threadIdx.x; u < nc; u += blockDim.x) {
        // candidate u: (l, p) in lexicographic order among the allowed pairs
        auto cand = [&](int v, int& l, int& p) {
            if (i != j) {
                l = v / M;
                p = v - l * M;
            } else {
                l = 0;
                int rem = v;
                while (rem >= M - 1 - l) {
                    rem -= M - 1 - l;
                    ++l;
                }
                p = l + 1 + rem;
            }
        };
        int lu, pu;
        cand(u, lu, pu);
        const double eu = lam[i * M + lu] + lam[j * M + pu];
        int rank = 0;
        for (int v = 0; v < nc; ++v) {
            if (v == u) continue;
            int lv, pv;
            cand(v, lv, pv);
            const double ev = lam[i * M + lv] + lam[j * M + pv], df = ev - eu;
            bool before;
            if (fabs(df) <= LSD_TIE * (1.0 + fabs(eu) + fabs(ev))) before = (lv < lu) || (lv == lu && pv < pu);
            else before = df < 0.0;
            rank += before ? 1 : 0;
        }
        if (rank < d.K) {
            int* q = pairs + ((size_t)om * d.K + rank) * 2;
            if (atomicCAS(q, -1, lu) != -1) atomicOr(err, 2);  // two candidates on one rank
            q[1] = pu;
        }
    }
}

// Gram, H0 and the Gram against Omega_{i+1,j}: one warp per entry (r, c).
__global__ void k_lsd_blocks(LsdDev d, const int* pairs, const double* S1, const double* h1, const double* T,
                             const double* P, const int* pid, const int* lo, const int* hi, double* S_lsd,
                             double* H_lsd, double* G_next) {
    const int om = blockIdx.y, i = om % d.L, j = om / d.L, M = d.M, K = d.K, LM = d.L * d.M;
    const int e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= K * K) return;
    const int r = e / K, c = e - r * K;
    const int* pr = pairs + ((size_t)om * K + r) * 2;
    const int* pc = pairs + ((size_t)om * K + c) * 2;
    // a rank left empty by the selection (reported there): no index to read
    if (pr[0] < 0 || pr[1] < 0 || pc[0] < 0 || pc[1] < 0 ||
        (i + 1 < d.L && (pairs[((size_t)(om + 1) * K + c) * 2] < 0 || pairs[((size_t)(om + 1) * K + c) * 2 + 1] < 0))) {
        if (lane == 0) {
            const size_t o = (size_t)om * K * K + e;
            S_lsd[o] = H_lsd[o] = G_next[o] = nan("");
        }
        return;
    }
    const int a = i * M + pr[0], b = j * M + pr[1], cc = i * M + pc[0], dd = j * M + pc[1];
    const double sac = S1[a * LM + cc], sbd = S1[b * LM + dd], sad = S1[a * LM + dd], sbc = S1[b * LM + cc];
    // (xy|zw) = T_{xy} . P_{zw} over the support of the pair zw; 0 when a pair's
    // supports are disjoint (no pair density listed)
    auto eri = [&](int x, int y, int z, int w) -> double {
        const int k1 = pid[x * LM + y], k2 = pid[z * LM + w];
        double s = 0.0;
        if (k1 >= 0 && k2 >= 0)
            for (int m = lo[k2] + lane; m < hi[k2]; m += 32) s += T[(size_t)k1 * d.ng + m] * P[(size_t)k2 * d.ng + m];
        return warp_sum(s);
    };
    const double one = h1[a * LM + cc] * sbd + sac * h1[b * LM + dd] - h1[a * LM + dd] * sbc - sad * h1[b * LM + cc];
    const double two = eri(a, cc, b, dd) - eri(a, dd, b, cc);
    double gn = 0.0;
    if (i + 1 < d.L) {
        const int* pn = pairs + ((size_t)(om + 1) * K + c) * 2;  // Omega_{i+1,j}
        const int c2 = (i + 1) * M + pn[0], d2 = j * M + pn[1];
        gn = S1[a * LM + c2] * S1[b * LM + d2] - S1[a * LM + d2] * S1[b * LM + c2];
    }
    if (lane == 0) {
        const size_t o = (size_t)om * K * K + e;
        S_lsd[o] = sac * sbd - sad * sbc;
        H_lsd[o] = one + two;
        G_next[o] = gn;
    }
}

}  // namespace swr

// ------------------------------------------------------------- host side
using namespace swr;

namespace {
std::string g_lsd_err;

swr_status lsd_fail(swr_status s, const char* msg) {
    g_lsd_err = msg;
    set_setup_error(msg);
    return s;
}

// Composite rule panels on [lo, hi] with edges at the breakpoints inside and
// panels of width <= panel between them (k step + s0, the last edge exact).
void lsd_panels(double lo, double hi, double panel, const std::vector<double>& brk, std::vector<double>& edges,
                std::vector<int>& ebase) {
    std::vector<double> pts = {lo, hi};
    for (double b : brk)
        if (b > lo && b < hi) pts.push_back(b);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    for (size_t s = 0; s + 1 < pts.size(); ++s) {
        const double s0 = pts[s], s1 = pts[s + 1];
        int n = (int)ceil((s1 - s0) / panel - 1e-12);
        if (n < 1) n = 1;
        const double step = (s1 - s0) / n;
        const size_t first = edges.size();
        for (int k = 0; k < n; ++k) edges.push_back(k == 0 ? s0 : (double)k * step + s0);
        edges.push_back(s1);
        for (int k = 0; k < n; ++k) ebase.push_back((int)(first + k));
    }
}

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    T* get(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, (n ? n : 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
};
}  // namespace

extern "C" swr_status swr_lsd_build(const swr_lsd_problem* p, swr_lsd_result* out) {
    if (!p || !out) return lsd_fail(SWR_EINVAL, "swr_lsd_build: problem or result is NULL");
    if (!out->lam || !out->coef || !out->S1 || !out->h1 || !out->J1 || !out->pairs || !out->S_lsd || !out->H_lsd ||
        !out->G_next)
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: every result buffer must be given");
    if (!(p->box_hi > p->box_lo) || p->L < 1 || p->L > 16 || !(p->overlap >= 0.0))
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: need box_lo < box_hi, 1 <= L <= 16, overlap >= 0");
    if (p->kd < 2 || p->kd > LSD_KD_MAX || p->M < 1 || p->M > p->kd)
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: need 2 <= kd <= 64 and 1 <= M <= kd");
    if (p->K < 1 || p->K > p->M * (p->M - 1) / 2)
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: need 1 <= K <= M (M - 1) / 2 (determinants of a diagonal subdomain)");
    if (p->q_p < 2 || p->q_p > LSD_Q_MAX || !(p->panel > 0.0))
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: need 2 <= q_p <= 16 and panel > 0");
    if (p->n_nuclei < 0 || p->n_nuclei > 3 || (p->n_nuclei > 0 && !(p->eta_en > 0.0)) || !(p->eta_ee > 0.0))
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: at most 3 nuclei; eta_en > 0 with nuclei; eta_ee > 0");
    if (!(p->xb_factor > 0.0) || !(p->eps_b > 0.0) || !(p->v_inf >= 0.0) || !(p->delta >= 0.0))
        return lsd_fail(SWR_EINVAL, "swr_lsd_build: need xb_factor > 0, eps_b > 0, v_inf >= 0, delta >= 0");
    LsdDev d;
    memset(&d, 0, sizeof(d));
    d.L = p->L;
    d.M = p->M;
    d.K = p->K;
    d.kd = p->kd;
    d.q = p->q_p;
    d.a = p->box_lo;
    d.H = (p->box_hi - p->box_lo) / p->L;
    d.eps = p->overlap;
    const double width = d.H + d.eps;  // |D_i|
    d.xb = p->xb_factor * width;
    d.eps_b = p->eps_b;
    d.v_inf = p->v_inf;
    const double hc = 2.0 * d.xb / (p->kd - 1);
    d.delta = p->delta > 0.0 ? p->delta : 0.5 / (hc * hc);
    d.eta_en = p->eta_en;
    d.eta_ee = p->eta_ee;
    d.ee_coef = p->ee_coef;
    d.harmonic = p->harmonic;
    d.n_nuc = p->n_nuclei;
    for (int A = 0; A < p->n_nuclei; ++A) {
        d.xn[A] = p->x_nuc[A];
        d.zn[A] = p->Z_nuc[A];
    }
    const double margin = std::max(p->eps_b, 8.0 / sqrt(2.0 * d.delta));
    // local rules (breakpoints where the barrier's step starts and ends) and the global rule
    std::vector<double> edges;
    std::vector<int> ebase, nbase = {0};
    for (int i = 0; i < p->L; ++i) {
        const double xc = d.a + (i + 0.5) * d.H, e = 0.5 * p->eps_b;
        const size_t before = ebase.size();
        lsd_panels(xc - d.xb - margin, xc + d.xb + margin, p->panel,
                   {xc - d.xb - e, xc - d.xb + e, xc + d.xb - e, xc + d.xb + e}, edges, ebase);
        nbase.push_back(nbase.back() + (int)(ebase.size() - before) * p->q_p);
    }
    const int n_local_panels = (int)ebase.size();
    const double gm = d.xb - 0.5 * width + margin;
    const double glo = p->box_lo - 0.5 * p->overlap - gm, ghi = p->box_hi + 0.5 * p->overlap + gm;
    lsd_panels(glo, ghi, p->panel, {}, edges, ebase);
    const int n_global_panels = (int)ebase.size() - n_local_panels;
    d.ng = n_global_panels * p->q_p;
    const int LM = p->L * p->M, nloc = nbase.back();
    // pair densities of orbitals in the same or neighbouring subdomains, with the
    // node range where both are above the Gaussian tails
    std::vector<int> pa, pc, plo, phi, pid(LM * LM, -1);
    auto node_of = [&](double x) {  // first global node at or after x
        const double pw = (ghi - glo) / n_global_panels;
        int pnl = (int)floor((x - glo) / pw);
        pnl = std::min(std::max(pnl, 0), n_global_panels);
        return pnl * p->q_p;
    };
    for (int a = 0; a < LM; ++a)
        for (int c = a; c < LM; ++c) {
            const int ia = a / p->M, ic = c / p->M;
            const double xa = d.a + (ia + 0.5) * d.H, xc2 = d.a + (ic + 0.5) * d.H;
            const double lo = std::max(xa, xc2) - d.xb - margin, hi = std::min(xa, xc2) + d.xb + margin;
            if (!(hi > lo)) continue;  // supports (x_ci -+ (x_b + margin)) apart
            pid[a * LM + c] = pid[c * LM + a] = (int)pa.size();
            pa.push_back(a);
            pc.push_back(c);
            plo.push_back(node_of(lo));
            phi.push_back(std::min(d.ng, node_of(hi) + p->q_p));
        }
    d.n_pairs = (int)pa.size();
    if (d.n_pairs > 65535) return lsd_fail(SWR_EINVAL, "swr_lsd_build: more than 65535 orbital pairs (L M too large)");
    // device work
    DevBuf db;
    double* dt = db.get<double>(LSD_Q_MAX);
    double* dw = db.get<double>(LSD_Q_MAX);
    double* dedges = db.get<double>(edges.size());
    int* debase = db.get<int>(ebase.size());
    double* dx = db.get<double>((size_t)(nloc + d.ng));
    double* dwx = db.get<double>((size_t)(nloc + d.ng));
    int* dnbase = db.get<int>(nbase.size());
    double* dgtab = db.get<double>((size_t)nloc * 2 * LSD_KD_MAX);
    double* dlam = db.get<double>((size_t)LM);
    double* dcoef = db.get<double>((size_t)p->L * p->kd * p->M);
    double* dF = db.get<double>((size_t)LM * d.ng);
    double* ddF = db.get<double>((size_t)LM * d.ng);
    double* dS1 = db.get<double>((size_t)LM * LM);
    double* dh1 = db.get<double>((size_t)LM * LM);
    double* dJ1 = db.get<double>((size_t)LM * LM);
    int* dpa = db.get<int>(pa.size());
    int* dpc = db.get<int>(pc.size());
    int* dplo = db.get<int>(plo.size());
    int* dphi = db.get<int>(phi.size());
    int* dpid = db.get<int>(pid.size());
    double* dP = db.get<double>((size_t)d.n_pairs * d.ng);
    double* dT = db.get<double>((size_t)d.n_pairs * d.ng);
    double* dWm = db.get<double>((size_t)d.ng * d.ng);
    const size_t nblk = (size_t)p->L * p->L * p->K * p->K;
    int* dpairs = db.get<int>((size_t)p->L * p->L * p->K * 2);
    double* dSl = db.get<double>(nblk);
    double* dHl = db.get<double>(nblk);
    double* dGn = db.get<double>(nblk);
    int* derr = db.get<int>(1);
    if (!dt || !dw || !dedges || !debase || !dx || !dwx || !dnbase || !dgtab || !dlam || !dcoef || !dF || !ddF ||
        !dS1 || !dh1 || !dJ1 || !dpa || !dpc || !dplo || !dphi || !dpid || !dP || !dT || !dpairs || !dSl || !dHl ||
        !dGn || !derr || !dWm) {
        cudaGetLastError();
        return lsd_fail(SWR_ENOMEM, "swr_lsd_build: device allocation failed");
    }
    cudaError_t e = cudaSuccess;
#define LSD_CU(call)                                                               \
    do {                                                                           \
        if (e == cudaSuccess) e = (call);                                          \
    } while (0)
    LSD_CU(cudaMemcpy(dedges, edges.data(), edges.size() * sizeof(double), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(debase, ebase.data(), ebase.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dnbase, nbase.data(), nbase.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dpa, pa.data(), pa.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dpc, pc.data(), pc.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dplo, plo.data(), plo.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dphi, phi.data(), phi.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemcpy(dpid, pid.data(), pid.size() * sizeof(int), cudaMemcpyHostToDevice));
    LSD_CU(cudaMemset(dpairs, 0xff, (size_t)p->L * p->L * p->K * 2 * sizeof(int)));
    LSD_CU(cudaMemset(derr, 0, sizeof(int)));
    if (e == cudaSuccess) {
        k_lsd_gl<<<1, LSD_Q_MAX>>>(p->q_p, dt, dw);
        const int nn = (n_local_panels + n_global_panels) * p->q_p;
        k_lsd_nodes<<<(nn + 255) / 256, 256>>>(dedges, debase, n_local_panels + n_global_panels, dt, dw, p->q_p, dx,
                                                dwx);
        const int n = (p->kd + 1) & ~1, nt = 256;
        const size_t smem = (4 * (size_t)n * n + 2 * nt) * sizeof(double);
        LSD_CU(cudaFuncSetAttribute(k_lsd_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lsd_local<<<p->L, nt, smem>>>(d, dx, dwx, dnbase, dgtab, dlam, dcoef, derr);
        const double* xg = dx + nloc;
        const double* wg = dwx + nloc;
        k_lsd_table<<<dim3((d.ng + 127) / 128, LM), 128>>>(d, xg, dcoef, dF, ddF);
        k_lsd_one<<<(LM * LM + 7) / 8, 256>>>(d, xg, wg, dF, ddF, dS1, dh1, dJ1);
        k_lsd_pairs<<<dim3((d.ng + 255) / 256, d.n_pairs), 256>>>(d, wg, dF, dpa, dpc, dP);
        k_lsd_w<<<dim3((d.ng + 255) / 256, d.ng), 256>>>(d, xg, dWm);
        k_lsd_pw<<<dim3((d.ng + 255) / 256, d.n_pairs), 256>>>(d, dWm, dP, dplo, dphi, dT);
        k_lsd_select<<<p->L * p->L, 256>>>(d, dlam, dpairs, derr);
        k_lsd_blocks<<<dim3((p->K * p->K + 7) / 8, p->L * p->L), 256>>>(d, dpairs, dS1, dh1, dT, dP, dpid, dplo, dphi,
                                                                       dSl, dHl, dGn);
        LSD_CU(cudaGetLastError());
        LSD_CU(cudaDeviceSynchronize());
    }
    int herr = 0;
    LSD_CU(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->lam, dlam, (size_t)LM * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->coef, dcoef, (size_t)p->L * p->kd * p->M * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->S1, dS1, (size_t)LM * LM * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->h1, dh1, (size_t)LM * LM * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->J1, dJ1, (size_t)LM * LM * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->pairs, dpairs, (size_t)p->L * p->L * p->K * 2 * sizeof(int), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->S_lsd, dSl, nblk * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->H_lsd, dHl, nblk * sizeof(double), cudaMemcpyDeviceToHost));
    LSD_CU(cudaMemcpy(out->G_next, dGn, nblk * sizeof(double), cudaMemcpyDeviceToHost));
#undef LSD_CU
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "swr_lsd_build: %s", cudaGetErrorString(e));
        return lsd_fail(SWR_ECUDA, msg);
    }
    if (herr & 1) return lsd_fail(SWR_ESINGULAR, "swr_lsd_build: an orbital basis overlap is not positive definite");
    if (herr & 2) return lsd_fail(SWR_ENUMERIC, "swr_lsd_build: the tie rule does not order the determinants");
    return SWR_OK;
}
