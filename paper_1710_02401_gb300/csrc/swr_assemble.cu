// swr_assemble.cu -- Galerkin assembly of the local SWR systems on sm_103a.
//
// Sec. 5.1 of the paper ("Construction of the local approximate solutions")
// defines on each subdomain A_i = <v,v>, H~_i = <v,(H0 + R_i) v>, Q_i = <x v, v>,
// "computed once for all".  Here the local basis is the tensor product of 1-D
// Gaussians (Sec. 2, Eq. gauss1d), so everything except the electron-electron
// term factorises coordinate by coordinate:
//   A = S (x) S,  K = Kf (+) Kf,  V_en = U (+) U,  Q = X (+) X,  R = R1 (+) R2,
// with (+) the Kronecker sum.  The local bases are orthonormalised per
// coordinate by a Cholesky factor of S (X_d = L_d^{-T}, so A' = I), the
// electron-electron block is assembled sum-factorised as two batched DGEMMs
// (q x q by q x kd^2, then kd^2 x q by q x kd^2), and the time-invariant step
// matrices are inverted by blocked Gauss-Jordan elimination.
#include <math.h>
#include <stdio.h>

#include "swr_internal.cuh"

namespace swr {

// ------------------------------------------------------------ Gauss-Legendre

// Nodes/weights of the n-point Gauss-Legendre rule on [-1,1] by Newton
// iteration on the three-term recurrence of P_n (n <= SWR_MAX_QP).
__device__ void gauss_legendre(int n, double* t, double* wt) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // i-th root in decreasing order, initial guess of Tricomi type
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? x : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dp = n * (x * pn - pm) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        // recompute derivative at the converged root
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? x : p1, pm = (n == 1) ? 1.0 : p0;
        dp = n * (x * pn - pm) / (x * x - 1.0);
        int j = n - 1 - i;  // ascending order
        t[j] = x;
        wt[j] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

__device__ inline double panel_break(double lo, double hi, double eps, int n_mid, int p) {
    // breakpoints: lo, lo+eps, middle zone cut in n_mid equal panels, hi-eps, hi
    if (p == 0) return lo;
    if (p == n_mid + 2) return hi;
    if (p == n_mid + 1) return hi - eps;
    if (p == 1) return lo + eps;
    return lo + eps + (hi - lo - 2.0 * eps) * (double)(p - 1) / (double)n_mid;
}

// K1: quadrature nodes, weights, partition-of-unity weights, 1-D potential,
// centres, basis values/derivatives at nodes and at the 4 line positions.
__global__ void k_tabulate(SwrDeviceView v) {
    const int sid = blockIdx.x, d = blockIdx.y;
    const SubDev& s = v.sub[sid];
    if (d >= s.N) return;
    const InstDev& in = v.inst[s.inst];
    __shared__ double t[SWR_MAX_QP], wt[SWR_MAX_QP];
    gauss_legendre(in.q_p, t, wt);
    __syncthreads();
    double* T = v.arena + s.t1[d];
    T1Layout lay(s.q, s.kd);
    const double lo = s.lo[d], hi = s.hi[d], eps = in.eps;
    const int kd = s.kd, q = s.q, idx = s.idx[d];
    for (int n = threadIdx.x; n < q; n += blockDim.x) {
        int p = n / in.q_p, i = n % in.q_p;
        double p0 = panel_break(lo, hi, eps, in.n_mid, p), p1 = panel_break(lo, hi, eps, in.n_mid, p + 1);
        double x = 0.5 * (p1 - p0) * t[i] + 0.5 * (p1 + p0);
        T[lay.x() + n] = x;
        T[lay.w() + n] = 0.5 * (p1 - p0) * wt[i];
        double chi = 1.0;
        if (p == 0 && idx > 0) chi = 0.5;
        if (p == in.n_mid + 1 && idx < in.L - 1) chi = 0.5;
        T[lay.chi() + n] = chi;
        double vx = 0.5 * in.harmonic * x * x;
        for (int A = 0; A < in.n_nuc; ++A) {
            double r = x - in.x_nuc[A];
            vx -= in.Z_nuc[A] / sqrt(r * r + in.eta_en * in.eta_en);
        }
        T[lay.v1() + n] = vx;
    }
    for (int j = threadIdx.x; j < kd; j += blockDim.x)
        T[lay.alpha() + j] = (kd > 1) ? lo + (hi - lo) * (double)j / (double)(kd - 1) : 0.5 * (lo + hi);
    __syncthreads();
    const double dl = s.delta;
    for (int e = threadIdx.x; e < q * kd; e += blockDim.x) {
        int n = e / kd, j = e % kd;
        double r = T[lay.x() + n] - T[lay.alpha() + j];
        double f = exp(-dl * r * r);
        T[lay.B() + e] = f;
        T[lay.D() + e] = -2.0 * dl * r * f;
    }
    for (int e = threadIdx.x; e < 4 * kd; e += blockDim.x) {
        int l = e / kd, j = e % kd;
        double r = line_pos(lo, hi, eps, l) - T[lay.alpha() + j];
        double f = exp(-dl * r * r);
        T[lay.Lv() + e] = f;
        T[lay.Ld() + e] = -2.0 * dl * r * f;
    }
}

// K3a: 1-D Galerkin matrices of one coordinate by quadrature:
// S = <phi,phi>, Kf = <phi',phi'>, Xpos = <x phi,phi>, U = <v1 phi,phi>, Schi = <chi phi,phi>.
__global__ void k_mat1d(SwrDeviceView v) {
    const int sid = blockIdx.x, d = blockIdx.y;
    const SubDev& s = v.sub[sid];
    if (d >= s.N) return;
    double* T = v.arena + s.t1[d];
    T1Layout lay(s.q, s.kd);
    const int kd = s.kd, q = s.q;
    const double *x = T + lay.x(), *w = T + lay.w(), *chi = T + lay.chi(), *v1 = T + lay.v1();
    const double *B = T + lay.B(), *D = T + lay.D();
    for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
        int a = e / kd, c = e % kd;
        if (c < a) continue;
        double sS = 0, sK = 0, sX = 0, sU = 0, sC = 0;
        for (int n = 0; n < q; ++n) {
            double bb = w[n] * B[n * kd + a] * B[n * kd + c];
            sS += bb;
            sK += w[n] * D[n * kd + a] * D[n * kd + c];
            sX += bb * x[n];
            sU += bb * v1[n];
            sC += bb * chi[n];
        }
        double vals[5] = {sS, sK, sX, sU, sC};
        for (int m = 0; m < 5; ++m) {
            T[lay.mat(m) + a * kd + c] = vals[m];
            T[lay.mat(m) + c * kd + a] = vals[m];
        }
    }
}

// K4: per-coordinate orthonormalisation.  Cholesky S = L L^T (FP64, in shared
// memory), X = L^{-T} (upper triangular), then the orthonormal-basis 1-D
// matrices Tp = X^T Kf X, Up = X^T U X, Pp = X^T Schi X, Xp = X^T Xpos X,
// the transformed tables B' = B X, D' = D X, L' = L X and the Robin mass
// Rp = sum over interior sides of l' l'^T.
#define ORTH_MAX_KD 96
// Symmetric eigen-decomposition A = V diag(A_jj) V^T of an n x n matrix in
// shared memory by the cyclic Jacobi method with round-robin ordering: a
// sweep is n'-1 rounds (n' = n rounded up to even) of n'/2 disjoint index
// pairs, whose rotations commute and are applied together (two-sided on A,
// from the right on V).  Rotation of pair (p, q): t = sgn(r)/(|r| + sqrt(1+r^2)),
// r = (a_qq - a_pp)/(2 a_pq), c = 1/sqrt(1+t^2), s = t c zeroes a_pq.  Sweeps
// run until the off-diagonal mass is below 1e-28 of the diagonal one (at most
// 40).  On return A holds the eigenvalues on its diagonal, V the eigenvectors
// in its columns.
__device__ void jacobi_eig(double* A, double* V, int n) {
    __shared__ double s_c[ORTH_MAX_KD / 2], s_s[ORTH_MAX_KD / 2];
    __shared__ int s_p[ORTH_MAX_KD / 2], s_q[ORTH_MAX_KD / 2];
    __shared__ double s_red[2][32];
    __shared__ int s_done;
    const int m = n + (n & 1), np = m / 2;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0, dia = 0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const double a = A[e];
            if (e / n == e % n) dia += a * a;
            else off += a * a;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[0][threadIdx.x >> 5] = off;
            s_red[1][threadIdx.x >> 5] = dia;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double o2 = 0, d2 = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                o2 += s_red[0][w];
                d2 += s_red[1][w];
            }
            s_done = !(o2 > 1e-28 * d2);
        }
        __syncthreads();
        if (s_done) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int k = threadIdx.x; k < np; k += blockDim.x) {
                int p = (k == 0) ? r : (r + k) % (m - 1);
                int q = (k == 0) ? m - 1 : (r - k + (m - 1)) % (m - 1);
                double c = 1.0, sn = 0.0;
                if (p < n && q < n) {
                    const double apq = A[p * n + q];
                    if (apq != 0.0) {
                        const double rr = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                        const double t = (rr >= 0.0 ? 1.0 : -1.0) / (fabs(rr) + sqrt(1.0 + rr * rr));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                    }
                } else {
                    p = q = -1;
                }
                s_p[k] = p;
                s_q[k] = q;
                s_c[k] = c;
                s_s[k] = sn;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
                const int k = e / n, i = e - k * n, p = s_p[k], q = s_q[k];
                if (p < 0) continue;
                const double c = s_c[k], sn = s_s[k];
                const double aip = A[i * n + p], aiq = A[i * n + q];
                A[i * n + p] = c * aip - sn * aiq;
                A[i * n + q] = sn * aip + c * aiq;
                const double vip = V[i * n + p], viq = V[i * n + q];
                V[i * n + p] = c * vip - sn * viq;
                V[i * n + q] = sn * vip + c * viq;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
                const int k = e / n, j = e - k * n, p = s_p[k], q = s_q[k];
                if (p < 0) continue;
                const double c = s_c[k], sn = s_s[k];
                const double apj = A[p * n + j], aqj = A[q * n + j];
                A[p * n + j] = c * apj - sn * aqj;
                A[q * n + j] = sn * apj + c * aqj;
            }
            __syncthreads();
        }
    }
}

// Right-looking Cholesky of the n x n matrix in L (lower triangle; block-wide).
// Returns 1 when a pivot is not above tau * (largest diagonal entry).
__device__ int chol_block(double* L, int n, double tau) {
    __shared__ int s_bad;
    __shared__ double s_dmax;
    if (threadIdx.x == 0) {
        s_bad = 0;
        double m = 0;
        for (int j = 0; j < n; ++j) m = fmax(m, L[j * n + j]);
        s_dmax = m;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double pj = L[j * n + j];
            if (!(pj > tau * s_dmax)) { s_bad = 1; pj = 1.0; }
            L[j * n + j] = sqrt(pj);
        }
        __syncthreads();
        const double ljj = L[j * n + j];
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) L[i * n + j] /= ljj;
        __syncthreads();
        for (int e = threadIdx.x; e < (n - j - 1) * (n - j - 1); e += blockDim.x) {
            int i = j + 1 + e / (n - j - 1), c = j + 1 + e % (n - j - 1);
            if (c <= i) L[i * n + c] -= L[i * n + j] * L[c * n + j];
        }
        __syncthreads();
    }
    const int bad = s_bad;
    __syncthreads();
    return bad;
}

// L (Cholesky factor, lower) -> X = L^{-T} in L (upper triangular, explicit
// zeros below the diagonal); W is n x n scratch.
__device__ void chol_inv_t(double* L, double* W, int n) {
    for (int col = threadIdx.x; col < n; col += blockDim.x) {  // W <- L^{-1}
        for (int i = 0; i < n; ++i) {
            double acc = (i == col) ? 1.0 : 0.0;
            for (int k = col; k < i; ++k) acc -= L[i * n + k] * W[k * n + col];
            W[i * n + col] = (i < col) ? 0.0 : acc / L[i * n + i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        L[i * n + j] = W[j * n + i];  // X[i][j] = Linv[j][i]
    }
    __syncthreads();
}

__global__ void k_orth(SwrDeviceView v) {
    const int sid = blockIdx.x, d = blockIdx.y;
    const SubDev& s = v.sub[sid];
    if (d >= s.N) return;
    const double tau = v.inst[s.inst].orth_tau;
    extern __shared__ double sm[];
    const int kd = s.kd, q = s.q;
    double* Ls = sm;                 // kd*kd: L then X
    double* Ts = sm + kd * kd;       // kd*kd: temporary
    double* rowbuf = sm + 2 * kd * kd;  // 8 warps * kd
    double* T = v.arena + s.t1[d];
    T1Layout lay(q, kd);
    const double* Sg = T + lay.mat(M_S);
    double* Xc = T + lay.mat(M_XO);  // canonical X (global scratch; X is stored there at the end)
    for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) Ls[e] = Sg[e];
    __syncthreads();
    const int canonical = chol_block(Ls, kd, tau);
    if (canonical) {
        // canonical orthogonalisation: S = U diag(lam) U^T, keep lam > tau lam_max,
        // Xc = U_r lam_r^{-1/2}; the other columns are zero, so the dropped
        // directions stay zero in H', G, c0, b' and the norm
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) Ls[e] = Sg[e];
        __syncthreads();
        jacobi_eig(Ls, Ts, kd);
        __shared__ double s_lmax;
        if (threadIdx.x == 0) {
            double m = 0;
            for (int j = 0; j < kd; ++j) m = fmax(m, Ls[j * kd + j]);
            s_lmax = m;
        }
        __syncthreads();
        int* keep = (int*)rowbuf;  // kd flags
        for (int j = threadIdx.x; j < kd; j += blockDim.x) keep[j] = Ls[j * kd + j] > tau * s_lmax;
        __syncthreads();
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
            const int j = e % kd;
            Xc[e] = keep[j] ? Ts[e] / sqrt(Ls[j * kd + j]) : 0.0;
        }
        __syncthreads();
        // Xc^T S Xc equals I only to eps lam_max / lam (small kept eigenvalues):
        // Gram of the kept columns, G = Xc^T S Xc (e_j for dropped j), is
        // factorised and Xc re-orthonormalised, X = Xc G_L^{-T}, so X^T S X = I
        // to rounding
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {  // Ts = S Xc
            const int i = e / kd, j = e % kd;
            double acc = 0;
            for (int k = 0; k < kd; ++k) acc += Sg[i * kd + k] * Xc[k * kd + j];
            Ts[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {  // Ls = Xc^T Ts
            const int i = e / kd, j = e % kd;
            double acc = 0;
            if (keep[i] && keep[j])
                for (int k = 0; k < kd; ++k) acc += Xc[k * kd + i] * Ts[k * kd + j];
            else
                acc = (i == j) ? 1.0 : 0.0;
            Ls[e] = acc;
        }
        __syncthreads();
        if (chol_block(Ls, kd, 1e-3)) {  // G is near the identity: a failure is a fault
            if (threadIdx.x == 0) atomicOr(v.err, SWR_ERR_SINGULAR);
            return;
        }
    }
    chol_inv_t(Ls, Ts, kd);  // Ls = L^{-T}
    if (canonical) {
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {  // X = Xc L^{-T}
            const int i = e / kd, j = e % kd;
            double acc = 0;
            for (int k = 0; k < kd; ++k) acc += Xc[i * kd + k] * Ls[k * kd + j];
            Ts[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) Ls[e] = Ts[e];
        __syncthreads();
    }
    // from here on X (in Ls) is dense in general: the sums run over all k (with
    // the upper-triangular Cholesky X the extra terms are exact zeros)
    for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) T[lay.mat(M_XO) + e] = Ls[e];
    // congruence transforms X^T M X for M in {Kf, U, Schi, Xpos}
    const int srcm[4] = {M_KF, M_U, M_SCHI, M_XPOS};
    const int dstm[4] = {M_TP, M_UP, M_PP, M_XP};
    for (int m = 0; m < 4; ++m) {
        const double* Mg = T + lay.mat(srcm[m]);
        __syncthreads();
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {  // Ts = M X
            int i = e / kd, j = e % kd;
            double acc = 0;
            for (int k = 0; k < kd; ++k) acc += Mg[i * kd + k] * Ls[k * kd + j];
            Ts[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {  // X^T Ts
            int i = e / kd, j = e % kd;
            double acc = 0;
            for (int k = 0; k < kd; ++k) acc += Ls[k * kd + i] * Ts[k * kd + j];
            T[lay.mat(dstm[m]) + e] = acc;
        }
    }
    __syncthreads();
    // tables: rows of B, D (q rows each) and Lv, Ld (4 rows each) times X
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* rb = rowbuf + warp * kd;
    const long long bases[4] = {lay.B(), lay.D(), lay.Lv(), lay.Ld()};
    const int rows[4] = {q, q, 4, 4};
    for (int tb = 0; tb < 4; ++tb) {
        for (int r = warp; r < rows[tb]; r += nw) {
            double* row = T + bases[tb] + (long long)r * kd;
            for (int k = lane; k < kd; k += 32) rb[k] = row[k];
            __syncwarp();
            for (int j = lane; j < kd; j += 32) {
                double acc = 0;
                for (int k = 0; k < kd; ++k) acc += rb[k] * Ls[k * kd + j];
                row[j] = acc;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // Robin mass of the interior sides of this coordinate: lo -> line 0, hi -> line 3
    for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
        int i = e / kd, j = e % kd;
        double acc = 0;
        if (s.edge_mask & (1 << (2 * d + 0))) acc += T[lay.Lv() + 0 * kd + i] * T[lay.Lv() + 0 * kd + j];
        if (s.edge_mask & (1 << (2 * d + 1))) acc += T[lay.Lv() + 3 * kd + i] * T[lay.Lv() + 3 * kd + j];
        T[lay.mat(M_RP) + e] = acc;
    }
}

// ------------------------------------------------------- electron-electron

// Work buffer layout of a 2-electron subdomain (doubles): P1 [q][kd^2],
// P2 [q][kd^2], Wv [q][q], Mee [q][kd^2].
struct EeWork {
    int q, kd2;
    __host__ __device__ EeWork(int q_, int kd) : q(q_), kd2(kd * kd) {}
    __host__ __device__ long long P1() const { return 0; }
    __host__ __device__ long long P2() const { return (long long)q * kd2; }
    __host__ __device__ long long Wv() const { return 2LL * q * kd2; }
    __host__ __device__ long long Mee() const { return 2LL * q * kd2 + (long long)q * q; }
    __host__ __device__ long long size() const { return 3LL * q * kd2 + (long long)q * q; }
};

// P_d[n][(a,c)] = B'_d[n][a] B'_d[n][c]; Wv[n1][n2] = w1 w2 ee / sqrt((x1-x2)^2 + eta^2).
__global__ void k_ee_operands(SwrDeviceView v) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    if (s.N != 2) return;
    const InstDev& in = v.inst[s.inst];
    const int kd = s.kd, q = s.q, kd2 = kd * kd;
    EeWork ew(q, kd);
    double* W = v.arena + s.work;
    T1Layout lay(q, kd);
    const double* T0 = v.arena + s.t1[0];
    const double* T1 = v.arena + s.t1[1];
    for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < (long long)q * kd2;
         e += (long long)blockDim.x * gridDim.y) {
        int n = (int)(e / kd2), ac = (int)(e % kd2), a = ac / kd, c = ac % kd;
        W[ew.P1() + e] = T0[lay.B() + n * kd + a] * T0[lay.B() + n * kd + c];
        W[ew.P2() + e] = T1[lay.B() + n * kd + a] * T1[lay.B() + n * kd + c];
    }
    for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < (long long)q * q;
         e += (long long)blockDim.x * gridDim.y) {
        int n1 = (int)(e / q), n2 = (int)(e % q);
        double r = T0[lay.x() + n1] - T1[lay.x() + n2];
        W[ew.Wv() + e] = T0[lay.w() + n1] * T1[lay.w() + n2] * in.ee_coef / sqrt(r * r + in.eta_ee * in.eta_ee);
    }
}

// Batched FP64 GEMM  C = op(A) * B  with 64x64 tiles.  One batch entry per
// subdomain (blockIdx.z); its sizes and offsets come from a GemmJob.

#define GT 64
#define GK 16
__global__ void __launch_bounds__(256) k_dgemm(SwrDeviceView v, const GemmJob* jobs) {
    const GemmJob jb = jobs[blockIdx.z];
    const int tm = blockIdx.y * GT, tn = blockIdx.x * GT;
    if (jb.M <= 0 || tm >= jb.M || tn >= jb.N) return;
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const double* A = v.arena + jb.a;
    const double* B = v.arena + jb.b;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < jb.K; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            int kk = e / GT, mm = e % GT;
            int gk = k0 + kk, gm = tm + mm;
            double val = 0.0;
            if (gk < jb.K && gm < jb.M)
                val = jb.transA ? A[(long long)gk * jb.lda + gm] : A[(long long)gm * jb.lda + gk];
            As[kk][mm] = val;
            int gn = tn + mm;
            Bs[kk][mm] = (gk < jb.K && gn < jb.N) ? B[(long long)gk * jb.ldb + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double ar[4], br[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ar[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) br[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* C = v.arena + jb.c;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gm = tm + ty + 16 * i, gn = tn + tx + 16 * j;
            if (gm >= jb.M || gn >= jb.N) continue;
            if (jb.mode == 0) {
                C[(long long)gm * jb.ldc + gn] = acc[i][j];
            } else {
                // gm = (a,c) = a*kd + c, gn = (b,d) = b*kd + e; H'[(a + kd b), (c + kd e)]
                int kd = jb.kd;
                int a = gm / kd, c = gm % kd, b = gn / kd, e = gn % kd;
                long long K = (long long)kd * kd;
                C[(long long)(a + kd * b) * K + (c + kd * e)] = acc[i][j];
            }
        }
}

// H' += Kronecker-sum terms:  kappa (Tp (+) Tp) + (Up (+) Up) + kappa mu_re (Rp (+) Rp).
// For N = 1 this writes H' = kappa Tp + Up + kappa mu_re Rp (no e-e block).
__global__ void k_h_kron(SwrDeviceView v, int has_ee) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int kd = s.kd, K = s.K;
    T1Layout lay(s.q, kd);
    const double* T0 = v.arena + s.t1[0];
    const double* T1 = v.arena + s.t1[s.N == 2 ? 1 : 0];
    double* Hm = v.arena + s.Hm;
    const double kap = in.kappa, kmu = in.kappa * in.mu_re;
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < (long long)K * K;
         e += (long long)blockDim.x * gridDim.x) {
        int r = (int)(e / K), c = (int)(e % K);
        double h;
        if (s.N == 1) {
            h = kap * T0[lay.mat(M_TP) + r * kd + c] + T0[lay.mat(M_UP) + r * kd + c] +
                kmu * T0[lay.mat(M_RP) + r * kd + c];
            Hm[e] = h;
        } else {
            int a = r % kd, b = r / kd, cc = c % kd, dd = c / kd;
            h = 0.0;
            if (b == dd)
                h += kap * T0[lay.mat(M_TP) + a * kd + cc] + T0[lay.mat(M_UP) + a * kd + cc] +
                     kmu * T0[lay.mat(M_RP) + a * kd + cc];
            if (a == cc)
                h += kap * T1[lay.mat(M_TP) + b * kd + dd] + T1[lay.mat(M_UP) + b * kd + dd] +
                     kmu * T1[lay.mat(M_RP) + b * kd + dd];
            Hm[e] = (has_ee ? Hm[e] : 0.0) + h;
        }
    }
}

// Symmetrise H' (the sum-factorised e-e block is symmetric up to rounding).
__global__ void k_symmetrize(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K;
    double* Hm = v.arena + s.Hm;
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < (long long)K * K;
         e += (long long)blockDim.x * gridDim.x) {
        int r = (int)(e / K), c = (int)(e % K);
        if (c <= r) continue;
        double m = 0.5 * (Hm[(long long)r * K + c] + Hm[(long long)c * K + r]);
        Hm[(long long)r * K + c] = m;
        Hm[(long long)c * K + r] = m;
    }
}

// Step matrix into G: TISE  M = I + dt H';  TDSE  M0 = I + i dt/2 (H' + i kappa mu_im R'),
// R' = Rp (+) Rp (complex, interleaved re/im).
__global__ void k_step_matrix(SwrDeviceView v) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int K = s.K, kd = s.kd;
    const double* Hm = v.arena + s.Hm;
    double* G = v.arena + s.Gm;
    T1Layout lay(s.q, kd);
    const double* T0 = v.arena + s.t1[0];
    const double* T1 = v.arena + s.t1[s.N == 2 ? 1 : 0];
    for (long long e = threadIdx.x + (long long)blockIdx.x * blockDim.x; e < (long long)K * K;
         e += (long long)blockDim.x * gridDim.x) {
        int r = (int)(e / K), c = (int)(e % K);
        double id = (r == c) ? 1.0 : 0.0;
        if (in.mode == SWR_MODE_TISE) {
            G[e] = id + in.dt * Hm[e];
        } else {
            double rr;
            if (s.N == 1) {
                rr = T0[lay.mat(M_RP) + r * kd + c];
            } else {
                int a = r % kd, b = r / kd, cc = c % kd, dd = c / kd;
                rr = 0.0;
                if (b == dd) rr += T0[lay.mat(M_RP) + a * kd + cc];
                if (a == cc) rr += T1[lay.mat(M_RP) + b * kd + dd];
            }
            double hi = in.kappa * in.mu_im * rr;   // imaginary part of H'
            // I + i dt/2 (Hr + i Hi) = (I - dt/2 Hi) + i dt/2 Hr
            G[2 * e] = id - 0.5 * in.dt * hi;
            G[2 * e + 1] = 0.5 * in.dt * Hm[e];
        }
    }
}

// ------------------------------------------------------ Gauss-Jordan inverse

template <typename T> __device__ inline T ld_el(const double* p, long long i);
template <> __device__ inline double ld_el<double>(const double* p, long long i) { return p[i]; }
template <> __device__ inline cplx ld_el<cplx>(const double* p, long long i) { return mkc(p[2 * i], p[2 * i + 1]); }
template <typename T> __device__ inline void st_el(double* p, long long i, T x);
template <> __device__ inline void st_el<double>(double* p, long long i, double x) { p[i] = x; }
template <> __device__ inline void st_el<cplx>(double* p, long long i, cplx x) { p[2 * i] = x.re; p[2 * i + 1] = x.im; }
__device__ inline double inv_el(double x) { return 1.0 / x; }
__device__ inline cplx inv_el(cplx x) {
    double d = x.re * x.re + x.im * x.im;
    return mkc(x.re / d, -x.im / d);
}
__device__ inline double mag2(double x) { return x * x; }
__device__ inline double mag2(cplx x) { return x.re * x.re + x.im * x.im; }
__device__ inline double neg(double x) { return -x; }
__device__ inline cplx neg(cplx x) { return mkc(-x.re, -x.im); }
__device__ inline double zero_el(double) { return 0.0; }
__device__ inline cplx zero_el(cplx) { return mkc(0.0, 0.0); }
__device__ inline double one_el(double) { return 1.0; }
__device__ inline cplx one_el(cplx) { return mkc(1.0, 0.0); }

#define GJ_NB 32
// Scratch per subdomain (elements of T): Pinv [NB][NB], Rp [NB][K], Cp [K][NB].
template <typename T>
__global__ void k_gj_panel(SwrDeviceView v, int kb) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const int K = s.K, k0 = kb * GJ_NB;
    if (k0 >= K) return;
    const int nb = min(GJ_NB, K - k0);
    double* M = v.arena + s.Gm;
    double* W = v.arena + s.work;
    __shared__ T P[GJ_NB][GJ_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        P[i][j] = ld_el<T>(M, (long long)(k0 + i) * K + k0 + j);
    }
    __syncthreads();
    // unblocked in-place Gauss-Jordan inversion of the nb x nb block (no pivoting:
    // the step matrices have a positive definite Hermitian part)
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        __shared__ T piv_inv;
        if (threadIdx.x == 0) {
            T pv = P[p][p];
            double m = mag2(pv);
            if (!(m > 1e-280) || !isfinite(m)) { s_bad = 1; pv = one_el(T()); }
            piv_inv = inv_el(pv);
        }
        __syncthreads();
        T pinv = piv_inv;
        // column p of the other rows, saved before the update
        __shared__ T colp[GJ_NB];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) colp[i] = P[i][p];
        __syncthreads();
        // row p scaled
        for (int j = threadIdx.x; j < nb; j += blockDim.x) P[p][j] = (j == p) ? pinv : pinv * P[p][j];
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            int i = e / nb, j = e % nb;
            if (i == p) continue;
            if (j == p) P[i][j] = neg(colp[i] * pinv);
            else P[i][j] = P[i][j] - colp[i] * P[p][j];
        }
        __syncthreads();
    }
    if (s_bad && threadIdx.x == 0) atomicOr(v.err, SWR_ERR_SINGULAR);
    // scratch
    double* Pinv = W;
    double* Rp = W + (sizeof(T) / 8) * GJ_NB * GJ_NB;
    double* Cp = Rp + (sizeof(T) / 8) * (long long)GJ_NB * K;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) st_el<T>(Pinv, e / nb * GJ_NB + e % nb, P[e / nb][e % nb]);
    // Rp = Pinv * M[kb, :]   (nb x K)
    for (long long e = threadIdx.x; e < (long long)nb * K; e += blockDim.x) {
        int i = (int)(e / K), j = (int)(e % K);
        T acc = zero_el(T());
        for (int t = 0; t < nb; ++t) acc = acc + P[i][t] * ld_el<T>(M, (long long)(k0 + t) * K + j);
        st_el<T>(Rp, (long long)i * K + j, acc);
    }
    // Cp = M[:, kb]   (K x nb)
    for (long long e = threadIdx.x; e < (long long)K * nb; e += blockDim.x) {
        int i = (int)(e / nb), j = (int)(e % nb);
        st_el<T>(Cp, (long long)i * GJ_NB + j, ld_el<T>(M, (long long)i * K + k0 + j));
    }
}

// Rank-nb update of the whole matrix for block column kb (TILE x TILE tiles:
// 64 for real, 32 for complex so that the staged panels stay under 48 KB).
template <typename T> struct GjTile { static const int v = 64; };
template <> struct GjTile<cplx> { static const int v = 32; };

template <typename T>
__global__ void __launch_bounds__(256) k_gj_update(SwrDeviceView v, int kb) {
    constexpr int TL = GjTile<T>::v;
    const int sid = blockIdx.z;
    const SubDev& s = v.sub[sid];
    const int K = s.K, k0 = kb * GJ_NB;
    if (k0 >= K) return;
    const int tm = blockIdx.y * TL, tn = blockIdx.x * TL;
    if (tm >= K || tn >= K) return;
    const int nb = min(GJ_NB, K - k0);
    double* M = v.arena + s.Gm;
    const double* W = v.arena + s.work;
    const double* Pinv = W;
    const double* Rp = W + (sizeof(T) / 8) * GJ_NB * GJ_NB;
    const double* Cp = Rp + (sizeof(T) / 8) * (long long)GJ_NB * K;
    __shared__ T Cs[TL][GJ_NB + 1];
    __shared__ T Rs[GJ_NB][TL + 1];
    for (int e = threadIdx.x; e < TL * GJ_NB; e += 256) {
        int i = e / GJ_NB, t = e % GJ_NB;
        int gi = tm + i;
        Cs[i][t] = (gi < K && t < nb) ? ld_el<T>(Cp, (long long)gi * GJ_NB + t) : zero_el(T());
    }
    for (int e = threadIdx.x; e < GJ_NB * TL; e += 256) {
        int t = e / TL, j = e % TL;
        int gj = tn + j;
        T r = zero_el(T());
        if (gj < K && t < nb) {
            if (gj >= k0 && gj < k0 + nb) r = ld_el<T>(Pinv, (long long)t * GJ_NB + (gj - k0));
            else r = ld_el<T>(Rp, (long long)t * K + gj);
        }
        Rs[t][j] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TL * TL; e += 256) {
        int i = e / TL, j = e % TL;
        int gi = tm + i, gj = tn + j;
        if (gi >= K || gj >= K) continue;
        bool ri = gi >= k0 && gi < k0 + nb, cj = gj >= k0 && gj < k0 + nb;
        long long idx = (long long)gi * K + gj;
        if (ri) {
            st_el<T>(M, idx, Rs[gi - k0][j]);     // row block: Pinv * M[kb,:] (Pinv on the diagonal block)
        } else {
            T acc = zero_el(T());
#pragma unroll 8
            for (int t = 0; t < GJ_NB; ++t) acc = acc + Cs[i][t] * Rs[t][j];
            if (cj) st_el<T>(M, idx, neg(acc));            // -C * Pinv
            else st_el<T>(M, idx, ld_el<T>(M, idx) - acc); // M - C * R
        }
    }
}

// ------------------------------------------------------------ initial data

// c0 = (B'1^T W f1) (x) (B'2^T W f2) for phi0 = prod_e exp(-gamma (x_e - x0_e)^2)
// (projection of Sec. 6.1 in the orthonormal basis: c' = X^T c~).
// out[sid] = partial PoU norm^2 of c0 (later summed per instance).
__global__ void k_project(SwrDeviceView v, double* norm_part) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int kd = s.kd, q = s.q;
    T1Layout lay(q, kd);
    __shared__ double u[2][ORTH_MAX_KD * 4];
    __shared__ double nrm[2];
    for (int d = 0; d < s.N; ++d) {
        const double* T = v.arena + s.t1[d];
        for (int a = threadIdx.x; a < kd; a += blockDim.x) {
            double acc = 0;
            for (int n = 0; n < q; ++n) {
                double r = T[lay.x() + n] - in.x0[d];
                acc += T[lay.w() + n] * exp(-in.gamma0 * r * r) * T[lay.B() + n * kd + a];
            }
            u[d][a] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0;
            for (int a = 0; a < kd; ++a)
                for (int c = 0; c < kd; ++c) acc += u[d][a] * T[lay.mat(M_PP) + a * kd + c] * u[d][c];
            nrm[d] = acc;
        }
        __syncthreads();
    }
    double* c0 = v.arena + s.c0;
    const bool cpx = in.mode == SWR_MODE_TDSE;
    for (int m = threadIdx.x; m < s.K; m += blockDim.x) {
        double val = (s.N == 1) ? u[0][m] : u[0][m % kd] * u[1][m / kd];
        c0[m] = val;                 // planar: real block ...
        if (cpx) c0[s.K + m] = 0.0;  // ... then imaginary block
    }
    if (threadIdx.x == 0) norm_part[sid] = (s.N == 1) ? nrm[0] : nrm[0] * nrm[1];
}

// Antisymmetric states (Appendix A): the initial data of each mirror pair
// (sigma(i) = (i2, i1) of subdomain (i1, i2)) replaced by its antisymmetric
// part, c0_i <- (c0_i - swap(c0_sigma(i))) / 2 and c0_sigma(i) = -swap(c0_i)
// (swap: coefficient (a, b) -> (b, a)), with the partition-of-unity norm
// c0^T (Pp (x) Pp) c0 of both for the normalisation that follows.  One block
// per subdomain; the block of the upper (or diagonal) subdomain of a pair
// writes both.
__global__ void k_anti_c0(SwrDeviceView v, double* norm_part) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    if (!in.anti || s.N != 2) return;
    const int loc = sid - in.sub_base, i1 = loc % in.L, i2 = loc / in.L;
    if (i1 > i2) return;
    const int msid = in.sub_base + i2 + in.L * i1;
    const int kd = s.kd, K = s.K;
    __shared__ double y[32 * 32], tmp[32 * 32];
    __shared__ double red[8];
    double* c0 = v.arena + s.c0;
    double* cm = v.arena + v.sub[msid].c0;
    for (int c = threadIdx.x; c < K; c += blockDim.x) y[c] = 0.5 * (c0[c] - cm[c / kd + kd * (c % kd)]);
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        c0[c] = y[c];
        if (msid != sid) cm[c / kd + kd * (c % kd)] = -y[c];
    }
    T1Layout lay(s.q, kd);
    const double* P1 = v.arena + s.t1[0] + lay.mat(M_PP);
    const double* P2 = v.arena + s.t1[1] + lay.mat(M_PP);
    for (int it = threadIdx.x; it < kd * kd; it += blockDim.x) {  // tmp[c][b] = sum_e y[c + kd e] P2[b][e]
        const int c = it / kd, b = it - c * kd;
        double acc = 0;
        for (int e = 0; e < kd; ++e) acc = fma(y[c + kd * e], P2[b * kd + e], acc);
        tmp[it] = acc;
    }
    __syncthreads();
    double part = 0;
    for (int m = threadIdx.x; m < K; m += blockDim.x) {  // y[(a,b)] sum_c P1[a][c] tmp[c][b]
        const int b = m / kd, a = m - b * kd;
        double z = 0;
        for (int c = 0; c < kd; ++c) z = fma(P1[a * kd + c], tmp[c * kd + b], z);
        part += y[m] * z;
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        norm_part[sid] = t;
        norm_part[msid] = t;
    }
}

// Per-instance normalisation of c0 (TISE with normalisation).
__global__ void k_normalize_c0(SwrDeviceView v, const double* norm_part) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    if (in.mode != SWR_MODE_TISE || !in.normalize) return;
    __shared__ double sc;
    if (threadIdx.x == 0) {
        double acc = 0;
        for (int j = 0; j < in.n_sub; ++j) acc += norm_part[in.sub_base + j];
        sc = 1.0 / sqrt(acc);
    }
    __syncthreads();
    double* c0 = v.arena + s.c0;
    for (int m = threadIdx.x; m < s.K; m += blockDim.x) c0[m] *= sc;
}

// ------------------------------------------------------------- host driver

static inline unsigned div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Launches of an assembly besides the e-e block (3) and the Gauss-Jordan
// panels/updates (2 per block column): tabulate, mat1d, orth, h_kron,
// symmetrize, step_matrix, project, anti_c0, normalize_c0.
extern const int kAssembleLaunchesFixed = 9;

struct TgState;
cudaError_t tg_update(const TgState* g, const SwrDeviceView& v, cudaStream_t st, int kb, int max_K);
bool tg_has_ee(const TgState* g);
cudaError_t te_products(const TgState* g, const SwrDeviceView& v, cudaStream_t st, const GemmJob* d_jobs1,
                        const GemmJob* d_jobs2);

// tg: the tensor-core Gauss-Jordan state (swr_tcgj.cu) or null for the FP64 updates.
cudaError_t launch_assemble(const SwrDeviceView& v, cudaStream_t st, int max_q, int max_kd, int max_K,
                            bool any_ee, bool any_tdse, bool any_tise, const GemmJob* d_jobs1,
                            const GemmJob* d_jobs2, double* d_norm_part, const TgState* tg) {
    dim3 g2(v.n_sub, 2);
    k_tabulate<<<g2, 256, 0, st>>>(v);
    k_mat1d<<<g2, 256, 0, st>>>(v);
    size_t sm = (2 * (size_t)max_kd * max_kd + 8 * (size_t)max_kd) * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_orth<<<g2, 256, sm, st>>>(v);
    if (any_ee) {
        k_ee_operands<<<dim3(v.n_sub, 16), 256, 0, st>>>(v);
        if (tg_has_ee(tg)) {
            // the same two products on the tensor cores (FP64 emulated by BF16 slices)
            cudaError_t e = te_products(tg, v, st, d_jobs1, d_jobs2);
            if (e != cudaSuccess) return e;
        } else {
            int kd2 = max_kd * max_kd;
            // Mee = Wv (q x q) * P2 (q x kd^2)
            k_dgemm<<<dim3(div_up(kd2, GT), div_up(max_q, GT), v.n_sub), 256, 0, st>>>(v, d_jobs1);
            // V'ee[(a,c),(b,e)] = P1^T (kd^2 x q) * Mee (q x kd^2), scattered into H'
            k_dgemm<<<dim3(div_up(kd2, GT), div_up(kd2, GT), v.n_sub), 256, 0, st>>>(v, d_jobs2);
        }
    }
    dim3 ge(div_up((long long)max_K * max_K, 256 * 8), v.n_sub);
    k_h_kron<<<ge, 256, 0, st>>>(v, any_ee ? 1 : 0);
    k_symmetrize<<<ge, 256, 0, st>>>(v);
    k_step_matrix<<<ge, 256, 0, st>>>(v);
    int nkb = (max_K + GJ_NB - 1) / GJ_NB;
    for (int kb = 0; kb < nkb; ++kb) {
        if (any_tdse) {
            dim3 gu(div_up(max_K, 32), div_up(max_K, 32), v.n_sub);
            k_gj_panel<cplx><<<v.n_sub, 256, 0, st>>>(v, kb);
            if (tg) {
                cudaError_t e = tg_update(tg, v, st, kb, max_K);
                if (e != cudaSuccess) return e;
            } else {
                k_gj_update<cplx><<<gu, 256, 0, st>>>(v, kb);
            }
        } else {
            dim3 gu(div_up(max_K, 64), div_up(max_K, 64), v.n_sub);
            k_gj_panel<double><<<v.n_sub, 256, 0, st>>>(v, kb);
            if (tg) {
                cudaError_t e = tg_update(tg, v, st, kb, max_K);
                if (e != cudaSuccess) return e;
            } else {
                k_gj_update<double><<<gu, 256, 0, st>>>(v, kb);
            }
        }
    }
    k_project<<<v.n_sub, 256, 0, st>>>(v, d_norm_part);
    k_anti_c0<<<v.n_sub, 256, 0, st>>>(v, d_norm_part);
    k_normalize_c0<<<v.n_sub, 256, 0, st>>>(v, d_norm_part);
    return cudaGetLastError();
}

}  // namespace swr
