// swr_tcgj.cu -- trailing updates of the blocked Gauss-Jordan inversion of the
// step matrices (Sec. 5.4 step 2: the local systems (I + dt H') and
// I + i dt/2 H') on the 5th-generation tensor cores, with FP64 emulated by
// exact BF16 slices.
//
// The update of block column kb is M <- M - C R for the pivot column block C
// (K x nb, nb = 32) and the pivot row block R (nb x K, Pinv on the pivot
// columns), a rank-32 product.  Every row i of C is written as
// 2^e_i sum_s 2^(-7(s+1)) A_s[i] with A_s integers in [-127, 127] (9 slices,
// 63 bits), every column j of R likewise with 2^f_j; BF16 holds these
// integers exactly, a product of two slices summed over the 32 (64 for
// complex data) inner terms stays below 2^24 and is exact in the tensor
// cores' FP32 accumulator, and so is the sum of the (at most 9) slice pairs
// of one level L = s + u.  The kernel keeps one tensor-memory accumulator per
// level L = 0..9 (53 slice pairs) and forms
//     (C R)_ij = 2^(e_i + f_j - 14) sum_L 2^(-7 L) acc_L[i][j]
// in FP64.  A pair of level L contributes at most (inner length) 2^(-7 L) of
// max|C_i| max|R_j|: the dropped levels (L >= 10) and the slicing remainders
// (2^-63) stay below 2^-63 times the inner length, under the rounding of an
// FP64 dot product.  Complex data (real time) take two real products with a
// 64-long inner dimension:
//     Re(C R) = [Cr | Ci] [Rr ; -Ri],   Im(C R) = [Cr | Ci] [Ri ; Rr].
//
// Operands: the slices live in global memory as [slice][row][inner] BF16
// arrays (rows of all subdomains concatenated) and reach shared memory by
// tensor-map bulk copies (cp.async.bulk.tensor, boxes of 8 inner elements
// by 128 (A) or 32 (B) rows, no swizzle: each box is a column of K-major
// core matrices, 16 bytes per row); one thread issues them against an
// mbarrier with the expected byte count, then issues the tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32 in tensor memory, M = 128, N = 32 for real
// and 16 for complex data) and
// commits them to a second mbarrier.  Both waits are bounded: on timeout the
// error flag is set, the products in flight are waited for (bounded), the
// tensor memory is freed and the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "swr_internal.cuh"

namespace swr {

#define TG_NB 32        // Gauss-Jordan block (the same as the FP64 path's)
#define TG_M 128        // rows of C per CTA
#define TG_S 9          // slices per operand
#define TG_LV 10        // levels L = s + u kept: 0..9
#define TG_TMEM 512     // tensor-memory columns per CTA (TG_LV x N x parts <= 512)
#define TG_THREADS 128
#define TG_SPIN (1LL << 22)

template <typename T> struct TgInner { static const int v = 32; };   // inner length of one product
template <> struct TgInner<cplx> { static const int v = 64; };
template <typename T> struct TgParts { static const int v = 1; };    // products per tile
template <> struct TgParts<cplx> { static const int v = 2; };
template <typename T> struct TgN { static const int v = 32; };       // columns of R per CTA
template <> struct TgN<cplx> { static const int v = 16; };

__device__ inline double tg_re(double x) { return x; }
__device__ inline double tg_re(cplx x) { return x.re; }
__device__ inline double tg_im(double) { return 0.0; }
__device__ inline double tg_im(cplx x) { return x.im; }
template <typename T> __device__ inline T tg_ld(const double* p, long long i);
template <> __device__ inline double tg_ld<double>(const double* p, long long i) { return p[i]; }
template <> __device__ inline cplx tg_ld<cplx>(const double* p, long long i) { return mkc(p[2 * i], p[2 * i + 1]); }

// Exponent e with |x| < 2^e for every |x| <= amax (0 for amax = 0).
__device__ inline int tg_exponent(double amax) {
    int e = 0;
    if (amax > 0.0) frexp(amax, &e);
    return e;
}

// The TG_S slices of x * 2^-e (|x 2^-e| < 1), each an integer in [-127, 127].
__device__ inline void tg_slice(double x, int e, __nv_bfloat16* out, long long slice_stride) {
    double r = ldexp(x, -e);
#pragma unroll
    for (int s = 0; s < TG_S; ++s) {
        r *= 128.0;
        const double a = trunc(r);
        r -= a;
        out[s * slice_stride] = __double2bfloat16(a);
    }
}

// Slices of the pivot column block C = M[:, kb] (scratch Cp, K x TG_NB) of every
// subdomain: A[s][row0 + i][k], k over [Re C_i | Im C_i] (zero beyond nb).
template <typename T>
__global__ void k_tg_slice_a(SwrDeviceView v, int kb, __nv_bfloat16* As, int* Aexp, const long long* rowoff,
                             long long R) {
    constexpr int KI = TgInner<T>::v;
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, k0 = kb * TG_NB;
    if (k0 >= K) return;
    const int nb = min(TG_NB, K - k0);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const double* W = v.arena + s.work;
    const double* Cp = W + (sizeof(T) / 8) * ((long long)TG_NB * TG_NB + (long long)TG_NB * K);
    double amax = 0.0;
    for (int t = 0; t < nb; ++t) {
        const T c = tg_ld<T>(Cp, (long long)i * TG_NB + t);
        amax = fmax(amax, fmax(fabs(tg_re(c)), fabs(tg_im(c))));
    }
    const int e = tg_exponent(amax);
    const long long row = rowoff[sid] + i;
    Aexp[row] = e;
    for (int k = 0; k < KI; ++k) {
        const int t = k % TG_NB;
        double x = 0.0;
        if (t < nb) {
            const T c = tg_ld<T>(Cp, (long long)i * TG_NB + t);
            x = k < TG_NB ? tg_re(c) : tg_im(c);
        }
        tg_slice(x, e, As + row * KI + k, R * KI);
    }
}

// Slices of the pivot row block R (Rp, Pinv on the pivot columns) by columns:
// B[p][s][col0 + j][k]; real: k over R[:, j]; complex: p = 0 gives
// [Re R[:, j] ; -Im R[:, j]], p = 1 gives [Im R[:, j] ; Re R[:, j]].
template <typename T>
__global__ void k_tg_slice_b(SwrDeviceView v, int kb, __nv_bfloat16* Bs, int* Bexp, const long long* coloff,
                             long long C) {
    constexpr int KI = TgInner<T>::v;
    constexpr int P = TgParts<T>::v;
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const int K = s.K, k0 = kb * TG_NB;
    if (k0 >= K) return;
    const int nb = min(TG_NB, K - k0);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const double* W = v.arena + s.work;
    const double* Pinv = W;
    const double* Rp = W + (sizeof(T) / 8) * TG_NB * TG_NB;
    const bool piv = j >= k0 && j < k0 + nb;
    auto rel = [&](int t) -> T {
        return piv ? tg_ld<T>(Pinv, (long long)t * TG_NB + (j - k0)) : tg_ld<T>(Rp, (long long)t * K + j);
    };
    double amax = 0.0;
    for (int t = 0; t < nb; ++t) {
        const T r = rel(t);
        amax = fmax(amax, fmax(fabs(tg_re(r)), fabs(tg_im(r))));
    }
    const int e = tg_exponent(amax);
    const long long col = coloff[sid] + j;
    Bexp[col] = e;
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < KI; ++k) {
            const int t = k % TG_NB;
            double x = 0.0;
            if (t < nb) {
                const T r = rel(t);
                if (P == 1) x = tg_re(r);
                else if (p == 0) x = k < TG_NB ? tg_re(r) : -tg_im(r);
                else x = k < TG_NB ? tg_im(r) : tg_re(r);
            }
            tg_slice(x, e, Bs + ((long long)p * TG_S * C + col) * KI + k, C * KI);
        }
}

__device__ inline unsigned tg_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Levels of one output element combined exactly on the integer pipe: every
// level accumulator is an integer below 2^24 in magnitude (exact in FP32), so
// with B bits per slice the levels 0..LH-1 and LH..LV-1 sum exactly into two
// int64 values, hi = sum_{L<LH} acc_L 2^(B (LH-1-L)) and lo = sum_{L>=LH}
// acc_L 2^(B (LV-1-L)); the element is hi 2^(-B (LH-1)) + lo 2^(-B (LV-1)),
// formed with two conversions and one FMA on the FP64 pipe.
struct TgLevels {
    long long hi, lo;
};
template <int B, int LV, int LH>
__device__ inline void tg_level_add(TgLevels& t, int L, float acc) {
    const long long a = (long long)__float2int_rz(acc);
    if (L < LH) t.hi += a << (B * (LH - 1 - L));
    else t.lo += a << (B * (LV - 1 - L));
}
template <int B, int LV, int LH>
__device__ inline double tg_level_value(const TgLevels& t, int ex) {
    return fma((double)t.lo, ldexp(1.0, ex - B * (LV - 1)), (double)t.hi * ldexp(1.0, ex - B * (LH - 1)));
}

// K-major, no swizzle: start, lbo = bytes between core matrices adjacent in
// the inner (K) direction, sbo = bytes between core matrices adjacent in M/N.
__device__ inline unsigned long long tg_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    unsigned long long d = (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ULL << 46;
    return d;
}

__device__ inline bool tg_wait(unsigned mbar, unsigned parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ inline void tg_tma3(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

// One 128 x N tile of the update of block column kb of subdomain blockIdx.z.
// Dynamic shared memory: A slices [S][KI/8 boxes][128 rows][16 B] then B slices
// [P][S][KI/8][N rows][16 B].
template <typename T>
__global__ void __launch_bounds__(TG_THREADS, 1) k_tg_update(SwrDeviceView v, int kb,
                                                             const __grid_constant__ CUtensorMap mapA,
                                                             const __grid_constant__ CUtensorMap mapB,
                                                             const int* Aexp, const int* Bexp,
                                                             const long long* rowoff, const long long* coloff) {
    constexpr int KI = TgInner<T>::v, P = TgParts<T>::v, NBOX = KI / 8, TG_N = TgN<T>::v;
    constexpr unsigned A_BYTES = TG_S * NBOX * TG_M * 16, B_BYTES = P * TG_S * NBOX * TG_N * 16;
    constexpr unsigned TMEM_COLS = TG_TMEM;
    static_assert(P * TG_LV * TG_N <= TG_TMEM, "level accumulators exceed the tensor memory");
    const int sid = blockIdx.z;
    const SubDev& s = v.sub[sid];
    const int K = s.K, k0 = kb * TG_NB;
    const int tm = blockIdx.y * TG_M, tn = blockIdx.x * TG_N;
    if (k0 >= K || tm >= K || tn >= K) return;
    const int nb = min(TG_NB, K - k0);
    extern __shared__ __align__(1024) unsigned char tg_sm[];
    unsigned char* Asm = tg_sm;
    unsigned char* Bsm = tg_sm + A_BYTES;
    __shared__ __align__(8) unsigned long long bar_ld, bar_mma;
    __shared__ unsigned tmem_slot;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tg_smem(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tg_smem(&bar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tg_smem(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // operands: one thread posts every box against bar_ld
    if (threadIdx.x == 0) {
        const unsigned mb = tg_smem(&bar_ld);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(A_BYTES + B_BYTES)
                     : "memory");
        const int row0 = (int)(rowoff[sid] + tm), col0 = (int)(coloff[sid] + tn);
        for (int sl = 0; sl < TG_S; ++sl)
            for (int b = 0; b < NBOX; ++b)
                tg_tma3(tg_smem(Asm + (sl * NBOX + b) * (TG_M * 16)), &mapA, b * 8, row0, sl, mb);
        for (int p = 0; p < P; ++p)
            for (int sl = 0; sl < TG_S; ++sl)
                for (int b = 0; b < NBOX; ++b)
                    tg_tma3(tg_smem(Bsm + ((p * TG_S + sl) * NBOX + b) * (TG_N * 16)), &mapB, b * 8, col0,
                            p * TG_S + sl, mb);
    }
    if (!tg_wait(tg_smem(&bar_ld), 0, TG_SPIN)) s_fail = 1;
    __syncthreads();
    if (s_fail && threadIdx.x == 0) tg_wait(tg_smem(&bar_ld), 0, TG_SPIN);  // copies in flight, before the CTA ends
    bool issued = false;
    if (!s_fail && threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // kind::f16: D F32, A and B BF16, both K-major, N, M = 128
        const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TG_N >> 3) << 17) |
                               ((unsigned)(TG_M >> 4) << 24);
        for (int p = 0; p < P; ++p)
            for (int L = 0; L < TG_LV; ++L)
                for (int sa = (L < TG_S ? 0 : L - TG_S + 1); sa <= L && sa < TG_S; ++sa) {
                    const int sb = L - sa;
#pragma unroll
                    for (int kk = 0; kk < KI / 16; ++kk) {
                        const unsigned long long ad =
                            tg_desc(tg_smem(Asm + (sa * NBOX + 2 * kk) * (TG_M * 16)), TG_M * 16, 128);
                        const unsigned long long bd =
                            tg_desc(tg_smem(Bsm + ((p * TG_S + sb) * NBOX + 2 * kk) * (TG_N * 16)), TG_N * 16, 128);
                        const unsigned acc = (sa > (L < TG_S ? 0 : L - TG_S + 1) || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(
                                tmem + (unsigned)((p * TG_LV + L) * TG_N)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tg_smem(&bar_mma))
                     : "memory");
        issued = true;
    }
    __syncthreads();
    if (!s_fail && !tg_wait(tg_smem(&bar_mma), 0, TG_SPIN)) s_fail = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicOr(v.err, SWR_ERR_TIMEOUT);
            if (issued) tg_wait(tg_smem(&bar_mma), 0, TG_SPIN);  // products in flight, before the memory is freed
        }
    } else {
        double* M = v.arena + s.Gm;
        const double* W = v.arena + s.work;
        const double* Pinv = W;
        const double* Rp = W + (sizeof(T) / 8) * TG_NB * TG_NB;
        const int gi = tm + warp * 32 + lane;
        const bool row_ok = gi < K;
        const int ei = row_ok ? Aexp[rowoff[sid] + gi] : 0;
        const bool ri = gi >= k0 && gi < k0 + nb;
#pragma unroll 1
        for (int c0 = 0; c0 < TG_N; c0 += 16) {
            TgLevels lv[P][16];
#pragma unroll
            for (int p = 0; p < P; ++p) {
#pragma unroll
                for (int j = 0; j < 16; ++j) lv[p][j] = TgLevels{0, 0};
#pragma unroll 1
                for (int L = 0; L < TG_LV; ++L) {
                    unsigned r[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((p * TG_LV + L) * TG_N + c0)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) tg_level_add<7, TG_LV, 5>(lv[p][j], L, __uint_as_float(r[j]));
                }
            }
            if (!row_ok) continue;
#pragma unroll 4
            for (int j = 0; j < 16; ++j) {
                const int gj = tn + c0 + j;
                if (gj >= K) continue;
                const long long idx = (long long)gi * K + gj;
                const bool cj = gj >= k0 && gj < k0 + nb;
                const int ex = ei + Bexp[coloff[sid] + gj] - 14;
                if (P == 1) {
                    if (ri) M[idx] = cj ? Pinv[(long long)(gi - k0) * TG_NB + (gj - k0)] : Rp[(long long)(gi - k0) * K + gj];
                    else if (cj) M[idx] = -tg_level_value<7, TG_LV, 5>(lv[0][j], ex);
                    else M[idx] = M[idx] - tg_level_value<7, TG_LV, 5>(lv[0][j], ex);
                } else {
                    double re, im;
                    if (ri) {
                        const double* src = cj ? Pinv + 2 * ((long long)(gi - k0) * TG_NB + (gj - k0))
                                               : Rp + 2 * ((long long)(gi - k0) * K + gj);
                        re = src[0];
                        im = src[1];
                    } else {
                        const double dr = tg_level_value<7, TG_LV, 5>(lv[0][j], ex),
                                     di = tg_level_value<7, TG_LV, 5>(lv[P - 1][j], ex);
                        re = cj ? -dr : M[2 * idx] - dr;
                        im = cj ? -di : M[2 * idx + 1] - di;
                    }
                    M[2 * idx] = re;
                    M[2 * idx + 1] = im;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// --------------------------------------------- e-e block of the assembly
//
// The sum-factorised e-e block (Sec. 5.1: the local Hamiltonian's matrix of
// the electron-electron potential, B^T diag(w V_ee) B written as two
// products, Mee = Wv P2 and V'ee = P1^T Mee scattered into H') with FP64
// emulated on the tensor cores like the Gauss-Jordan updates, but with an
// inner dimension up to 384 (the quadrature nodes of a coordinate): 6-bit
// slices (11 of them, integers in [-63, 63]) keep a level's sum exact in
// the FP32 accumulator over the whole inner dimension (11 pairs x 63^2 x 384
// < 2^24), so the level accumulators run through every inner chunk of 32
// and are combined in FP64 once:
//     C_ij = 2^(e_i + f_j - 12) sum_{L <= 10} 2^(-6 L) acc_L[i][j]
// with e_i the exponent of row i of A over the whole inner dimension and f_j
// that of column j of B; the dropped levels and the slicing remainders stay
// below 2^-66 times the inner length.  Each inner chunk's slices reach
// shared memory by tensor-map bulk copies, the 66 slice pairs of the chunk go
// to the tensor cores, and the next chunk is loaded once they completed.
#define TE_S 11          // 6-bit slices per operand
#define TE_LV 11         // levels kept: 0..10
#define TE_N 32          // columns of C per CTA
#define TE_KC 32         // inner chunk

__device__ inline void te_slice(double x, int e, __nv_bfloat16* out, long long slice_stride) {
    double r = ldexp(x, -e);
#pragma unroll
    for (int s = 0; s < TE_S; ++s) {
        r *= 64.0;
        const double a = trunc(r);
        r -= a;
        out[s * slice_stride] = __double2bfloat16(a);
    }
}

// Rows of op(A) of every job (one thread per row): A(i, k) = A[i lda + k], or
// A[k lda + i] when transposed; slices As[s][row0 + i][k] (k < KIP, zero-padded).
__global__ void k_te_slice_rows(SwrDeviceView v, const GemmJob* jobs, const long long* row0, __nv_bfloat16* As,
                                int* Aexp, long long R, int KIP) {
    const GemmJob jb = jobs[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (jb.M <= 0 || i >= jb.M) return;
    const double* A = v.arena + jb.a;
    auto el = [&](int k) { return jb.transA ? A[(long long)k * jb.lda + i] : A[(long long)i * jb.lda + k]; };
    double amax = 0.0;
    for (int k = 0; k < jb.K; ++k) amax = fmax(amax, fabs(el(k)));
    const int e = tg_exponent(amax);
    const long long row = row0[blockIdx.y] + i;
    Aexp[row] = e;
    for (int k = 0; k < KIP; ++k) te_slice(k < jb.K ? el(k) : 0.0, e, As + row * KIP + k, R * KIP);
}

// Columns of B of every job (one thread per column): B(k, j) = B[k ldb + j];
// slices Bs[s][col0 + j][k].
__global__ void k_te_slice_cols(SwrDeviceView v, const GemmJob* jobs, const long long* col0, __nv_bfloat16* Bs,
                                int* Bexp, long long C, int KIP) {
    const GemmJob jb = jobs[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (jb.M <= 0 || j >= jb.N) return;
    const double* B = v.arena + jb.b;
    double amax = 0.0;
    for (int k = 0; k < jb.K; ++k) amax = fmax(amax, fabs(B[(long long)k * jb.ldb + j]));
    const int e = tg_exponent(amax);
    const long long col = col0[blockIdx.y] + j;
    Bexp[col] = e;
    for (int k = 0; k < KIP; ++k)
        te_slice(k < jb.K ? B[(long long)k * jb.ldb + j] : 0.0, e, Bs + col * KIP + k, C * KIP);
}

// One 128 x 32 tile of C = op(A) B of job blockIdx.z.  Dynamic shared memory
// (one inner chunk): A slices [S][4 boxes][128 rows][16 B], B slices
// [S][4][32 rows][16 B].
__global__ void __launch_bounds__(TG_THREADS, 1) k_te_gemm(SwrDeviceView v, const GemmJob* jobs,
                                                           const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           const int* Aexp, const int* Bexp,
                                                           const long long* row0, const long long* col0) {
    constexpr int NBOX = TE_KC / 8;
    constexpr unsigned A_BYTES = TE_S * NBOX * TG_M * 16, B_BYTES = TE_S * NBOX * TE_N * 16;
    static_assert(TE_LV * TE_N <= TG_TMEM, "level accumulators exceed the tensor memory");
    const GemmJob jb = jobs[blockIdx.z];
    const int tm = blockIdx.y * TG_M, tn = blockIdx.x * TE_N;
    if (jb.M <= 0 || tm >= jb.M || tn >= jb.N) return;
    extern __shared__ __align__(1024) unsigned char te_sm[];
    unsigned char* Asm = te_sm;
    unsigned char* Bsm = te_sm + A_BYTES;
    __shared__ __align__(8) unsigned long long bar_ld, bar_mma;
    __shared__ unsigned tmem_slot;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tg_smem(&tmem_slot)),
                     "r"(TG_TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tg_smem(&bar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tg_smem(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    const int ra = (int)(row0[blockIdx.z] + tm), cb = (int)(col0[blockIdx.z] + tn);
    const int nch = (jb.K + TE_KC - 1) / TE_KC;
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TE_N >> 3) << 17) |
                           ((unsigned)(TG_M >> 4) << 24);
    int issued_mma = 0;
    for (int c = 0; c < nch; ++c) {
        if (threadIdx.x == 0) {
            const unsigned mb = tg_smem(&bar_ld);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(A_BYTES + B_BYTES)
                         : "memory");
            for (int sl = 0; sl < TE_S; ++sl)
                for (int b = 0; b < NBOX; ++b) {
                    tg_tma3(tg_smem(Asm + (sl * NBOX + b) * (TG_M * 16)), &mapA, c * TE_KC + b * 8, ra, sl, mb);
                    tg_tma3(tg_smem(Bsm + (sl * NBOX + b) * (TE_N * 16)), &mapB, c * TE_KC + b * 8, cb, sl, mb);
                }
        }
        if (!tg_wait(tg_smem(&bar_ld), (unsigned)(c & 1), TG_SPIN)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            if (threadIdx.x == 0) tg_wait(tg_smem(&bar_ld), (unsigned)(c & 1), TG_SPIN);  // copies in flight
            break;
        }
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int L = 0; L < TE_LV; ++L) {
                const int s0 = L < TE_S ? 0 : L - TE_S + 1;
                for (int sa = s0; sa <= L && sa < TE_S; ++sa) {
                    const int sb = L - sa;
#pragma unroll
                    for (int kk = 0; kk < TE_KC / 16; ++kk) {
                        const unsigned long long ad =
                            tg_desc(tg_smem(Asm + (sa * NBOX + 2 * kk) * (TG_M * 16)), TG_M * 16, 128);
                        const unsigned long long bd =
                            tg_desc(tg_smem(Bsm + (sb * NBOX + 2 * kk) * (TE_N * 16)), TE_N * 16, 128);
                        const unsigned acc = (c > 0 || sa > s0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(
                                tmem + (unsigned)(L * TE_N)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tg_smem(&bar_mma))
                         : "memory");
        }
        ++issued_mma;
        // the next chunk overwrites the slices: wait for this chunk's products
        if (!tg_wait(tg_smem(&bar_mma), (unsigned)(c & 1), TG_SPIN)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicOr(v.err, SWR_ERR_TIMEOUT);
            if (issued_mma > 0) tg_wait(tg_smem(&bar_mma), (unsigned)((issued_mma - 1) & 1), TG_SPIN);
        }
    } else {
        double* Cm = v.arena + jb.c;
        const int gm = tm + warp * 32 + lane;
        const bool row_ok = gm < jb.M;
        const int ei = row_ok ? Aexp[row0[blockIdx.z] + gm] : 0;
#pragma unroll 1
        for (int c0 = 0; c0 < TE_N; c0 += 16) {
            TgLevels lv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) lv[j] = TgLevels{0, 0};
#pragma unroll 1
            for (int L = 0; L < TE_LV; ++L) {
                unsigned r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(L * TE_N + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) tg_level_add<6, TE_LV, 6>(lv[j], L, __uint_as_float(r[j]));
            }
            if (!row_ok) continue;
#pragma unroll 4
            for (int j = 0; j < 16; ++j) {
                const int gn = tn + c0 + j;
                if (gn >= jb.N) continue;
                const double val = tg_level_value<6, TE_LV, 6>(lv[j], ei + Bexp[col0[blockIdx.z] + gn] - 12);
                if (jb.mode == 0) {
                    Cm[(long long)gm * jb.ldc + gn] = val;
                } else {
                    // gm = (a, c), gn = (b, e): H'[(a + kd b), (c + kd e)]
                    const int kd = jb.kd;
                    const int a = gm / kd, cc = gm % kd, b = gn / kd, e = gn % kd;
                    Cm[(long long)(a + kd * b) * ((long long)kd * kd) + (cc + kd * e)] = val;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM));
}

// ------------------------------------------------------------- host side

// Tensor-core Gauss-Jordan state of a context: the slice arrays (device
// memory carved by the caller), per-subdomain row offsets, and the tensor maps.
struct TgState {
    __nv_bfloat16 *As = nullptr, *Bs = nullptr;
    int *Aexp = nullptr, *Bexp = nullptr;
    long long* d_off = nullptr;  // [n_sub] row (= column) offset of each subdomain
    long long R = 0;             // rows (= columns) of all subdomains
    bool cplx_data = false;
    CUtensorMap mapA, mapB;
    // e-e block: slices of op(A) rows and B columns of both products
    bool ee = false;
    __nv_bfloat16 *Ae = nullptr, *Be = nullptr;
    int *Aeexp = nullptr, *Beexp = nullptr;
    long long *d_row0 = nullptr, *d_col0 = nullptr;
    long long Re = 0, Ce = 0;
    int KIP = 0, max_rows = 0, max_cols = 0;
    CUtensorMap mapAe, mapBe;
};

static size_t al256b(size_t x) { return (x + 255) & ~(size_t)255; }

// Sizes of the e-e slice arrays: rows max(q, kd^2) and columns kd^2 per
// two-electron subdomain, inner dimension q padded to 32.
static void te_sizes(const int* qs, const int* kds, const int* nel, int n_sub, long long* R, long long* C, int* KIP) {
    *R = 0;
    *C = 0;
    int qmax = 0;
    for (int i = 0; i < n_sub; ++i) {
        if (nel[i] != 2) continue;
        const long long k2 = (long long)kds[i] * kds[i];
        *R += qs[i] > k2 ? qs[i] : k2;
        *C += k2;
        qmax = qs[i] > qmax ? qs[i] : qmax;
    }
    *KIP = ((qmax + TE_KC - 1) / TE_KC) * TE_KC;
}

// Bytes of device scratch the tensor-core path needs for subdomains of the
// given sizes (slices of both operands of the Gauss-Jordan updates and of the
// e-e products, exponents, offsets).
size_t tg_scratch_bytes(const int* Ks, const int* qs, const int* kds, const int* nel, int n_sub, bool cplx_data,
                        bool any_ee) {
    long long R = 0;
    for (int i = 0; i < n_sub; ++i) R += Ks[i];
    const int KI = cplx_data ? 64 : 32, P = cplx_data ? 2 : 1;
    const size_t a = (size_t)TG_S * R * KI * 2, b = (size_t)P * TG_S * R * KI * 2;
    size_t tot = al256b(a) + al256b(b) + 2 * al256b((size_t)R * 4) + al256b((size_t)n_sub * 8);
    if (any_ee) {
        long long Re, Ce;
        int KIP;
        te_sizes(qs, kds, nel, n_sub, &Re, &Ce, &KIP);
        tot += al256b((size_t)TE_S * Re * KIP * 2) + al256b((size_t)TE_S * Ce * KIP * 2) + al256b((size_t)Re * 4) +
               al256b((size_t)Ce * 4) + 2 * al256b((size_t)n_sub * 8);
    }
    return tot;
}

typedef CUresult (*PFN_encode_tiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t tg_encode(CUtensorMap* map, void* base, long long rows, int KI, int planes, int box_rows) {
    if (rows < 1) rows = 1;
    static PFN_encode_tiled enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) return e != cudaSuccess ? e : cudaErrorUnknown;
        enc = (PFN_encode_tiled)f;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)KI, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)KI * 2, (cuuint64_t)rows * KI * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Lays out the scratch at `base` (tg_scratch_bytes), uploads the offsets and
// encodes the tensor maps.
cudaError_t tg_setup(TgState** out, void* base, const int* Ks, const int* qs, const int* kds, const int* nel, int n_sub,
                     bool cplx_data, bool any_ee, cudaStream_t st) {
    TgState* g = new TgState();
    g->cplx_data = cplx_data;
    std::vector<long long> off(n_sub);
    long long R = 0;
    for (int i = 0; i < n_sub; ++i) {
        off[i] = R;
        R += Ks[i];
    }
    g->R = R;
    const int KI = cplx_data ? 64 : 32, P = cplx_data ? 2 : 1;
    char* p = (char*)base;
    const size_t a = (size_t)TG_S * R * KI * 2, b = (size_t)P * TG_S * R * KI * 2;
    g->As = (__nv_bfloat16*)p;
    p += (a + 255) & ~(size_t)255;
    g->Bs = (__nv_bfloat16*)p;
    p += (b + 255) & ~(size_t)255;
    g->Aexp = (int*)p;
    p += ((size_t)R * 4 + 255) & ~(size_t)255;
    g->Bexp = (int*)p;
    p += ((size_t)R * 4 + 255) & ~(size_t)255;
    g->d_off = (long long*)p;
    p += al256b((size_t)n_sub * 8);
    cudaError_t e = cudaMemcpyAsync(g->d_off, off.data(), n_sub * sizeof(long long), cudaMemcpyHostToDevice, st);
    std::vector<long long> r0(n_sub, 0), c0(n_sub, 0);
    if (any_ee) {
        g->ee = true;
        te_sizes(qs, kds, nel, n_sub, &g->Re, &g->Ce, &g->KIP);
        long long ro = 0, co = 0;
        for (int i = 0; i < n_sub; ++i) {
            r0[i] = ro;
            c0[i] = co;
            if (nel[i] != 2) continue;
            const long long k2 = (long long)kds[i] * kds[i];
            ro += qs[i] > k2 ? qs[i] : k2;
            co += k2;
            g->max_rows = (int)(qs[i] > k2 ? qs[i] : k2) > g->max_rows ? (int)(qs[i] > k2 ? qs[i] : k2) : g->max_rows;
            g->max_cols = (int)k2 > g->max_cols ? (int)k2 : g->max_cols;
        }
        g->Ae = (__nv_bfloat16*)p;
        p += al256b((size_t)TE_S * g->Re * g->KIP * 2);
        g->Be = (__nv_bfloat16*)p;
        p += al256b((size_t)TE_S * g->Ce * g->KIP * 2);
        g->Aeexp = (int*)p;
        p += al256b((size_t)g->Re * 4);
        g->Beexp = (int*)p;
        p += al256b((size_t)g->Ce * 4);
        g->d_row0 = (long long*)p;
        p += al256b((size_t)n_sub * 8);
        g->d_col0 = (long long*)p;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->d_row0, r0.data(), n_sub * sizeof(long long), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->d_col0, c0.data(), n_sub * sizeof(long long), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e == cudaSuccess && g->ee) e = tg_encode(&g->mapAe, g->Ae, g->Re, g->KIP, TE_S, TG_M);
    if (e == cudaSuccess && g->ee) e = tg_encode(&g->mapBe, g->Be, g->Ce, g->KIP, TE_S, TE_N);
    if (e == cudaSuccess) e = tg_encode(&g->mapA, g->As, R, KI, TG_S, TG_M);
    if (e == cudaSuccess) e = tg_encode(&g->mapB, g->Bs, R, KI, P * TG_S, cplx_data ? TgN<cplx>::v : TgN<double>::v);
    if (e != cudaSuccess) {
        delete g;
        return e;
    }
    *out = g;
    return cudaSuccess;
}

void tg_release(TgState* g) { delete g; }

bool tg_has_ee(const TgState* g) { return g && g->ee; }

// The two e-e products of every two-electron subdomain (jobs of k_dgemm's
// form): slices of op(A) rows and B columns, then the tensor-core product.
cudaError_t te_products(const TgState* g, const SwrDeviceView& v, cudaStream_t st, const GemmJob* d_jobs1,
                        const GemmJob* d_jobs2) {
    constexpr unsigned SM0 = TE_S * (TE_KC / 8) * TG_M * 16 + TE_S * (TE_KC / 8) * TE_N * 16;
    constexpr unsigned SM = SM0 > 120 * 1024 ? SM0 : 120 * 1024;  // one CTA per SM: it takes all tensor memory
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_te_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
        attr = true;
    }
    const int rows = g->max_rows, cols = g->max_cols;
    for (int jn = 0; jn < 2; ++jn) {
        const GemmJob* jobs = jn == 0 ? d_jobs1 : d_jobs2;
        k_te_slice_rows<<<dim3((rows + 127) / 128, v.n_sub), 128, 0, st>>>(v, jobs, g->d_row0, g->Ae, g->Aeexp, g->Re,
                                                                           g->KIP);
        k_te_slice_cols<<<dim3((cols + 127) / 128, v.n_sub), 128, 0, st>>>(v, jobs, g->d_col0, g->Be, g->Beexp, g->Ce,
                                                                           g->KIP);
        k_te_gemm<<<dim3((cols + TE_N - 1) / TE_N, (rows + TG_M - 1) / TG_M, v.n_sub), TG_THREADS, SM, st>>>(
            v, jobs, g->mapAe, g->mapBe, g->Aeexp, g->Beexp, g->d_row0, g->d_col0);
    }
    return cudaGetLastError();
}

static inline unsigned tg_div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Slices and tensor-core update of block column kb for every subdomain.
cudaError_t tg_update(const TgState* g, const SwrDeviceView& v, cudaStream_t st, int kb, int max_K) {
    const dim3 gs(tg_div_up(max_K, 128), v.n_sub);
    if (g->cplx_data) {
        constexpr int TN = TgN<cplx>::v;
        const dim3 gu(tg_div_up(max_K, TN), tg_div_up(max_K, TG_M), v.n_sub);
        constexpr unsigned SM = TG_S * 8 * TG_M * 16 + 2 * TG_S * 8 * TN * 16;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_tg_update<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
            attr = true;
        }
        k_tg_slice_a<cplx><<<gs, 128, 0, st>>>(v, kb, g->As, g->Aexp, g->d_off, g->R);
        k_tg_slice_b<cplx><<<gs, 128, 0, st>>>(v, kb, g->Bs, g->Bexp, g->d_off, g->R);
        k_tg_update<cplx><<<gu, TG_THREADS, SM, st>>>(v, kb, g->mapA, g->mapB, g->Aexp, g->Bexp, g->d_off, g->d_off);
    } else {
        constexpr int TN = TgN<double>::v;
        const dim3 gu(tg_div_up(max_K, TN), tg_div_up(max_K, TG_M), v.n_sub);
        // the CTA takes all 512 tensor-memory columns: request more than half of
        // the SM's shared memory so that a second CTA never waits in its allocation
        constexpr unsigned SM0 = TG_S * 4 * TG_M * 16 + TG_S * 4 * TN * 16;
        constexpr unsigned SM = SM0 > 120 * 1024 ? SM0 : 120 * 1024;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_tg_update<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
            attr = true;
        }
        k_tg_slice_a<double><<<gs, 128, 0, st>>>(v, kb, g->As, g->Aexp, g->d_off, g->R);
        k_tg_slice_b<double><<<gs, 128, 0, st>>>(v, kb, g->Bs, g->Bexp, g->d_off, g->R);
        k_tg_update<double><<<gu, TG_THREADS, SM, st>>>(v, kb, g->mapA, g->mapB, g->Aexp, g->Bexp, g->d_off, g->d_off);
    }
    return cudaGetLastError();
}

}  // namespace swr
