// swr_cluster.cu -- the imaginary-time window on thread-block clusters, with
// the step matrices held on chip for the whole window.
//
// The recursion of the other window kernels (Sec. 5.2, system SIT; Sec. 5.4
// steps 2 and 4):
//     y^{n+1} = G (y^n / s_n + kappa dt b'^{n+1}),   s_n^2 = sum_i y_i^n . (Pp (x) Pp) y_i^n,
// stop when ||c^n - c^{n-1}|| <= tol with c^n = y^n / s_n.
//
// One cluster of CS CTAs (one CTA per SM) per subdomain: CTA j of the cluster
// owns the j-th block of rows of the subdomain's G.  Those rows never leave
// the SM: the FP32 hi plane sits in shared memory, the lo plane in tensor
// memory (written once with tcgen05.st, read back every step with tcgen05.ld),
// so a step reads no step-matrix bytes from L2 or HBM.  Per step n:
//   1. y^n is complete in every CTA of the cluster (double-single pairs, stored
//      there through distributed shared memory by the owners of its rows
//      before the cluster barrier that ended step n-1);
//   2. own rows of z^n = (Pp (x) Pp) y^n (double-single Kronecker products) and
//      the partial of s_n^2; it is published together with the partial of
//      D_{n-1} = ||c^{n-1} - c^{n-2}||^2 computed at step n-1, and the
//      instance's arrival counter is incremented (release);
//   3. while the counter fills: own rows of u = G y^n (the product does not
//      wait for s_n: y^{n+1} = G (y^n / s_n + kappa dt b'^{n+1})
//      = u / s_n + w^{n+1}, with w^{n+1} = kappa dt G b'^{n+1} formed for every
//      step before the window, swr_robin.cu);
//   4. the instance sums (same order, same bits in every CTA) and the
//      decisions of the other window kernels: stop at n-1 on D_{n-1} <= tol^2,
//      at n on the cap or a non-positive s_n;
//   5. own rows of y^{n+1} = u / s_n + w^{n+1} in double-single into every CTA
//      of the cluster (the history row and the partial of D_n follow from
//      them at step n+1);
//   6. cluster barrier.
// There is no grid barrier: the clusters of one instance meet only at its
// counter, those of different instances never wait on each other.  Every
// counter wait is bounded; a CTA that gives up raises SWR_ERR_TIMEOUT and
// writes a stop flag into every CTA of its cluster before the cluster
// barrier, so the cluster always leaves together after the same barrier and
// no remote store can target a CTA that has exited.
#include <math.h>

#include "swr_internal.cuh"

namespace swr {

#define CL_THREADS 512
#define CL_WARPS (CL_THREADS / 32)
#define CL_SMEM_MIN (120 * 1024)  // at least this much shared memory: one CTA per SM
#define CL_POLL 5                  // slots polled per lane: instances of at most 160 CTAs
#define CL_SMEM_MAX (226 * 1024)  // dynamic shared memory budget per CTA

__device__ inline unsigned cl_smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline unsigned cl_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ inline unsigned cl_nctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Cluster-wide barrier: shared-memory stores of every CTA (local and remote)
// before it are visible to every CTA after it.
__device__ inline void cl_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Stores into CTA `rank` of the cluster at the address of `local` in this CTA.
__device__ inline unsigned cl_map(const void* local, unsigned rank) {
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(cl_smem_u32(local)), "r"(rank));
    return ra;
}
__device__ inline void cl_store2(const void* local, unsigned rank, float h, float l) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(cl_map(local, rank)), "f"(h), "f"(l) : "memory");
}
__device__ inline void cl_store_int(const void* local, unsigned rank, int x) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cl_map(local, rank)), "r"(x) : "memory");
}
__device__ inline unsigned cl_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void cl_red_release(unsigned* p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// Matrix-vector layout of one CTA: warp w owns the column segment
// [w sw, (w+1) sw) of its rows, lane l the rows l + 32 k (k < rpl), so a thread
// holds rpl x sw elements (index e = k sw + j); sw is a multiple of 4 with
// 16 sw >= ld.  The G_hi values of elements e < hs sit in shared memory
// ([w][e/4][l][e%4], 16-byte loads without bank conflicts), the rest and every
// G_lo value in tensor memory (lane 32 (w mod 4) + l).
__host__ __device__ inline int cluster_sw(int K) { return 4 * ((df32_ld(K) + 63) / 64); }
__host__ __device__ inline int cluster_rpl(int rows) { return (rows + 31) / 32; }

// Shared memory of one CTA (bytes) before the G_hi elements: y^n double
// buffer | P1, P2 | Kronecker scratch | own rows of y and z (3 steps each)
// | own rows of w^{n+1} | segment partials [rpl][16][32] (double-single pairs).
__host__ __device__ inline int cluster_vlen(int kmax) { return 16 * cluster_sw(kmax); }
__host__ __device__ inline size_t cluster_smem_vectors(int kmax, int kdmax, int rows_max) {
    const size_t ld = (size_t)cluster_vlen(kmax);  // y and v padded to 16 segments, zero past K
    return (2 * ld + 2 * (size_t)kdmax * kdmax + (size_t)rows_max + 2 * (size_t)kdmax + 7 * (size_t)rows_max +
            (size_t)cluster_rpl(rows_max) * CL_THREADS) *
           sizeof(float2);
}
__host__ __device__ inline size_t cluster_smem_bytes(int kmax, int kdmax, int rows_max, int hs) {
    return (size_t)hs * CL_THREADS * sizeof(float) + cluster_smem_vectors(kmax, kdmax, rows_max);
}

__device__ inline void cl_st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline void cl_ld2_relaxed(const unsigned long long* p, unsigned long long& a, unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
// A float carried in the low half of a word whose high half is the step tag.
__device__ inline unsigned long long cl_tagged(float x, unsigned tag) {
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(x);
}
__device__ inline float cl_untag(unsigned long long w) { return __uint_as_float((unsigned)(w & 0xffffffffULL)); }

// Tensor-memory store of one column and load of four, lane quarter q.
__device__ inline void cl_tst1(unsigned tmem, unsigned q, int col, float a) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(tmem + ((q * 32u) << 16) + (unsigned)col),
                 "r"(__float_as_uint(a)));
}
__device__ inline void cl_tld4(unsigned tmem, unsigned q, int col, unsigned (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(tmem + ((q * 32u) << 16) + (unsigned)col));
}

// 1/sqrt(a) in double-single: FP32 estimate and two Newton steps
// y <- y + y (1 - a y^2) / 2 in double-single arithmetic (~2^-46 relative).
__device__ inline float2 cl_rsqrt(float2 a) {
    float2 y = make_float2(rsqrtf(a.x), 0.f);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const float2 r = dsp_add(make_float2(1.f, 0.f), dsp_neg(dsp_mul(a, dsp_mul(y, y))));
        y = dsp_add(y, dsp_mul(y, make_float2(0.5f * r.x, 0.5f * r.y)));
    }
    return y;
}

template <int RPL, bool ONEP>
__global__ void __launch_bounds__(CL_THREADS, 1) k_window_cluster(SweepArgs A) {
    extern __shared__ __align__(16) unsigned char cl_sm[];
    __shared__ float2 red2[CL_WARPS];
    __shared__ float2 s_poll[CL_POLL][32][2];  // polled partials (s^2, D) per lane and slot
    __shared__ float2 s_is[2];    // 1/s_n, 1/s_{n-1} (after the decisions of step n)
    __shared__ float2 s_dpart;    // partial of D_{n-1} from this CTA's rows
    __shared__ float2 s_sn;       // s_n
    __shared__ unsigned tmem_slot;
    __shared__ int s_stop, s_fail, s_leave, s_wend;
    // set (also by the peers) when the cluster leaves after the barrier of step
    // n, by step parity: a peer already in step n+1 writes the other entry
    __shared__ int cl_flag[2];
    const SwrDeviceView& v = A.v;
    const int t = blockIdx.x;  // one row task per CTA, the tasks of a subdomain in one cluster
    const TaskCache tc = make_task_cache(A, t);
    const unsigned CS = cl_nctarank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = tc.K, kd = tc.kd, nr = tc.nr, r0 = tc.r0;
    const int ld = df32_ld(K), sw = cluster_sw(K), rpl = cluster_rpl(nr), ne = rpl * sw;
    const int hsm = A.cl_hs;                      // G_hi elements per thread in shared memory (all CTAs)
    const int hs = ne < hsm ? ne : hsm;           // this CTA's (a multiple of 4)
    const int ht = ne - hs;                       // G_hi elements per thread in tensor memory
    const int ldm = cluster_vlen(A.kmax), kdm = A.kdmax, nrm = A.rows_max;
    float* Gsm = (float*)cl_sm;                           // [16][hsm/4][32][4]
    float2* ybuf = (float2*)(Gsm + (size_t)hsm * CL_THREADS);  // [2][ldm]
    float2* P1 = ybuf + 2 * ldm;
    float2* P2 = P1 + kdm * kdm;
    float2* tmp = P2 + kdm * kdm;        // [nrm + 2 kdm]
    float2* yown = tmp + nrm + 2 * kdm;  // [3][nrm]
    float2* zown = yown + 3 * nrm;       // [3][nrm]
    float2* wown = zown + 3 * nrm;       // [nrm] own rows of w^{n+1}
    float2* segp = wown + nrm;           // [rpl][16][32] segment partials
    const unsigned q = (unsigned)warp & 3u;  // tensor-memory lane quarter of this warp
    const float* Ghg = (const float*)(v.arena + tc.Gf);
    const float* Glg = Ghg + (size_t)K * ld;
    const int t0 = A.inst_task0[tc.inst], t1 = A.inst_task0[tc.inst + 1];
    const bool stop_rule = tc.ngf_stop != 0;
    const float2 tol2 = ds_split(tc.ngf_tol * tc.ngf_tol);

    // ----------------------------------------------------------------- set-up
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cl_smem_u32(&tmem_slot)),
                     "r"(A.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_stop = 0;
        s_fail = 0;
        s_leave = 0;
        cl_flag[0] = cl_flag[1] = 0;
        s_dpart = make_float2(0.f, 0.f);
        s_is[0] = s_is[1] = make_float2(1.f, 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // this thread's elements: rows l + 32 k, columns w sw + j; G_hi of e < hs to
    // shared memory, the rest to tensor memory at [4 ne + (w/4) ht, ...), G_lo
    // to tensor memory at [(w/4) ne, ...); zero outside the matrix
    {
        const int cb = warp * sw, tlo = (warp >> 2) * ne, thi = 4 * ne + (warp >> 2) * ht;
        for (int e = 0; e < ne; ++e) {
            const int k = e / sw, j = e - k * sw, i = lane + 32 * k, c = cb + j;
            const bool in = i < nr && c < ld;
            const float gh = in ? Ghg[(size_t)(r0 + i) * ld + c] : 0.f;
            const float gl = in ? Glg[(size_t)(r0 + i) * ld + c] : 0.f;
            if (e < hs) Gsm[(((size_t)warp * (hsm >> 2) + (e >> 2)) * 32 + lane) * 4 + (e & 3)] = gh;
            else cl_tst1(tmem, q, thi + (e - hs), gh);
            if (!ONEP) cl_tst1(tmem, q, tlo + e, gl);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    // Kronecker factors, y^0 = c0 (double-single), history row 0, zero padding
    {
        const double* P1g = v.arena + tc.p1;
        const double* P2g = v.arena + tc.p2;
        for (int e = tid; e < kd * kd; e += CL_THREADS) {
            P1[e] = ds_split(P1g[e]);
            P2[e] = ds_split(P2g[e]);
        }
        const double* c0 = v.arena + tc.c0;
        double* h0 = v.arena + tc.hist;
        for (int c = tid; c < ldm; c += CL_THREADS) {
            ybuf[c] = c < K ? ds_split(c0[c]) : make_float2(0.f, 0.f);
            ybuf[ldm + c] = make_float2(0.f, 0.f);
        }
        for (int i = tid; i < nr; i += CL_THREADS) h0[r0 + i] = c0[r0 + i];
    }
    const int wp = A.win_prev[tc.inst];
    // w^n = kappa dt G b'^n of the previous iteration's Robin data, rows of ldw
    const float2* Wg = reinterpret_cast<const float2*>(v.arena + v.sub[tc.sid].Wr);
    const int ldw = df32_ld(K);
    const int wi = tid - 32;  // threads 32.. carry the own rows of w^{n+1} through the step
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    cl_sync();  // every CTA of the cluster initialised before the first remote store
    asm volatile("tcgen05.fence::after_thread_sync;");

    for (int n = 0;; ++n) {
        const float2* yn = ybuf + (size_t)(n & 1) * ldm;
        float2* yo_n = yown + (size_t)(n % 3) * nrm;
        float2* zo_n = zown + (size_t)(n % 3) * nrm;
        // own row of w^{n+1} (held beyond the previous window at its last step),
        // loaded now and used after the product
        float2 wreg = make_float2(0.f, 0.f);
        if (wp > 0 && wi >= 0 && wi < nr) {
            const unsigned long long u =
                __ldcg(reinterpret_cast<const unsigned long long*>(Wg + (long long)min(n + 1, wp) * ldw + r0 + wi));
            wreg = make_float2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
        }
        // ---- phase A: own rows of y^n and z^n = (Pp (x) Pp) y^n (double-single,
        //      warps 0..14: tmp[bb][c] = sum_e Y[c][e] P2[b0+bb][e] with 4 threads
        //      per entry, z[(a, b)] = sum_c P1[a][c] tmp[b-b0][c] with 8 per row);
        //      warp 15: the partial of D_{n-1} from the own rows of steps n-1, n-2
        if (warp < CL_WARPS - 1) {
            const int ta = tid, na = CL_THREADS - 32;
            for (int i = ta; i < nr; i += na) yo_n[i] = yn[r0 + i];
            if (tc.N == 2) {
                const int b0 = r0 / kd, nb = (r0 + nr - 1) / kd - b0 + 1, items = nb * kd;
                for (int base = 0; base < items; base += na / 4) {
                    const int it = base + (ta >> 2), g = ta & 3;
                    float2 acc = make_float2(0.f, 0.f);
                    if (it < items) {
                        const int bb = it / kd, c = it - bb * kd;
                        const float2* p2 = P2 + (b0 + bb) * kd;
                        for (int e = g; e < kd; e += 4) ds_fma(acc.x, acc.y, yn[c + kd * e], p2[e]);
                    }
                    acc = dsp_shfl_add(acc, 1);
                    acc = dsp_shfl_add(acc, 2);
                    if (it < items && g == 0) tmp[it] = acc;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(CL_THREADS - 32) : "memory");
                for (int base = 0; base < nr; base += na / 8) {
                    const int i = base + (ta >> 3), g = ta & 7;
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
                    if (i < nr && g == 0) zo_n[i] = acc;
                }
            } else {
                for (int base = 0; base < nr; base += na / 8) {
                    const int i = base + (ta >> 3), g = ta & 7;
                    float2 acc = make_float2(0.f, 0.f);
                    if (i < nr) {
                        const float2* p1 = P1 + (r0 + i) * kd;
                        for (int c = g; c < kd; c += 8) ds_fma(acc.x, acc.y, p1[c], yn[c]);
                    }
                    acc = dsp_shfl_add(acc, 1);
                    acc = dsp_shfl_add(acc, 2);
                    acc = dsp_shfl_add(acc, 4);
                    if (i < nr && g == 0) zo_n[i] = acc;
                }
            }
        } else if (n >= 2 && stop_rule) {
            // D_{n-1} = ||y^{n-1}/s_{n-1} - y^{n-2}/s_{n-2}||^2 over the own rows, with
            // y1 is1 - y2 is2 = is1 (y1 - y2) + y2 (is1 - is2): the differences of
            // nearby iterates are formed before any rounding of the products
            const float2 is1 = s_is[0], is2 = s_is[1];
            const float2 dis = dsp_add(is1, dsp_neg(is2));
            const float2* y1 = yown + (size_t)((n + 2) % 3) * nrm;
            const float2* y2 = yown + (size_t)((n + 1) % 3) * nrm;
            const float2* z1 = zown + (size_t)((n + 2) % 3) * nrm;
            const float2* z2 = zown + (size_t)((n + 1) % 3) * nrm;
            float2 acc = make_float2(0.f, 0.f);
            for (int i = lane; i < nr; i += 32) {
                const float2 d = dsp_add(dsp_mul(is1, dsp_add(y1[i], dsp_neg(y2[i]))), dsp_mul(y2[i], dis));
                const float2 e = dsp_add(dsp_mul(is1, dsp_add(z1[i], dsp_neg(z2[i]))), dsp_mul(z2[i], dis));
                acc = dsp_add(acc, dsp_mul(d, e));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = dsp_shfl_add(acc, o);
            if (lane == 0) s_dpart = acc;
        }
        __syncthreads();
        // ---- partial of s_n^2 (own rows), published with the partial of D_{n-1}
        {
            float2 acc = make_float2(0.f, 0.f);
            for (int i = tid; i < nr; i += CL_THREADS) acc = dsp_add(acc, dsp_mul(yo_n[i], zo_n[i]));
            if (tid < ((nr + 31) & ~31)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc = dsp_shfl_add(acc, o);
                if (lane == 0) red2[warp] = acc;
            }
        }
        __syncthreads();
        const unsigned tag = (unsigned)(n + 1);
        unsigned long long* slots = A.cl_slots + (size_t)(n & 1) * A.n_tasks * 4;
        const bool dprev = n >= 2 && stop_rule;
        if (tid == 0) {
            float2 a = make_float2(0.f, 0.f);
            for (int w = 0; w < (nr + 31) / 32 && w < CL_WARPS; ++w) a = dsp_add(a, red2[w]);
            const float2 d = dprev ? s_dpart : make_float2(0.f, 0.f);
            unsigned long long* my = slots + (size_t)t * 4;
            cl_st_relaxed(my + 0, cl_tagged(a.x, tag));
            cl_st_relaxed(my + 1, cl_tagged(a.y, tag));
            cl_st_relaxed(my + 2, cl_tagged(d.x, tag));
            cl_st_relaxed(my + 3, cl_tagged(d.y, tag));
        }
        // ---- own rows of u = G y^n (s_n is not needed yet): each thread its
        //      rpl rows over its warp's column segment (y^n broadcast from
        //      shared memory), chunks of 4 columns, the next chunk's
        //      tensor-memory loads in flight while the current one is used
        {
            const int cb = warp * sw, tlo = (warp >> 2) * ne, thi = 4 * ne + (warp >> 2) * ht;
            float ah[RPL], al[RPL];
#pragma unroll
            for (int k = 0; k < RPL; ++k) ah[k] = al[k] = 0.f;
            // two statically named register buffers (a runtime buffer index
            // would put them in local memory)
            unsigned loA[RPL][4], thA[RPL][4], loB[RPL][4], thB[RPL][4];
            auto issue = [&](int j0, unsigned (&lo)[RPL][4], unsigned (&th)[RPL][4]) {
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    if (k < rpl) {
                        const int e = k * sw + j0;
                        if (!ONEP) cl_tld4(tmem, q, tlo + e, lo[k]);
                        if (e >= hs) cl_tld4(tmem, q, thi + (e - hs), th[k]);
                    }
                }
            };
            // a second accumulator set for the odd chunks: two independent
            // chains per row
            float bh[RPL], bl[RPL];
#pragma unroll
            for (int k = 0; k < RPL; ++k) bh[k] = bl[k] = 0.f;
            auto use = [&](int j0, const unsigned (&lo)[RPL][4], const unsigned (&th)[RPL][4], float (&ah)[RPL],
                           float (&al)[RPL]) {
                const float4 va = *reinterpret_cast<const float4*>(yn + cb + j0);
                const float4 vb = *reinterpret_cast<const float4*>(yn + cb + j0 + 2);
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    if (k < rpl) {
                        const int e = k * sw + j0;
                        float4 g;
                        if (e < hs)
                            g = *reinterpret_cast<const float4*>(
                                Gsm + (((size_t)warp * (hsm >> 2) + (e >> 2)) * 32 + lane) * 4);
                        else
                            g = make_float4(__uint_as_float(th[k][0]), __uint_as_float(th[k][1]),
                                            __uint_as_float(th[k][2]), __uint_as_float(th[k][3]));
                        const float l0 = ONEP ? 0.f : __uint_as_float(lo[k][0]);
                        const float l1 = ONEP ? 0.f : __uint_as_float(lo[k][1]);
                        const float l2 = ONEP ? 0.f : __uint_as_float(lo[k][2]);
                        const float l3 = ONEP ? 0.f : __uint_as_float(lo[k][3]);
                        ds_fma(ah[k], al[k], make_float2(g.x, l0), make_float2(va.x, va.y));
                        ds_fma(ah[k], al[k], make_float2(g.y, l1), make_float2(va.z, va.w));
                        ds_fma(ah[k], al[k], make_float2(g.z, l2), make_float2(vb.x, vb.y));
                        ds_fma(ah[k], al[k], make_float2(g.w, l3), make_float2(vb.z, vb.w));
                    }
                }
            };
            issue(0, loA, thA);
            for (int j0 = 0; j0 < sw; j0 += 8) {
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (j0 + 4 < sw) issue(j0 + 4, loB, thB);
                use(j0, loA, thA, ah, al);
                if (j0 + 4 < sw) {
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (j0 + 8 < sw) issue(j0 + 8, loA, thA);
                    use(j0 + 4, loB, thB, bh, bl);
                }
            }
#pragma unroll
            for (int k = 0; k < RPL; ++k)
                if (k < rpl)
                    segp[((size_t)k * CL_WARPS + warp) * 32 + lane] =
                        dsp_add(make_float2(ah[k], al[k]), make_float2(bh[k], bl[k]));
        }
        if (wi >= 0 && wi < nr) wown[wi] = wreg;
        __syncthreads();
        if (warp == 0) {
            // ---- the instance's partials: every word tagged with this step (bounded
            //      polls per slot), summed in slot order, the same bits in every CTA
            float2 ss = make_float2(0.f, 0.f), sd = make_float2(0.f, 0.f);
            bool ok = true;
            // lane l owns the slots t0 + l + 32 u (u < CL_POLL); each round issues the
            // loads of all its slots still missing (in groups of three), so the wait
            // after the last arrival is one L2 round trip, not one per slot
            unsigned todo = 0;
#pragma unroll
            for (int u = 0; u < CL_POLL; ++u) {
                s_poll[u][lane][0] = s_poll[u][lane][1] = make_float2(0.f, 0.f);
                if (t0 + lane + 32 * u < t1) todo |= 1u << u;
            }
            long long it = 0;
            while (todo && ok) {
                // loads in flight together for groups of at most 3 slots (registers)
#pragma unroll
                for (int g0 = 0; g0 < CL_POLL; g0 += 3) {
                    unsigned long long w[3][4];
#pragma unroll
                    for (int du = 0; du < 3; ++du) {
                        const int u = g0 + du;
                        if (u < CL_POLL && (todo & (1u << u))) {
                            const unsigned long long* wp_ = slots + (size_t)(t0 + lane + 32 * u) * 4;
                            cl_ld2_relaxed(wp_, w[du][0], w[du][1]);
                            cl_ld2_relaxed(wp_ + 2, w[du][2], w[du][3]);
                        }
                    }
#pragma unroll
                    for (int du = 0; du < 3; ++du) {
                        const int u = g0 + du;
                        if (u < CL_POLL && (todo & (1u << u)) && (unsigned)(w[du][0] >> 32) == tag &&
                            (unsigned)(w[du][1] >> 32) == tag && (unsigned)(w[du][2] >> 32) == tag &&
                            (unsigned)(w[du][3] >> 32) == tag) {
                            s_poll[u][lane][0] = make_float2(cl_untag(w[du][0]), cl_untag(w[du][1]));
                            s_poll[u][lane][1] = make_float2(cl_untag(w[du][2]), cl_untag(w[du][3]));
                            todo &= ~(1u << u);
                        }
                    }
                }
                if (todo) {
                    if (++it > A.spin_limit) {
                        atomicOr(v.err, SWR_ERR_TIMEOUT);
                        ok = false;
                    } else if ((it & 255) == 0 && *(volatile int*)v.err) {
                        ok = false;
                    }
                }
            }
            // slot order: lane-strided partial sums, combined below in lane order
#pragma unroll
            for (int u = 0; u < CL_POLL; ++u) {
                ss = dsp_add(ss, s_poll[u][lane][0]);
                sd = dsp_add(sd, s_poll[u][lane][1]);
            }
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) s_fail = 1;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ss = dsp_shfl_add(ss, o);
                sd = dsp_shfl_add(sd, o);
            }
            if (lane == 0) {
                // ---- decisions of step n (those of the other window kernels)
                int stop = s_fail;
                if (!stop) {
                    const float2 isn = tc.normalize ? cl_rsqrt(ss) : make_float2(1.f, 0.f);
                    const float2 sn = tc.normalize ? dsp_mul(ss, isn) : make_float2(1.f, 0.f);
                    const bool bad = !(isfinite(sn.x) && sn.x > 0.f);
                    if (dprev && sd.x + sd.y <= tol2.x + tol2.y) {
                        stop = 1;  // window ends at n - 1
                        s_wend = n - 1;
                    } else if (n >= tc.maxs || bad) {
                        stop = 1;  // window ends at n
                        s_wend = n;
                    }
                    s_sn = sn;
                    s_is[1] = s_is[0];
                    s_is[0] = isn;
                }
                s_stop = stop;
            }
        } else if (n >= 1) {
            // ---- meanwhile: history row n
            double* hrow = v.arena + tc.hist + (long long)n * K;
            for (int i = tid - 32; i < nr; i += CL_THREADS - 32) hrow[r0 + i] = dsp_to_double(yo_n[i]);
        }
        __syncthreads();
        if (!s_stop) {
            if (tc.first && tid == CL_THREADS - 1) A.snorm[(long long)tc.inst * (A.cap + 1) + n] = dsp_to_double(s_sn);
            const float2 isf = s_is[0];
            // ---- row sums over the 16 segments (4 threads per row, fixed order),
            //      y^{n+1} = u / s_n + w^{n+1} into every CTA of the cluster
            {
                float2* ynext = ybuf + (size_t)((n + 1) & 1) * ldm;
                for (int base = 0; base < 4 * nr; base += CL_THREADS) {
                    const int it = base + tid, i = it >> 2, p = it & 3;
                    float2 y = make_float2(0.f, 0.f);
                    if (i < nr) {
                        const float2* sp = segp + ((size_t)(i >> 5) * CL_WARPS) * 32 + (i & 31);
#pragma unroll
                        for (int w = p; w < CL_WARPS; w += 4) y = dsp_add(y, sp[(size_t)w * 32]);
                    }
                    y = dsp_shfl_add(y, 1);
                    y = dsp_shfl_add(y, 2);
                    if (i < nr && p == 0) {
                        y = dsp_add(dsp_mul(y, isf), wown[i]);
                        for (unsigned r = 0; r < CS; ++r) cl_store2(ynext + r0 + i, r, y.x, y.y);
                    }
                }
            }
        } else {
            if (tid == 0 && tc.first && !s_fail) {
                // the window length and the normalisation of the last step
                A.snorm[(long long)tc.inst * (A.cap + 1) + n] = dsp_to_double(s_sn);
                A.win[tc.inst] = s_wend;
                if (!(isfinite(s_sn.x) && s_sn.x > 0.f)) atomicOr(v.err, SWR_ERR_NUMERIC);
                __threadfence();
                atomicSub(A.n_active, 1);
            }
            // this CTA leaves after the barrier: so does every CTA of its cluster
            if (tid < (int)CS) cl_store_int(&cl_flag[n & 1], (unsigned)tid, 1);
        }
        cl_sync();  // also a barrier of this CTA's threads
        // one read for the whole CTA; the entry is cleared for step n+2 before
        // this CTA arrives at the next barrier (no peer writes it before that)
        if (tid == 0) {
            s_leave = cl_flag[n & 1];
            cl_flag[n & 1] = 0;
        }
        __syncthreads();
        if (s_leave) break;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(A.tmem_cols));
}

// ------------------------------------------------------------- host side

static const void* cluster_kernel(int rows_max, bool onep) {
    switch (cluster_rpl(rows_max)) {
        case 1: return onep ? (const void*)k_window_cluster<1, true> : (const void*)k_window_cluster<1, false>;
        case 2: return onep ? (const void*)k_window_cluster<2, true> : (const void*)k_window_cluster<2, false>;
        case 3: return onep ? (const void*)k_window_cluster<3, true> : (const void*)k_window_cluster<3, false>;
        case 4: return onep ? (const void*)k_window_cluster<4, true> : (const void*)k_window_cluster<4, false>;
        default: return nullptr;
    }
}

// G_hi elements per thread kept in shared memory (a multiple of 4, at most
// rpl sw; the rest go to tensor memory), -1 when not even the vectors fit.
int cluster_hi_smem(int kmax, int kdmax, int rows_max) {
    const int ne = cluster_rpl(rows_max) * cluster_sw(kmax);
    const size_t fixed = cluster_smem_vectors(kmax, kdmax, rows_max), budget = CL_SMEM_MAX;
    if (fixed > budget) return -1;
    const long long h = (long long)((budget - fixed) / (CL_THREADS * sizeof(float))) & ~3LL;
    return h >= ne ? ne : (int)h;
}

size_t window_smem_cluster(int kmax, int kdmax, int rows_max, int hs) {
    const size_t b = cluster_smem_bytes(kmax, kdmax, rows_max, hs);
    return b < CL_SMEM_MIN ? CL_SMEM_MIN : b;
}

// Tensor-memory columns of one CTA (a power of two >= 32): the G_lo of every
// element and the G_hi of those past hs (four warps per lane quarter); 0 when
// more than 512 are needed or a CTA has more than 128 rows.
int cluster_tmem_cols(int kmax, int rows_max, int hs) {
    if (cluster_rpl(rows_max) > 4 || hs < 0) return 0;
    const int ne = cluster_rpl(rows_max) * cluster_sw(kmax);
    const int need = 4 * (ne + (ne - hs));
    int cols = 32;
    while (cols < need) cols <<= 1;
    return cols <= 512 ? cols : 0;
}

static cudaError_t cluster_config(const void* f, size_t smem, int cs) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && cs > 8) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Clusters of cs CTAs (both instantiations for the longest row block) that the
// device holds at once.
cudaError_t cluster_occupancy(int* clusters, int rows_max, size_t smem, int cs, int grid) {
    int best = 1 << 30;
    for (int o = 0; o < 2; ++o) {
        const void* f = cluster_kernel(rows_max, o == 1);
        if (!f) return cudaErrorInvalidValue;
        cudaError_t e = cluster_config(f, smem, cs);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, f, &cfg);
        if (e != cudaSuccess) return e;
        best = n < best ? n : best;
    }
    *clusters = best;
    return cudaSuccess;
}

cudaError_t launch_cluster_window(SweepArgs& a, int grid, int cs, size_t smem, cudaStream_t st, bool onep) {
    const void* f = cluster_kernel(a.rows_max, onep);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = cluster_config(f, smem, cs);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* params[] = {&a};
    return cudaLaunchKernelExC(&cfg, f, params);
}

}  // namespace swr
