// swr_noalloc.cu -- Res(k) recomputed without any device allocation.
//
// swr_residual_noalloc() repeats the interface-residual reduction of the last
// Schwarz iteration (the same k_residual / k_residual_reduce kernels that
// swr_step runs) but keeps its scratch -- the per-block partial sums, the two
// window-length arrays and the per-instance result -- in one file-scope
// __device__ array instead of the context's workspace.  It exists for callers
// that must not allocate device memory at the point of the call.
#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>
#include <stdio.h>

#include "swr_internal.cuh"

using namespace swr;

// Capacity of the static scratch, in doubles (2 MiB).  Layout of one call:
// [window ints: 2*n_inst, padded to doubles] [partials: RES_BLOCKS*n_sub] [res: n_inst]
#define SWR_NOALLOC_SCRATCH_DOUBLES (1 << 18)
#define SWR_NOALLOC_RES_BLOCKS 8

static __device__ __align__(256) double g_noalloc_scratch[SWR_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch (the host-side name is only a stand-in
// and must never be passed to a kernel), resolved once per device and CUDA
// context: the unique id of the current context is kept beside the address,
// so that after cudaDeviceReset (a new primary context) the address is
// resolved again instead of reusing one from the destroyed context.  The
// context id comes from the driver through the runtime's entry-point query
// (no link dependency on the driver library).
static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[64] = {nullptr};
static unsigned long long g_noalloc_ctx[64] = {0};

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);
typedef CUresult (*PFN_ctx_get_id)(CUcontext, unsigned long long*);

// Unique id of the current CUDA context, 0 when it cannot be read.
static unsigned long long current_context_id() {
    static PFN_ctx_get_current get_current = nullptr;
    static PFN_ctx_get_id get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = (PFN_ctx_get_current)f1;
            get_id = (PFN_ctx_get_id)f2;
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static cudaError_t noalloc_scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double*)p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

extern "C" swr_status swr_residual_noalloc(swr_ctx* ctx, double* res_host, size_t n) {
    if (!ctx || !res_host) return SWR_EINVAL;
    ResidualInputs r;
    if (!residual_inputs(ctx, &r)) {
        set_error(ctx, "swr_residual_noalloc: no Schwarz iteration completed since the last assembly, trace "
                       "restore or failed step");
        return SWR_ESTATE;
    }
    if (n != (size_t)r.n_inst) {
        set_error(ctx, "swr_residual_noalloc: n must equal the number of instances");
        return SWR_EINVAL;
    }
    const long long win_doubles = (2LL * r.n_inst + 1) / 2;
    const long long need = win_doubles + (long long)SWR_NOALLOC_RES_BLOCKS * r.n_sub + r.n_inst;
    if (need > SWR_NOALLOC_SCRATCH_DOUBLES) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "swr_residual_noalloc: problem needs %lld scratch doubles, the static limit is %d "
                 "(at most %lld subdomains for %d instances)", need, SWR_NOALLOC_SCRATCH_DOUBLES,
                 (SWR_NOALLOC_SCRATCH_DOUBLES - win_doubles - r.n_inst) / SWR_NOALLOC_RES_BLOCKS, r.n_inst);
        set_error(ctx, msg);
        return SWR_EINVAL;
    }
    double* base = nullptr;
    cudaError_t e = noalloc_scratch_for_current_device(&base);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ECUDA;
    }
    int* d_win = (int*)base;
    int* d_win_before = d_win + r.n_inst;
    double* d_part = base + win_doubles;
    double* d_res = d_part + (long long)SWR_NOALLOC_RES_BLOCKS * r.n_sub;
    // every partial slot and every result is overwritten by the kernels, so
    // nothing in the shared array has to be cleared between calls
    e = cudaMemcpyAsync(d_win, r.win_last, r.n_inst * sizeof(int), cudaMemcpyHostToDevice, r.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_win_before, r.win_before, r.n_inst * sizeof(int), cudaMemcpyHostToDevice, r.stream);
    if (e == cudaSuccess)
        e = launch_residual(r.v, r.stream, d_win, d_win_before, r.parity_last, r.k == 1 ? 1 : 0, d_part,
                            SWR_NOALLOC_RES_BLOCKS, d_res);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res_host, d_res, n * sizeof(double), cudaMemcpyDeviceToHost, r.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r.stream);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ECUDA;
    }
    return SWR_OK;
}
