// swr_codec.cu -- compact codes of interface-trace windows.
//
// The Robin data g_i(x, t_n) of a subdomain live on its interior edges (edge
// slot 2d + side) at the tangential quadrature nodes, for the steps of a time
// window.  A code is the projection of each edge's data onto a product basis:
// Phi_s(x) (discrete orthonormal polynomials of degree < S on the edge nodes,
// inner product sum_t w_t f g with the quadrature weights; S = 1 for the
// point-edges of a 1-electron problem) times Psi_t(n) (discrete orthonormal
// polynomials of degree < Tm in the step index, plain sum).  Layout per
// subdomain: [4 slots][nch channels][S][Tm] floats; absent slots are zero.
// The learned initial guess predicts codes; swr_trace_decode_set turns a code
// back into Robin data and into the Robin source b' of the next iteration,
// replacing the zero initial traces g^(0) = 0.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "swr_internal.cuh"

namespace swr {

struct CodecInputs {
    SwrDeviceView v;
    cudaStream_t stream;
    int n_sub, n_inst, window, nch, max_q;
    int* d_win_prev;
    std::vector<int>* win_prev_h;
    std::vector<int>* win_h;
    bool* codec_ready;
};
bool codec_inputs(swr_ctx* c, CodecInputs* r);
void set_error(swr_ctx* c, const char* msg);
void codec_release(const swr_ctx* c);

#define CODEC_SMAX 16
#define CODEC_TMAX 32

// Gram-Schmidt of the monomials/Chebyshev polynomials on the node set.
// Phi: [sid][4][q][S] (spatial, per slot), Psi: [window+1][Tm] (shared by all).
__global__ void k_codec_basis(SwrDeviceView v, double* Phi, double* Psi, int S, int Tm, int W, int qmax) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    T1Layout lay(s.q, s.kd);
    if (threadIdx.x == 0) {
        for (int slot = 0; slot < 4; ++slot) {
            double* P = Phi + ((long long)sid * 4 + slot) * qmax * S;
            for (int e = 0; e < qmax * S; ++e) P[e] = 0.0;
            if (s.gam_off[slot] < 0) continue;
            const int d = slot / 2;
            if (s.N == 1) {  // a point: one basis function equal to 1
                P[0] = 1.0;
                continue;
            }
            const double* To = v.arena + s.t1[1 - d];
            const int q = s.q;
            const double lo = s.lo[1 - d], hi = s.hi[1 - d];
            for (int k = 0; k < S; ++k) {
                for (int t = 0; t < q; ++t) {
                    double x = 2.0 * (To[lay.x() + t] - lo) / (hi - lo) - 1.0;
                    // Chebyshev T_k(x) as the starting vector
                    double t0 = 1.0, t1 = x, tk = (k == 0) ? 1.0 : x;
                    for (int m = 2; m <= k; ++m) {
                        tk = 2.0 * x * t1 - t0;
                        t0 = t1;
                        t1 = tk;
                    }
                    P[t * S + k] = tk;
                }
                for (int pass = 0; pass < 2; ++pass)
                    for (int j = 0; j < k; ++j) {
                        double dot = 0;
                        for (int t = 0; t < q; ++t) dot += To[lay.w() + t] * P[t * S + k] * P[t * S + j];
                        for (int t = 0; t < q; ++t) P[t * S + k] -= dot * P[t * S + j];
                    }
                double nrm = 0;
                for (int t = 0; t < q; ++t) nrm += To[lay.w() + t] * P[t * S + k] * P[t * S + k];
                nrm = sqrt(nrm);
                for (int t = 0; t < q; ++t) P[t * S + k] /= nrm;
            }
        }
        if (sid == 0) {
            for (int k = 0; k < Tm; ++k) {
                for (int n = 0; n <= W; ++n) {
                    double x = (W > 0) ? 2.0 * n / W - 1.0 : 0.0;
                    double t0 = 1.0, t1 = x, tk = (k == 0) ? 1.0 : x;
                    for (int m = 2; m <= k; ++m) {
                        tk = 2.0 * x * t1 - t0;
                        t0 = t1;
                        t1 = tk;
                    }
                    Psi[n * Tm + k] = tk;
                }
                for (int pass = 0; pass < 2; ++pass)
                    for (int j = 0; j < k; ++j) {
                        double dot = 0;
                        for (int n = 0; n <= W; ++n) dot += Psi[n * Tm + k] * Psi[n * Tm + j];
                        for (int n = 0; n <= W; ++n) Psi[n * Tm + k] -= dot * Psi[n * Tm + j];
                    }
                double nrm = 0;
                for (int n = 0; n <= W; ++n) nrm += Psi[n * Tm + k] * Psi[n * Tm + k];
                nrm = sqrt(nrm);
                for (int n = 0; n <= W; ++n) Psi[n * Tm + k] /= nrm;
            }
        }
    }
}

// code[sid][slot][ch][s][t] = sum_{node, n} w Phi[node][s] Psi[n][t] g[n][ch][node]
__global__ void k_codec_encode(SwrDeviceView v, const double* Phi, const double* Psi, int S, int Tm, int W, int qmax,
                               float* code) {
    const int sid = blockIdx.x, slot = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int nch = in.mode == SWR_MODE_TDSE ? 2 : 1;
    const long long per = 4LL * 2 * S * Tm;
    float* out = code + sid * per + (long long)slot * 2 * S * Tm;
    const int npts = (s.N == 1) ? 1 : s.q;
    T1Layout lay(s.q, s.kd);
    const double* P = Phi + ((long long)sid * 4 + slot) * qmax * S;
    const double* To = v.arena + s.t1[s.N == 2 ? 1 - slot / 2 : 0];
    for (int e = threadIdx.x; e < 2 * S * Tm; e += blockDim.x) {
        const int ch = e / (S * Tm), k = (e / Tm) % S, t = e % Tm;
        double acc = 0;
        if (s.gam_off[slot] >= 0 && ch < nch) {
            for (int n = 0; n <= W; ++n) {
                const double* g = v.arena + s.g + ((long long)n * nch + ch) * s.ngam + s.gam_off[slot];
                double sp = 0;
                for (int p = 0; p < npts; ++p) {
                    const double w = (s.N == 1) ? 1.0 : To[lay.w() + p];
                    sp += w * P[p * S + k] * g[p];
                }
                acc += Psi[n * Tm + t] * sp;
            }
        }
        out[e] = (float)acc;
    }
}

// g[n][ch][node] = sum_{s,t} code Phi Psi, written as the Robin data of the
// previous iteration.
__global__ void k_codec_decode(SwrDeviceView v, const double* Phi, const double* Psi, int S, int Tm, int W, int qmax,
                               const float* code) {
    const int sid = blockIdx.x;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int nch = in.mode == SWR_MODE_TDSE ? 2 : 1;
    const long long per = 4LL * 2 * S * Tm;
    for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < (long long)(W + 1) * nch * s.ngam;
         e += (long long)blockDim.x * gridDim.y) {
        const int node = (int)(e % s.ngam);
        const int ch = (int)((e / s.ngam) % nch);
        const int n = (int)(e / ((long long)s.ngam * nch));
        int slot = -1, p = 0;
        for (int sl = 3; sl >= 0; --sl)
            if (s.gam_off[sl] >= 0 && node >= s.gam_off[sl]) {
                slot = sl;
                p = node - s.gam_off[sl];
                break;
            }
        const float* c = code + sid * per + ((long long)slot * 2 + ch) * S * Tm;
        const double* P = Phi + ((long long)sid * 4 + slot) * qmax * S;
        double acc = 0;
        for (int k = 0; k < S; ++k) {
            double pt = 0;
            for (int t = 0; t < Tm; ++t) pt += (double)c[k * Tm + t] * Psi[n * Tm + t];
            acc += P[p * S + k] * pt;
        }
        v.arena[s.g + ((long long)n * nch + ch) * s.ngam + node] = acc;
    }
}

// b'[n] from the Robin data g[n] (the same projection as at the end of an iteration).
__global__ void k_bvec_from_g(SwrDeviceView v, int W) {
    const int sid = blockIdx.y;
    const SubDev& s = v.sub[sid];
    const InstDev& in = v.inst[s.inst];
    const int nch = in.mode == SWR_MODE_TDSE ? 2 : 1;
    const int kd = s.kd, q = s.q, K = s.K;
    T1Layout lay(q, kd);
    __shared__ double hsum[4][64];
    for (int item = blockIdx.x; item < (W + 1) * nch; item += gridDim.x) {
        const int n = item / nch, ch = item % nch;
        const double* gs = v.arena + s.g + ((long long)n * nch + ch) * s.ngam;
        double* bdst = v.arena + s.bvec + ((long long)n * nch + ch) * K;
        if (s.N == 1) {
            const double* T = v.arena + s.t1[0];
            for (int a = threadIdx.x; a < kd; a += blockDim.x) {
                double acc = 0;
                for (int sl = 0; sl < 2; ++sl) {
                    if (s.gam_off[sl] < 0) continue;
                    acc += gs[s.gam_off[sl]] * T[lay.Lv() + (sl ? 3 : 0) * kd + a];
                }
                bdst[a] = acc;
            }
        } else {
            for (int e = threadIdx.x; e < 4 * kd; e += blockDim.x) {
                int sl = e / kd, m = e % kd;
                double acc = 0;
                if (s.gam_off[sl] >= 0) {
                    const double* To = v.arena + s.t1[1 - sl / 2];
                    for (int t = 0; t < q; ++t) acc += To[lay.w() + t] * gs[s.gam_off[sl] + t] * To[lay.B() + t * kd + m];
                }
                hsum[sl][m] = acc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < K; e += blockDim.x) {
                int a = e % kd, b = e / kd;
                double acc = 0;
                for (int sl = 0; sl < 4; ++sl) {
                    if (s.gam_off[sl] < 0) continue;
                    int d = sl / 2, l = (sl % 2) ? 3 : 0;
                    const double* Td = v.arena + s.t1[d];
                    if (d == 0) acc += Td[lay.Lv() + l * kd + a] * hsum[sl][b];
                    else acc += hsum[sl][a] * Td[lay.Lv() + l * kd + b];
                }
                bdst[e] = acc;
            }
        }
        __syncthreads();
    }
}

}  // namespace swr

using namespace swr;

struct CodecState {
    int S = 0, Tm = 0, W = 0, qmax = 0;
    double *Phi = nullptr, *Psi = nullptr;
};

// The codec buffers are owned by a small registry keyed by context pointer.
#include <map>
#include <mutex>
static std::map<const swr_ctx*, CodecState> g_codecs;
static std::mutex g_codec_mutex;

extern "C" swr_status swr_trace_codec(swr_ctx* ctx, int S, int Tm, size_t* floats_per_sub) {
    CodecInputs r;
    if (!ctx || !floats_per_sub || !codec_inputs(ctx, &r)) return SWR_EINVAL;
    if (S < 1 || S > CODEC_SMAX || Tm < 1 || Tm > CODEC_TMAX || r.window < 1) {
        set_error(ctx, "swr_trace_codec: need 1 <= S <= 16, 1 <= Tm <= 32 and a fixed time window");
        return SWR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_codec_mutex);
    CodecState& cs = g_codecs[ctx];
    if (cs.Phi) cudaFree(cs.Phi);
    if (cs.Psi) cudaFree(cs.Psi);
    cs.S = S;
    cs.Tm = Tm;
    cs.W = r.window;
    cs.qmax = r.max_q;
    cudaError_t e = cudaMalloc(&cs.Phi, sizeof(double) * (size_t)r.n_sub * 4 * cs.qmax * S);
    if (e == cudaSuccess) e = cudaMalloc(&cs.Psi, sizeof(double) * (size_t)(cs.W + 1) * Tm);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ENOMEM;
    }
    k_codec_basis<<<r.n_sub, 32, 0, r.stream>>>(r.v, cs.Phi, cs.Psi, S, Tm, cs.W, cs.qmax);
    e = cudaStreamSynchronize(r.stream);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ECUDA;
    }
    *floats_per_sub = (size_t)4 * 2 * S * Tm;
    return SWR_OK;
}

// Code of the Robin data of the last iteration, into a device array
// [n_sub][4][2][S][Tm] floats.
extern "C" swr_status swr_trace_encode(swr_ctx* ctx, float* code_dev) {
    CodecInputs r;
    if (!ctx || !code_dev || !codec_inputs(ctx, &r)) return SWR_EINVAL;
    std::lock_guard<std::mutex> lock(g_codec_mutex);
    auto it = g_codecs.find(ctx);
    if (it == g_codecs.end() || !it->second.Phi) {
        set_error(ctx, "swr_trace_encode: call swr_trace_codec first");
        return SWR_ESTATE;
    }
    const CodecState& cs = it->second;
    k_codec_encode<<<dim3(r.n_sub, 4), 256, 0, r.stream>>>(r.v, cs.Phi, cs.Psi, cs.S, cs.Tm, cs.W, cs.qmax, code_dev);
    cudaError_t e = cudaStreamSynchronize(r.stream);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ECUDA;
    }
    return SWR_OK;
}

// Replaces the initial traces of the next Schwarz iteration by the decoded
// code (device array, same layout as swr_trace_encode).
extern "C" swr_status swr_trace_decode_set(swr_ctx* ctx, const float* code_dev) {
    CodecInputs r;
    if (!ctx || !code_dev || !codec_inputs(ctx, &r)) return SWR_EINVAL;
    std::lock_guard<std::mutex> lock(g_codec_mutex);
    auto it = g_codecs.find(ctx);
    if (it == g_codecs.end() || !it->second.Phi) {
        set_error(ctx, "swr_trace_decode_set: call swr_trace_codec first");
        return SWR_ESTATE;
    }
    const CodecState& cs = it->second;
    k_codec_decode<<<dim3(r.n_sub, 16), 256, 0, r.stream>>>(r.v, cs.Phi, cs.Psi, cs.S, cs.Tm, cs.W, cs.qmax, code_dev);
    k_bvec_from_g<<<dim3(64, r.n_sub), 256, 0, r.stream>>>(r.v, cs.W);
    std::vector<int> w(r.n_inst, cs.W);
    cudaError_t e = cudaMemcpyAsync(r.d_win_prev, w.data(), sizeof(int) * r.n_inst, cudaMemcpyHostToDevice, r.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r.stream);
    if (e != cudaSuccess) {
        set_error(ctx, cudaGetErrorString(e));
        return SWR_ECUDA;
    }
    *r.win_prev_h = w;
    *r.win_h = w;
    return SWR_OK;
}

void swr::codec_release(const swr_ctx* ctx) {
    std::lock_guard<std::mutex> lock(g_codec_mutex);
    auto it = g_codecs.find(ctx);
    if (it == g_codecs.end()) return;
    if (it->second.Phi) cudaFree(it->second.Phi);
    if (it->second.Psi) cudaFree(it->second.Psi);
    g_codecs.erase(it);
}
