// Coefficient gradients of the product: for y = H x with H = sum_q c_q T_q, and a cotangent dy,
//   g_q = d <dy, y> / d c_q = sum_i sum_r dy[i, r] (T_q x)[i, r]
// for every term q (T_q is term q with coefficient 1; r runs over the right-hand sides, so a
// complex vector stored as two real columns gives Re <dy, T_q x>). The gradient with respect to
// x is H^T dy = H dy (every term is real and Hermitian), i.e. another product.
//
// One thread per row: the row state by Alg. 4, then up to 32 terms per pass, each evaluated in
// the gather reading (a hop term ranks the produced state with Eq. (index) and reads x there),
// accumulated in FP64 registers, reduced per CTA in a fixed order, and summed over CTAs in a fixed
// order by a second kernel. The result does not depend on timing.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dq_device.cuh"
#include "dq_internal.h"

namespace dq {

constexpr int kGradChunk = 32;
constexpr int kGradThreads = 256;

struct GradTerm {
    int kind;
    int sh_i, sh_j;  // bit shifts of the digits of sites i and j (j unused by single-site kinds)
};

template <typename T>
__global__ void __launch_bounds__(kGradThreads) k_term_grads(DevSector S, const GradTerm* __restrict__ gt, int t0,
                                                             int tcnt, const T* __restrict__ x,
                                                             const T* __restrict__ dy, int nrhs,
                                                             const double* __restrict__ amp, bool use_sm,
                                                             double* __restrict__ partial) {
    extern __shared__ uint64_t sm[];
    __shared__ double red[kGradThreads / 32][kGradChunk];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    const int Q = S.Q;
    const uint64_t dm = (1ull << S.nb) - 1;
    const bool lin2 = S.n_sub == 2;
    double acc[kGradChunk];
#pragma unroll
    for (int u = 0; u < kGradChunk; ++u) acc[u] = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = d_unrank(S, off_s, str_s, i);
        const T* xi = x + i * nrhs;
        const T* di = dy + i * nrhs;
        double xd = 0.0;  // sum_r dy[i, r] x[i, r] for the diagonal kinds
        for (int r = 0; r < nrhs; ++r) xd += (double)__ldg(di + r) * (double)__ldg(xi + r);
#pragma unroll
        for (int u = 0; u < kGradChunk; ++u) {
            if (u >= tcnt) break;
            const GradTerm g = gt[t0 + u];
            const int ni = (int)((s >> g.sh_i) & dm);
            const int nj = g.sh_j >= 0 ? (int)((s >> g.sh_j) & dm) : 0;
            double v = 0.0;
            switch (g.kind) {
                case DQ_ZZ: v = ((double)ni - 0.5) * ((double)nj - 0.5) * xd; break;
                case DQ_Z: v = ((double)ni - 0.5) * xd; break;
                case DQ_NN: v = (double)(ni * nj) * xd; break;
                case DQ_N: v = (double)ni * xd; break;
                case DQ_U: v = 0.5 * (double)(ni * (ni - 1)) * xd; break;
                case DQ_XY:
                case DQ_HOP: {
                    // both directions of the Hermitian pair: b+_i b_j and b+_j b_i
#pragma unroll
                    for (int dir = 0; dir < 2; ++dir) {
                        const int su = dir ? g.sh_j : g.sh_i, sd = dir ? g.sh_i : g.sh_j;
                        const int nu = dir ? nj : ni, nd = dir ? ni : nj;
                        if (nu < Q - 1 && nd > 0) {
                            const uint64_t s2 = s + (1ull << su) - (1ull << sd);
                            const uint64_t j = lin2 ? d_rank_lin2(S, s2) : d_rank(S, off_s, str_s, s2);
                            const double a = g.kind == DQ_XY ? 0.5 : -amp[nu * Q + nd];
                            const T* xj = x + j * nrhs;
                            double t = 0.0;
                            for (int r = 0; r < nrhs; ++r) t += (double)__ldg(di + r) * (double)__ldg(xj + r);
                            v += a * t;
                        }
                    }
                    break;
                }
            }
            acc[u] += v;
        }
    }
    // CTA reduction in a fixed order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < kGradChunk; ++u) {
        double v = acc[u];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][u] = v;
    }
    __syncthreads();
    if (threadIdx.x < kGradChunk && threadIdx.x < tcnt) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_grad_finish(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    // one thread per term, blocks summed in order
    const int u = threadIdx.x;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += partial[(size_t)u * nb + b];
    out[u] = v;
}

}  // namespace dq

using namespace dq;

extern "C" int dq_term_grads(const dq_sector* s, const dq_term* terms, int n_terms, const void* x, const void* dy,
                             int dtype, int nrhs, double* d_grads, void* stream) {
    clear_error();
    if (!s || (n_terms > 0 && !terms) || !x || !dy || !d_grads) return set_error(DQ_EINVAL, "NULL argument");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    if (nrhs < 1 || nrhs > 64) return set_error(DQ_EINVAL, "nrhs must be in [1, 64]");
    if (n_terms == 0) return DQ_OK;
    std::vector<GradTerm> gt(n_terms);
    for (int q = 0; q < n_terms; ++q) {
        const dq_term& u = terms[q];
        if (u.kind < DQ_XY || u.kind > DQ_U) return set_error(DQ_EINVAL, "term %d: unknown kind %d", q, u.kind);
        if (u.i < 0 || u.i >= s->L) return set_error(DQ_EINVAL, "term %d: site i out of range", q);
        const bool pair = u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_HOP || u.kind == DQ_NN;
        if (pair && (u.j < 0 || u.j >= s->L || u.j == u.i))
            return set_error(DQ_EINVAL, "term %d: pair term needs two distinct sites in range", q);
        const bool spin = u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_Z;
        if (spin && s->Q != 2) return set_error(DQ_EINVAL, "term %d: spin-1/2 kinds need Q = 2", q);
        gt[q].kind = u.kind;
        gt[q].sh_i = s->nb * (s->L - 1 - u.i);
        gt[q].sh_j = pair ? s->nb * (s->L - 1 - u.j) : -1;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = 2 * sms;
    std::vector<double> amp((size_t)s->Q * s->Q);
    for (int a = 0; a < s->Q; ++a)
        for (int b = 0; b < s->Q; ++b) amp[(size_t)a * s->Q + b] = std::sqrt((double)((a + 1) * b));
    // scratch: terms, amplitude table, partials (freed before returning; the call synchronises)
    void *d_gt = nullptr, *d_amp = nullptr, *d_part = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&d_gt, sizeof(GradTerm) * n_terms);
    if (e == cudaSuccess) e = cudaMalloc(&d_amp, sizeof(double) * amp.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_part, sizeof(double) * kGradChunk * nb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_gt, gt.data(), sizeof(GradTerm) * n_terms, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_amp, amp.data(), sizeof(double) * amp.size(), cudaMemcpyHostToDevice, st);
    const bool use_sm = (size_t)s->dev.os_total * 16 <= 48 * 1024;
    const size_t smb = use_sm ? (size_t)s->dev.os_total * 16 : 0;
    const int tslot = e == cudaSuccess ? timing_start(st) : -1;
    int launched = 0;
    for (int t0 = 0; e == cudaSuccess && t0 < n_terms; t0 += kGradChunk, launched += 2) {
        const int tcnt = n_terms - t0 < kGradChunk ? n_terms - t0 : kGradChunk;
        if (dtype == DQ_F64)
            k_term_grads<double><<<nb, kGradThreads, smb, st>>>(s->dev, (const GradTerm*)d_gt, t0, tcnt,
                                                              (const double*)x, (const double*)dy, nrhs,
                                                              (const double*)d_amp, use_sm, (double*)d_part);
        else
            k_term_grads<float><<<nb, kGradThreads, smb, st>>>(s->dev, (const GradTerm*)d_gt, t0, tcnt,
                                                             (const float*)x, (const float*)dy, nrhs,
                                                             (const double*)d_amp, use_sm, (double*)d_part);
        k_grad_finish<<<1, tcnt, 0, st>>>((const double*)d_part, nb, d_grads + t0);
        e = cudaGetLastError();
    }
    timing_stop(tslot, st, launched);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_gt);
    cudaFree(d_amp);
    cudaFree(d_part);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "term gradients: %s", cudaGetErrorString(e));
    return DQ_OK;
}
