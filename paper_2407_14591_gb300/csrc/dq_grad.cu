// Coefficient gradients of the product: for y = H x with H = sum_q c_q T_q, and a cotangent dy,
//   g_q = d <dy, y> / d c_q = sum_i sum_r dy[i, r] (T_q x)[i, r]
// for every term q (T_q is term q with coefficient 1; r runs over the right-hand sides, so a
// complex vector stored as two real columns gives Re <dy, T_q x>). The gradient with respect to
// x is H^T dy = H dy (every term is real and Hermitian), i.e. another product.
//
// One thread per row: the row state by Alg. 4, then up to 32 terms per pass, each evaluated in
// the gather reading (a hop term ranks the produced state with Eq. (index) and reads x there),
// reduced per CTA in a fixed order, and summed over CTAs in a fixed order by a second kernel.
// The result does not depend on timing.
//
// Arithmetic. For Q = 2 (spins, the hot case) the products dy * x are fixed point: x and dy are
// scaled per column to int64 (dq_fixed.cuh), each product DY * X is formed in 128 bits and
// shifted onto one common grid 2^-G with |value| < 2^48, and every term sums these in an int64
// register (no FP64 work per row and term). The kind's factor (1/4, 1/2, 1, -1) and 2^-G are
// applied to each thread's sum, which then enters the FP64 reduction. Other Q use FP64 products
// (the boson amplitudes sqrt((n+1) n) are not integers).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
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

// (a * b) / 2^sh rounded to nearest, for 64 <= sh: the 128-bit product shifted onto the common
// grid of the fixed-point gradient sums.
__device__ __forceinline__ long long mul_shift(long long a, long long b, int sh) {
    if (sh >= 126) return 0;  // |a b| < 2^112 <= 2^(sh - 14): rounds to zero
    unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    long long hi = __mul64hi(a, b);
    if (sh > 64) {
        hi += 1ll << (sh - 65);
    } else {
        const unsigned long long nlo = lo + (1ull << 63);
        hi += nlo < lo ? 1 : 0;
    }
    return hi >> (sh - 64);
}

// Q = 2 gradients in fixed point (see the header). X, DY: int64 copies of x, dy; hx, hdy: their
// column scales. Row counts per thread stay below 2^14 (grid chosen by the host), so the int64
// sums of values below 2^48 cannot overflow.
__global__ void __launch_bounds__(kGradThreads)
    k_term_grads_fx(DevSector S, const GradTerm* __restrict__ gt, int t0, int tcnt, const long long* __restrict__ X,
                    const long long* __restrict__ DY, int nrhs, const ColScale* __restrict__ hx,
                    const ColScale* __restrict__ hdy, bool use_sm, double* __restrict__ partial) {
    extern __shared__ uint64_t sm[];
    __shared__ double red[kGradThreads / 32][kGradChunk];
    __shared__ GradTerm g_s[kGradChunk];
    __shared__ int sh_s[kMaxCols];
    __shared__ int G_s, bad_s;
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    if (threadIdx.x < tcnt) g_s[threadIdx.x] = gt[t0 + threadIdx.x];
    if (threadIdx.x == 0) {
        // common grid: the largest column bound of |dy x| lands below 2^(48 - lg nrhs)
        int lg = 0;
        while ((1 << lg) < nrhs) ++lg;
        int fmin = 1 << 30;
        for (int r = 0; r < nrhs; ++r) fmin = min(fmin, hx->F[r] + hdy->F[r]);
        G_s = fmin - 64 - lg;
        for (int r = 0; r < nrhs; ++r) sh_s[r] = hx->F[r] + hdy->F[r] - G_s;
        bad_s = hx->bad | hdy->bad;
    }
    __syncthreads();
    if (bad_s) {  // an Inf or NaN in x or dy: the gradients are NaN and the error word is raised
        if (threadIdx.x < tcnt) partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    const bool lin2 = S.n_sub == 2;
    long long acc[kGradChunk];
#pragma unroll
    for (int u = 0; u < kGradChunk; ++u) acc[u] = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = d_unrank(S, off_s, str_s, i);
        const long long* Xi = X + i * nrhs;
        const long long* Di = DY + i * nrhs;
        long long p = 0;  // sum_r dy[i, r] x[i, r] on the grid 2^-G
        for (int r = 0; r < nrhs; ++r) p += mul_shift(__ldg(Di + r), __ldg(Xi + r), sh_s[r]);
#pragma unroll
        for (int u = 0; u < kGradChunk; ++u) {
            if (u >= tcnt) break;
            const GradTerm g = g_s[u];
            const int ni = (int)((s >> g.sh_i) & 1ull);
            const int nj = g.sh_j >= 0 ? (int)((s >> g.sh_j) & 1ull) : 0;
            switch (g.kind) {
                case DQ_ZZ: acc[u] += ni == nj ? p : -p; break;  // (n_i - 1/2)(n_j - 1/2) = +-1/4
                case DQ_Z: acc[u] += ni ? p : -p; break;         // n_i - 1/2 = +-1/2
                case DQ_NN: acc[u] += (ni & nj) ? p : 0; break;
                case DQ_N: acc[u] += ni ? p : 0; break;
                case DQ_XY:
                case DQ_HOP:
                    if (ni != nj) {  // exactly one direction moves the particle
                        const uint64_t s2 = s ^ ((1ull << g.sh_i) | (1ull << g.sh_j));
                        const uint64_t j = lin2 ? d_rank_lin2(S, s2) : d_rank(S, off_s, str_s, s2);
                        const long long* Xj = X + j * nrhs;
                        long long h = 0;
                        for (int r = 0; r < nrhs; ++r) h += mul_shift(__ldg(Di + r), __ldg(Xj + r), sh_s[r]);
                        acc[u] += h;
                    }
                    break;
                default: break;  // DQ_U: n (n - 1) = 0 for Q = 2
            }
        }
    }
    // each thread's sums to FP64 with the kind's factor and 2^-G, then the fixed-order reduction
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < kGradChunk; ++u) {
        double f = 0.0;
        if (u < tcnt) {
            switch (g_s[u].kind) {
                case DQ_ZZ: f = 0.25; break;
                case DQ_Z: f = 0.5; break;
                case DQ_XY: f = 0.5; break;
                case DQ_HOP: f = -1.0; break;
                default: f = 1.0; break;
            }
        }
        double v = ldexp(f * (double)acc[u], -G_s);
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
    if (s->wide) return set_error(DQ_EINVAL, "dq_term_grads serves states of one 64-bit word (L * Nbits <= 64)");
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
    const bool fx = s->Q == 2;  // fixed-point route
    // at most 2^14 rows per thread on the fixed-point route (int64 sums of values < 2^48)
    const uint64_t min_blocks = (s->D + (uint64_t)kGradThreads * 16384 - 1) / ((uint64_t)kGradThreads * 16384);
    const int nb = (int)std::max<uint64_t>(2 * (uint64_t)sms, min_blocks);
    std::vector<double> amp((size_t)s->Q * s->Q);
    for (int a = 0; a < s->Q; ++a)
        for (int b = 0; b < s->Q; ++b) amp[(size_t)a * s->Q + b] = std::sqrt((double)((a + 1) * b));
    // workspace kept with the sector: column headers, terms, amplitude table, partial sums and (on
    // the fixed-point route) int64 copies of x and dy. The call synchronises before it returns,
    // so the next call may reuse it.
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_hdy = kColScaleBytes, o_gt = 2 * kColScaleBytes;
    const size_t o_amp = o_gt + al(sizeof(GradTerm) * n_terms);
    const size_t o_part = o_amp + al(sizeof(double) * amp.size());
    const size_t o_x = o_part + al(sizeof(double) * kGradChunk * nb);
    const size_t vec = fx ? al((size_t)s->D * nrhs * sizeof(long long)) : 0;
    const size_t need = o_x + 2 * vec;
    dq_sector* sw = const_cast<dq_sector*>(s);
    cudaError_t e = cudaSuccess;
    if (sw->grad_ws_bytes < need) {
        if (sw->grad_ws) cudaFree(sw->grad_ws);
        sw->grad_ws = nullptr;
        sw->grad_ws_bytes = 0;
        e = cudaMalloc(&sw->grad_ws, need);
        if (e != cudaSuccess) return set_error(DQ_ENOMEM, "term gradients workspace (%zu bytes): %s", need,
                                               cudaGetErrorString(e));
        sw->grad_ws_bytes = need;
    }
    char* ws = reinterpret_cast<char*>(sw->grad_ws);
    ColScale* hx = reinterpret_cast<ColScale*>(ws);
    ColScale* hdy = reinterpret_cast<ColScale*>(ws + o_hdy);
    GradTerm* d_gt = reinterpret_cast<GradTerm*>(ws + o_gt);
    double* d_amp = reinterpret_cast<double*>(ws + o_amp);
    double* d_part = reinterpret_cast<double*>(ws + o_part);
    long long* X = reinterpret_cast<long long*>(ws + o_x);
    long long* DYf = reinterpret_cast<long long*>(ws + o_x + vec);
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d_gt, gt.data(), sizeof(GradTerm) * n_terms, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_amp, amp.data(), sizeof(double) * amp.size(), cudaMemcpyHostToDevice, st);
    const bool use_sm = (size_t)s->dev.os_total * 16 <= 48 * 1024;
    const size_t smb = use_sm ? (size_t)s->dev.os_total * 16 : 0;
    const int tslot = e == cudaSuccess ? timing_start(st) : -1;
    int launched = 0;
    if (e == cudaSuccess && fx) {
        if (dtype == DQ_F64) {
            launch_col_prepass<double, long long>((const double*)x, X, s->D, nrhs, hx, sms, st);
            launch_col_prepass<double, long long>((const double*)dy, DYf, s->D, nrhs, hdy, sms, st);
        } else {
            launch_col_prepass<float, long long>((const float*)x, X, s->D, nrhs, hx, sms, st);
            launch_col_prepass<float, long long>((const float*)dy, DYf, s->D, nrhs, hdy, sms, st);
        }
        launched += 4;
    }
    for (int t0 = 0; e == cudaSuccess && t0 < n_terms; t0 += kGradChunk, launched += 2) {
        const int tcnt = n_terms - t0 < kGradChunk ? n_terms - t0 : kGradChunk;
        if (fx)
            k_term_grads_fx<<<nb, kGradThreads, smb, st>>>(s->dev, d_gt, t0, tcnt, X, DYf, nrhs, hx, hdy, use_sm,
                                                         d_part);
        else if (dtype == DQ_F64)
            k_term_grads<double><<<nb, kGradThreads, smb, st>>>(s->dev, d_gt, t0, tcnt, (const double*)x,
                                                              (const double*)dy, nrhs, d_amp, use_sm, d_part);
        else
            k_term_grads<float><<<nb, kGradThreads, smb, st>>>(s->dev, d_gt, t0, tcnt, (const float*)x,
                                                             (const float*)dy, nrhs, d_amp, use_sm, d_part);
        k_grad_finish<<<1, tcnt, 0, st>>>(d_part, nb, d_grads + t0);
        e = cudaGetLastError();
    }
    timing_stop(tslot, st, launched);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "term gradients: %s", cudaGetErrorString(e));
    return DQ_OK;
}
