// Device kernels: batched rank / unrank and the general matrix-free product y = H x.
//
// rank   = Alg. 2 / Eq. (index): sum over subsystems of offset_k(n_k, lambda_k) + stride_k(n_k,
//          lambda_k) * index_k(sigma^(k)), the local index read from the subsystem's table.
// unrank = Alg. 4: per subsystem, the particle number n_k with offset(n_k) <= idx <
//          offset(n_k + 1), the local index idx / stride, and the reverse table.
// product: every thread owns rows of y (the paper's workers own consecutive rows, Sec. 2.2),
//          unranks its row, evaluates the diagonal, applies every off-diagonal term, ranks each
//          produced state and gathers x at that index: y_i = d_i x_i + sum_j h_ij x_j. Each y_i
//          is written once by one thread, so no atomics are needed and the result is
//          deterministic. The sums are exact fixed point (dq_fixed.cuh): x is first scaled per
//          column to int64 (FP64 vectors) or int32 (FP32 vectors) by a two-kernel prepass.
#include <cstdint>

#include <cuda_runtime.h>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
#include "dq_row_fx.cuh"
#include "dq_internal.h"

namespace dq {

__global__ void k_state_at(DevSector S, const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                           bool use_sm) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t idx = in[t];
        if (idx >= S.D) {
            out[t] = ~0ull;
            atomicAdd(S.err, 1);
        } else {
            out[t] = d_unrank(S, off_s, str_s, idx);
        }
    }
}

__global__ void k_index_of(DevSector S, const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                           bool use_sm) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w = in[t];
        if (!d_valid(S, w)) {
            out[t] = ~0ull;
            atomicAdd(S.err, 1);
        } else {
            out[t] = d_rank(S, off_s, str_s, w);
        }
    }
}

// The same two functions for states of two words (64 < L * Nbits <= 128, or any sector through
// the two-word entry points): a state is stored as two uint64, the low word first.
__global__ void k_state_at_w(DevSector S, const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                             bool use_sm) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t idx = in[t];
        if (idx >= S.D) {
            out[2 * t] = ~0ull;
            out[2 * t + 1] = ~0ull;
            atomicAdd(S.err, 1);
        } else {
            const u128 w = d_unrank<u128>(S, off_s, str_s, idx);
            out[2 * t] = (uint64_t)w;
            out[2 * t + 1] = (uint64_t)(w >> 64);
        }
    }
}

__global__ void k_index_of_w(DevSector S, const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                             bool use_sm) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const u128 w = ((u128)in[2 * t + 1] << 64) | (u128)in[2 * t];
        if (!d_valid(S, w)) {
            out[t] = ~0ull;
            atomicAdd(S.err, 1);
        } else {
            out[t] = d_rank(S, off_s, str_s, w);
        }
    }
}

constexpr int kMaxCh = 8;  // right-hand sides handled per pass

// Row loop of the product kernels: each warp takes chunks of 32 R consecutive rows, lane l the
// rows base + l + 32 r (r < R), walked with walk_start / walk_next (one Alg. 4 unrank per chunk
// and lane, then mostly a read of the last subsystem's unrank list). The body sees the row index
// i and the walk rw (rw.s is the row's word).
#define WARP_ROWS_BEGIN(W)                                                                             \
    const uint64_t wid_ = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;                      \
    const uint64_t nwarp_ = ((uint64_t)gridDim.x * blockDim.x) >> 5;                                   \
    const uint64_t span_ = 32ull * (uint64_t)R;                                                        \
    for (uint64_t base_ = wid_ * span_; base_ < S.D; base_ += nwarp_ * span_) {                        \
        RowWalk<W> rw;                                                                                 \
        uint64_t i = base_ + (threadIdx.x & 31);                                                       \
        for (int r_ = 0; r_ < R && i < S.D; ++r_, i += 32) {                                           \
            if (r_ == 0)                                                                               \
                walk_start(S, off_s, str_s, i, rw);                                                    \
            else                                                                                       \
                walk_next(S, off_s, str_s, i, rw);
#define WARP_ROWS_END \
        }             \
    }


// y = H x, Q = 2 operator, FP64 vectors in exact fixed point (row_q2_fx). CH: right-hand
// sides per pass (1, or kMaxCh for nrhs > 1).
template <bool LIN2, int CH>
__global__ void __launch_bounds__(256)
    k_matvec_q2_fx(DevSector S, DevTermsQ2 H, const long long* __restrict__ X, double* __restrict__ y,
                   const ColScale* __restrict__ hdr, int ld, int col0, int ch, bool use_sm, int R) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    if (hdr->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += step)
            for (int c = 0; c < ch; ++c) y[i * ld + col0 + c] = __longlong_as_double(0x7ff8000000000000ll);
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    int sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sc[c] = c < ch ? H.emin - hdr->F[col0 + c] : 0;
    __shared__ uint64_t wm[kMaxLayers];
    stage_within(S, H, wm);
    WARP_ROWS_BEGIN(uint64_t)
        row_q2_fx<CH, LIN2>(S, H, off_s, str_s, wm, i, rw.s, X, ld, col0, ch, sc, y);
    WARP_ROWS_END
}

// y = H x, general-Q operator (bosons), FP64 vectors in exact fixed point: digit functions and
// n_i n_j pairs summed in int64, every allowed hop b+_a b_b a 128-bit multiply-add of its
// amplitude -t sqrt((n_a + 1) n_b) (an integer on the grid 2^emin) with the gathered X.
template <typename W, bool LIN2, int CH>
__global__ void __launch_bounds__(256)
    k_matvec_qg_fx(DevSector S, DevTermsQG H, const long long* __restrict__ X, double* __restrict__ y,
                   const ColScale* __restrict__ hdr, int ld, int col0, int ch, bool use_sm, int R) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    if (hdr->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += step)
            for (int c = 0; c < ch; ++c) y[i * ld + col0 + c] = __longlong_as_double(0x7ff8000000000000ll);
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    int sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sc[c] = c < ch ? H.emin - hdr->F[col0 + c] : 0;
    const int Q = S.Q;
    const uint32_t dm = (1u << S.nb) - 1;
    WARP_ROWS_BEGIN(W)
        const W s = rw.s;
        long long md = H.MC;
        for (int q = 0; q < H.nsite; ++q) md += __ldg(H.Msite + q * Q + (int)((uint32_t)(s >> H.site_sh[q]) & dm));
        for (int q = 0; q < H.npair; ++q) {
            const int a = (int)((uint32_t)(s >> H.pair_sh[2 * q]) & dm);
            const int b = (int)((uint32_t)(s >> H.pair_sh[2 * q + 1]) & dm);
            md += __ldg(H.Mpair + q) * (long long)(a * b);
        }
        I128 r[CH];
        const long long* Xi = X + i * ld + col0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            r[c] = {0, 0};
            if (c < ch) mac(r[c], md, __ldg(Xi + c));
        }
        for (int q = 0; q < H.nhop; ++q) {
            const int sa = H.hop_sh[2 * q], sb = H.hop_sh[2 * q + 1];
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int s_up = dir ? sb : sa, s_dn = dir ? sa : sb;  // b+_up b_dn
                const int nu = (int)((uint32_t)(s >> s_up) & dm), nd = (int)((uint32_t)(s >> s_dn) & dm);
                if (nu < Q - 1 && nd > 0) {
                    const W s2 = s + ((W)1 << s_up) - ((W)1 << s_dn);
                    const uint64_t j = LIN2 ? d_rank_lin2(S, s2) : d_rank(S, off_s, str_s, s2);
                    const long long M = __ldg(H.Mhop + ((size_t)q * Q + nu) * Q + nd);
                    const long long* Xj = X + j * ld + col0;
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (c < ch) mac(r[c], M, __ldg(Xj + c));
                }
            }
        }
        double* yi = y + i * ld + col0;
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c < ch) yi[c] = i128_to<double>(r[c], sc[c]);
    WARP_ROWS_END
}

// y = H x for FP32 vectors in fixed point (int32 X, int32 hop amplitudes, int64 hop sums, the
// diagonal on a finer int64 grid, one 128-bit combination and rounding per row): the Q = 2 form
// (row_q2_f32x) and the general-Q form.
template <bool LIN2, int CH>
__global__ void __launch_bounds__(256)
    k_matvec_q2_f32x(DevSector S, DevTermsQ2 H, const int* __restrict__ X, float* __restrict__ y,
                     const ColScale* __restrict__ hdr, int ld, int col0, int ch, bool use_sm, int R) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    if (hdr->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += step)
            for (int c = 0; c < ch; ++c) y[i * ld + col0 + c] = __int_as_float(0x7fc00000);
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    int sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sc[c] = c < ch ? H.emin32d - hdr->F[col0 + c] : 0;
    __shared__ uint64_t wm[kMaxLayers];
    stage_within(S, H, wm);
    WARP_ROWS_BEGIN(uint64_t)
        row_q2_f32x<CH, LIN2>(S, H, off_s, str_s, wm, i, rw.s, X, ld, col0, ch, sc, y);
    WARP_ROWS_END
}

template <typename W, bool LIN2, int CH>
__global__ void __launch_bounds__(256)
    k_matvec_qg_f32x(DevSector S, DevTermsQG H, const int* __restrict__ X, float* __restrict__ y,
                     const ColScale* __restrict__ hdr, int ld, int col0, int ch, bool use_sm, int R) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    if (hdr->bad) {
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += step)
            for (int c = 0; c < ch; ++c) y[i * ld + col0 + c] = __int_as_float(0x7fc00000);
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    int sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sc[c] = c < ch ? H.emin32d - hdr->F[col0 + c] : 0;
    const int Q = S.Q;
    const uint32_t dm = (1u << S.nb) - 1;
    WARP_ROWS_BEGIN(W)
        const W s = rw.s;
        long long md = H.MC32;
        for (int q = 0; q < H.nsite; ++q) md += __ldg(H.Msite32 + q * Q + (int)((uint32_t)(s >> H.site_sh[q]) & dm));
        for (int q = 0; q < H.npair; ++q) {
            const int a = (int)((uint32_t)(s >> H.pair_sh[2 * q]) & dm);
            const int b = (int)((uint32_t)(s >> H.pair_sh[2 * q + 1]) & dm);
            md += __ldg(H.Mpair32 + q) * (long long)(a * b);
        }
        long long hs[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) hs[c] = 0;
        for (int q = 0; q < H.nhop; ++q) {
            const int sa = H.hop_sh[2 * q], sb = H.hop_sh[2 * q + 1];
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int s_up = dir ? sb : sa, s_dn = dir ? sa : sb;  // b+_up b_dn
                const int nu = (int)((uint32_t)(s >> s_up) & dm), nd = (int)((uint32_t)(s >> s_dn) & dm);
                if (nu < Q - 1 && nd > 0) {
                    const W s2 = s + ((W)1 << s_up) - ((W)1 << s_dn);
                    const uint64_t j = LIN2 ? d_rank_lin2(S, s2) : d_rank(S, off_s, str_s, s2);
                    const long long M = __ldg(H.Mhop32 + ((size_t)q * Q + nu) * Q + nd);
                    const int* Xj = X + j * ld + col0;
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (c < ch) hs[c] += M * __ldg(Xj + c);
                }
            }
        }
        const int* Xi = X + i * ld + col0;
        float* yi = y + i * ld + col0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (c >= ch) continue;
            I128 r = {0, 0};
            mac(r, md, __ldg(Xi + c));
            add_i64_shl(r, hs[c], H.emin32 - H.emin32d);
            yi[c] = i128_to<float>(r, sc[c]);
        }
    WARP_ROWS_END
}

static int num_sms() { return sm_count_cached(); }

static inline size_t os_bytes(const DevSector& S) { return (size_t)S.os_total * 16; }
static inline bool os_in_smem(const DevSector& S) { return os_bytes(S) <= 48 * 1024; }

static unsigned grid_for(uint64_t n, int threads, int per_sm) {
    uint64_t need = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms() * per_sm;
    return (unsigned)(need < cap ? (need ? need : 1) : cap);
}

// Launches a grid-stride product kernel with 256 threads on as many blocks as can be resident at
// once (the occupancy calculator for this kernel's registers and this launch's dynamic shared
// memory, cached per kernel and size), capped by the row count: one wave, no tail of late blocks.
// The last kernel argument is R, the rows per lane of a warp's chunk (WARP_ROWS_BEGIN): as many
// as keep at least four chunks per warp, at most 16.
template <typename... KArgs, typename... Args>
static void launch_resident(void (*kernel)(KArgs...), uint64_t rows, size_t smb, cudaStream_t st, Args... args) {
    const int per_sm = occupancy_cached(reinterpret_cast<const void*>(kernel), 256, smb);
    const unsigned grid = grid_for(rows, 256, per_sm);
    const uint64_t lanes = (uint64_t)grid * 256;
    uint64_t R = rows / (lanes * 4);
    R = R < 1 ? 1 : (R > 16 ? 16 : R);
    kernel<<<grid, 256, smb, st>>>(args..., (int)R);
}

int launch_state_at_batch(const DevSector& S, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream) {
    bool sm = os_in_smem(S);
    k_state_at<<<grid_for(n, 256, 8), 256, sm ? os_bytes(S) : 0, (cudaStream_t)stream>>>(S, d_index, d_state, n, sm);
    return (int)cudaGetLastError();
}

int launch_index_of_batch(const DevSector& S, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream) {
    bool sm = os_in_smem(S);
    k_index_of<<<grid_for(n, 256, 8), 256, sm ? os_bytes(S) : 0, (cudaStream_t)stream>>>(S, d_state, d_index, n, sm);
    return (int)cudaGetLastError();
}

int launch_state_at_batch_w(const DevSector& S, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream) {
    bool sm = os_in_smem(S);
    k_state_at_w<<<grid_for(n, 256, 8), 256, sm ? os_bytes(S) : 0, (cudaStream_t)stream>>>(S, d_index, d_state, n, sm);
    return (int)cudaGetLastError();
}

int launch_index_of_batch_w(const DevSector& S, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream) {
    bool sm = os_in_smem(S);
    k_index_of_w<<<grid_for(n, 256, 8), 256, sm ? os_bytes(S) : 0, (cudaStream_t)stream>>>(S, d_state, d_index, n, sm);
    return (int)cudaGetLastError();
}

// FP64 vectors: column prepass into the terms' scratch, then the fixed-point kernel of the
// operator's form (Q = 2 bond layers or general Q).
static int launch_matvec_fx(const dq_sector* s, dq_terms* t, const double* x, double* y, int nrhs, cudaStream_t st) {
    const size_t need = kColScaleBytes + (size_t)s->D * nrhs * sizeof(long long);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    ColScale* h = reinterpret_cast<ColScale*>(t->scratch);
    long long* X = reinterpret_cast<long long*>(reinterpret_cast<char*>(t->scratch) + kColScaleBytes);
    launch_col_prepass<double, long long>(x, X, s->D, nrhs, h, num_sms(), st);
    const DevSector& S = s->dev;
    const bool sm = os_in_smem(S);
    const size_t smb = sm ? os_bytes(S) : 0;
    const bool lin2 = (S.n_sub == 2);
    const int tslot = timing_start(st);
    int passes = 0;
    for (int c0 = 0; c0 < nrhs; c0 += kMaxCh, ++passes) {
        const int ch = nrhs - c0 < kMaxCh ? nrhs - c0 : kMaxCh;
        if (t->q2) {
            if (nrhs == 1) {
                if (lin2)
                    launch_resident(k_matvec_q2_fx<true, 1>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
                else
                    launch_resident(k_matvec_q2_fx<false, 1>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
            } else {
                if (lin2)
                    launch_resident(k_matvec_q2_fx<true, kMaxCh>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
                else
                    launch_resident(k_matvec_q2_fx<false, kMaxCh>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
            }
        } else if (s->wide) {  // states of two words: Eq. (index) on 128-bit words
            if (nrhs == 1)
                launch_resident(k_matvec_qg_fx<u128, false, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            else
                launch_resident(k_matvec_qg_fx<u128, false, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
        } else {
            if (nrhs == 1) {
                if (lin2)
                    launch_resident(k_matvec_qg_fx<uint64_t, true, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
                else
                    launch_resident(k_matvec_qg_fx<uint64_t, false, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            } else {
                if (lin2)
                    launch_resident(k_matvec_qg_fx<uint64_t, true, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
                else
                    launch_resident(k_matvec_qg_fx<uint64_t, false, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            }
        }
    }
    timing_stop(tslot, st, 2 + passes);
    return (int)cudaGetLastError();
}

// FP32 vectors: column prepass to int32 into the terms' scratch, then the FP32 fixed-point kernel.
static int launch_matvec_f32x(const dq_sector* s, dq_terms* t, const float* x, float* y, int nrhs, cudaStream_t st) {
    const size_t need = kColScaleBytes + (size_t)s->D * nrhs * sizeof(int);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    ColScale* h = reinterpret_cast<ColScale*>(t->scratch);
    int* X = reinterpret_cast<int*>(reinterpret_cast<char*>(t->scratch) + kColScaleBytes);
    launch_col_prepass<float, int>(x, X, s->D, nrhs, h, num_sms(), st);
    const DevSector& S = s->dev;
    const bool sm = os_in_smem(S);
    const size_t smb = sm ? os_bytes(S) : 0;
    const bool lin2 = (S.n_sub == 2);
    const int tslot = timing_start(st);
    int passes = 0;
    for (int c0 = 0; c0 < nrhs; c0 += kMaxCh, ++passes) {
        const int ch = nrhs - c0 < kMaxCh ? nrhs - c0 : kMaxCh;
        const bool one = nrhs == 1;
        if (t->q2) {
            if (one && lin2) launch_resident(k_matvec_q2_f32x<true, 1>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
            else if (one) launch_resident(k_matvec_q2_f32x<false, 1>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
            else if (lin2) launch_resident(k_matvec_q2_f32x<true, kMaxCh>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
            else launch_resident(k_matvec_q2_f32x<false, kMaxCh>, S.D, smb, st, S, t->q2v, X, y, h, nrhs, c0, ch, sm);
        } else if (s->wide) {
            if (one) launch_resident(k_matvec_qg_f32x<u128, false, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            else launch_resident(k_matvec_qg_f32x<u128, false, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
        } else {
            if (one && lin2) launch_resident(k_matvec_qg_f32x<uint64_t, true, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            else if (one) launch_resident(k_matvec_qg_f32x<uint64_t, false, 1>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            else if (lin2) launch_resident(k_matvec_qg_f32x<uint64_t, true, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
            else launch_resident(k_matvec_qg_f32x<uint64_t, false, kMaxCh>, S.D, smb, st, S, t->qgv, X, y, h, nrhs, c0, ch, sm);
        }
    }
    timing_stop(tslot, st, 2 + passes);
    return (int)cudaGetLastError();
}

int launch_matvec(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (t->cluster) return launch_cluster_matvec(s, const_cast<dq_terms*>(t), x, y, dtype, nrhs, stream);
    if (t->panel_ok && nrhs == 1) return launch_panel_matvec(s, const_cast<dq_terms*>(t), x, y, dtype, stream);
    if (t->pw_ok && nrhs == 1) return launch_panel_w(s, const_cast<dq_terms*>(t), x, y, dtype, stream);
    if (t->pq_ok && nrhs == 1) return launch_panel_q(s, const_cast<dq_terms*>(t), x, y, dtype, stream);
    if (t->pb_ok && nrhs == 1) return launch_panel_pb(s, const_cast<dq_terms*>(t), x, y, dtype, stream);
    if (dtype == DQ_F64) return launch_matvec_fx(s, const_cast<dq_terms*>(t), (const double*)x, (double*)y, nrhs, st);
    return launch_matvec_f32x(s, const_cast<dq_terms*>(t), (const float*)x, (float*)y, nrhs, st);
}

}  // namespace dq

using namespace dq;

extern "C" int dq_matvec(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, int nrhs,
                         void* stream) {
    clear_error();
    if (!s || !t || !x || !y) return set_error(DQ_EINVAL, "NULL argument");
    if (t->sector != s) return set_error(DQ_EINVAL, "terms were compiled for another sector");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    if (nrhs < 1 || nrhs > 64) return set_error(DQ_EINVAL, "nrhs must be in [1, 64]");
    size_t bytes = (size_t)s->D * nrhs * (dtype == DQ_F64 ? 8 : 4);
    const char* xb = (const char*)x;
    char* yb = (char*)y;
    if (xb < yb + bytes && yb < xb + bytes) return set_error(DQ_EINVAL, "x and y overlap");
    int e = launch_matvec(s, t, x, y, dtype, nrhs, stream);
    if (e) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}
