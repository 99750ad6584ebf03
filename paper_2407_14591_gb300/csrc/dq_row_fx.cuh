// The row computations of the general Q = 2 product kernels in exact fixed point (FP64 vectors
// with int64 x and 128-bit rows, FP32 vectors with int32 x and int64 hop sums), and the walk over
// a bond layer's active pairs with the rank form each pair needs.
#pragma once

#include <cstdint>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

// Per layer l, the low positions p of the pairs (p, p + dist_l) that lie inside one subsystem,
// written by each block into shared memory (nl <= kMaxLayers words). Only partitions of three or
// more subsystems use them: with one or two subsystems (Lin's two tables) the full rank costs no
// more lookups than the incremental one, and every mask is left empty.
__device__ __forceinline__ void stage_within(const DevSector& S, const DevTermsQ2& H, uint64_t* wm) {
    for (int l = threadIdx.x; l < H.nl; l += blockDim.x) {
        const int d = H.dist[l];
        uint64_t w = 0;
        if (S.n_sub >= 3)
            for (uint64_t m = H.omask[l]; m; m &= m - 1) {
                const int p = __ffsll((long long)m) - 1;
                if (p + d < 64 && S.sub_of[p] == S.sub_of[p + d]) w |= 1ull << p;
            }
        wm[l] = w;
    }
    __syncthreads();
}

// Calls f(j, p) for every active pair of one layer of row i (word s): o = the active low
// positions, ow = those whose pair lies inside one subsystem, pm = the pair's two bits at p = 0.
// A pair inside subsystem k changes only c_k (Sec. 3.2), so its rank is incremental
// (d_rank_within: one rank-table lookup per side); the other pairs take the full Eq. (index)
// (or Lin's two tables). The two kinds run as two loops rather than a branch per pair, so that
// the lanes of a warp take the same rank form at the same time.
template <bool LIN2, typename F>
__device__ __forceinline__ void for_each_hop(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s,
                                             uint64_t i, uint64_t s, uint64_t o, uint64_t ow, uint64_t pm, F&& f) {
    if (!LIN2) {
        for (uint64_t m = ow; m; m &= m - 1) {
            const int p = __ffsll((long long)m) - 1;
            f(d_rank_within(S, str_s, i, s, s ^ (pm << p), S.sub_of[p]), p);
        }
        o ^= ow;
    }
    for (uint64_t m = o; m; m &= m - 1) {
        const int p = __ffsll((long long)m) - 1;
        const uint64_t w2 = s ^ (pm << p);
        f(LIN2 ? d_rank_lin2(S, w2) : d_rank(S, off_s, str_s, w2), p);
    }
}

// Row i (word s) of y = H x: X holds x as int64 (row-major, ld values per row, columns col0 .. col0+ch-1
// used), the coefficients are integers times 2^emin (DevTermsQ2), sc[c] = emin - F of column
// col0 + c. The diagonal is an int64 sum; every row result is a 128-bit sum rounded once.
// Layers with one hop amplitude add their gathered X in int64 and multiply once.
template <int CH, bool LIN2>
__device__ __forceinline__ void row_q2_fx(const DevSector& S, const DevTermsQ2& H, const uint64_t* off_s,
                                          const uint64_t* str_s, const uint64_t* wm, uint64_t i, uint64_t s,
                                          const long long* __restrict__ X, int ld, int col0, int ch, const int* sc,
                                          double* __restrict__ y) {
    long long md = H.MC;
    if (H.Mlin) {
        uint64_t m = s;
        while (m) {
            const int p = __ffsll((long long)m) - 1;
            m &= m - 1;
            md += __ldg(H.Mlin + p);
        }
    }
    for (int l = 0; l < H.nl; ++l) {
        uint64_t a = (s ^ (s >> H.dist[l])) & H.dmask[l];
        if (H.kpos[l] < 0) {
            md += __ldg(H.MKA + l) * (long long)__popcll(a);
        } else {
            while (a) {
                const int p = __ffsll((long long)a) - 1;
                a &= a - 1;
                md += __ldg(H.Mpos + H.kpos[l] + p);
            }
        }
    }
    I128 r[CH];
    const long long* Xi = X + i * ld + col0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        r[c] = {0, 0};
        if (c < ch) mac(r[c], md, __ldg(Xi + c));
    }
    for (int l = 0; l < H.nl; ++l) {
        const uint64_t o = (s ^ (s >> H.dist[l])) & H.omask[l];
        if (!o) continue;
        const uint64_t pm = 1ull | (1ull << H.dist[l]);
        const uint64_t ow = LIN2 ? 0ull : (o & wm[l]);
        if (H.apos[l] < 0) {
            long long sum[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) sum[c] = 0;
            for_each_hop<LIN2>(S, off_s, str_s, i, s, o, ow, pm, [&](uint64_t j, int) {
                const long long* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) sum[c] += __ldg(Xj + c);
            });
            const long long MA = __ldg(H.MKA + kMaxLayers + l);
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (c < ch) mac(r[c], MA, sum[c]);
        } else {
            const long long* Mp = H.Mpos + H.apos[l];
            for_each_hop<LIN2>(S, off_s, str_s, i, s, o, ow, pm, [&](uint64_t j, int p) {
                const long long M = __ldg(Mp + p);
                const long long* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) mac(r[c], M, __ldg(Xj + c));
            });
        }
    }
    double* yi = y + i * ld + col0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
        if (c < ch) yi[c] = i128_to<double>(r[c], sc[c]);
}

// Adds v * 2^sh (v an int64, 0 <= sh <= 60) to the 128-bit a.
__device__ __forceinline__ void add_i64_shl(I128& a, long long v, int sh) {
    const unsigned long long vlo = (unsigned long long)v << sh;
    const long long vhi = sh ? (v >> (64 - sh)) : (v < 0 ? -1ll : 0ll);
    const unsigned long long lo = a.lo + vlo;
    a.hi += vhi + (lo < a.lo ? 1ll : 0ll);
    a.lo = lo;
}

// Row i (word s) of y = H x for FP32 vectors in fixed point: X holds x as int32 (|X| < 2^30); hop
// amplitudes are int32 multiples of 2^emin32 (|m| < 2^24, fewer bits for rows with very many
// hops), so every hop is one 32x32 -> 64-bit product added to an int64 row sum (the host keeps
// max_hops * 2^(bits + 30) below 2^62); diagonal coefficients are int64 multiples of the finer
// 2^emin32d. The row is (diagonal X_i) + (hop sum << (emin32 - emin32d)) in 128 bits, rounded
// once to FP32 with sc = emin32d - F.
template <int CH, bool LIN2>
__device__ __forceinline__ void row_q2_f32x(const DevSector& S, const DevTermsQ2& H, const uint64_t* off_s,
                                            const uint64_t* str_s, const uint64_t* wm, uint64_t i, uint64_t s,
                                            const int* __restrict__ X, int ld, int col0, int ch, const int* sc,
                                            float* __restrict__ y) {
    long long md = H.MC32;
    if (H.Mlin32) {
        uint64_t m = s;
        while (m) {
            const int p = __ffsll((long long)m) - 1;
            m &= m - 1;
            md += __ldg(H.Mlin32 + p);
        }
    }
    for (int l = 0; l < H.nl; ++l) {
        uint64_t a = (s ^ (s >> H.dist[l])) & H.dmask[l];
        if (H.kpos[l] < 0) {
            md += (long long)__ldg(H.MKA32 + l) * (long long)__popcll(a);
        } else {
            while (a) {
                const int p = __ffsll((long long)a) - 1;
                a &= a - 1;
                md += __ldg(H.Mpos32 + H.kpos[l] + p);
            }
        }
    }
    long long hs[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) hs[c] = 0;
    for (int l = 0; l < H.nl; ++l) {
        const uint64_t o = (s ^ (s >> H.dist[l])) & H.omask[l];
        if (!o) continue;
        const uint64_t pm = 1ull | (1ull << H.dist[l]);
        const uint64_t ow = LIN2 ? 0ull : (o & wm[l]);
        if (H.apos[l] < 0) {
            long long sum[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) sum[c] = 0;
            for_each_hop<LIN2>(S, off_s, str_s, i, s, o, ow, pm, [&](uint64_t j, int) {
                const int* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) sum[c] += __ldg(Xj + c);
            });
            const long long MA = __ldg(H.MKA32 + kMaxLayers + l);
#pragma unroll
            for (int c = 0; c < CH; ++c) hs[c] += MA * sum[c];
        } else {
            const long long* Mp = H.Mpos32 + H.apos[l];
            for_each_hop<LIN2>(S, off_s, str_s, i, s, o, ow, pm, [&](uint64_t j, int p) {
                const long long M = __ldg(Mp + p);
                const int* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) hs[c] += M * __ldg(Xj + c);
            });
        }
    }
    const int* Xi = X + i * ld + col0;
    float* yi = y + i * ld + col0;
    const int sh = H.emin32 - H.emin32d;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        if (c >= ch) continue;
        I128 r = {0, 0};
        mac(r, md, __ldg(Xi + c));
        add_i64_shl(r, hs[c], sh);
        yi[c] = i128_to<float>(r, sc[c]);
    }
}

}  // namespace dq
