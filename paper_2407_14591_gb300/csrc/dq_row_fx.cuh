// The row computation of the Q = 2 product for FP64 vectors in exact fixed point, shared by the
// single-sector and the batched kernels.
#pragma once

#include <cstdint>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

// Rank of a hopped word of row i (word s) for the Q = 2 kernels; flip = the two bits of the pair
// (positions p and p + d). Lin's two tables (LIN2) and partitions of up to three subsystems use the
// full rank. With four or more subsystems a pair inside one subsystem takes the incremental rank
// (d_rank_within: one lookup per side instead of one per subsystem); measured on the 6x5 J1-J2
// lattice it is 13 % faster with five subsystems and slower with two or three, where the extra
// branch (lanes walk different pairs) and lookups cost more than they save.
template <bool LIN2>
__device__ __forceinline__ uint64_t hop_rank(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s,
                                             uint64_t i, uint64_t s, uint64_t flip, int p, int d) {
    if (LIN2) return d_rank_lin2(S, s ^ flip);
    if (S.n_sub >= 4) {
        const int ka = S.sub_of[p];
        if (ka == S.sub_of[p + d]) return d_rank_within(S, str_s, i, s, s ^ flip, ka);
    }
    return d_rank(S, off_s, str_s, s ^ flip);
}

// Row i of y = H x: X holds x as int64 (row-major, ld values per row, columns col0 .. col0+ch-1
// used), the coefficients are integers times 2^emin (DevTermsQ2), sc[c] = emin - F of column
// col0 + c. The diagonal is an int64 sum; every row result is a 128-bit sum rounded once.
// Layers with one hop amplitude add their gathered X in int64 and multiply once.
template <int CH, bool LIN2>
__device__ __forceinline__ void row_q2_fx(const DevSector& S, const DevTermsQ2& H, const uint64_t* off_s,
                                          const uint64_t* str_s, uint64_t i, const long long* __restrict__ X, int ld,
                                          int col0, int ch, const int* sc, double* __restrict__ y) {
    const uint64_t s = d_unrank(S, off_s, str_s, i);
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
        uint64_t o = (s ^ (s >> H.dist[l])) & H.omask[l];
        if (!o) continue;
        const uint64_t pm = 1ull | (1ull << H.dist[l]);
        if (H.apos[l] < 0) {
            long long sum[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) sum[c] = 0;
            while (o) {
                const int p = __ffsll((long long)o) - 1;
                o &= o - 1;
                const uint64_t j = hop_rank<LIN2>(S, off_s, str_s, i, s, pm << p, p, H.dist[l]);
                const long long* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) sum[c] += __ldg(Xj + c);
            }
            const long long MA = __ldg(H.MKA + kMaxLayers + l);
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (c < ch) mac(r[c], MA, sum[c]);
        } else {
            while (o) {
                const int p = __ffsll((long long)o) - 1;
                o &= o - 1;
                const uint64_t j = hop_rank<LIN2>(S, off_s, str_s, i, s, pm << p, p, H.dist[l]);
                const long long M = __ldg(H.Mpos + H.apos[l] + p);
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
}

// Adds v * 2^sh (v an int64, 0 <= sh <= 60) to the 128-bit a.
__device__ __forceinline__ void add_i64_shl(I128& a, long long v, int sh) {
    const unsigned long long vlo = (unsigned long long)v << sh;
    const long long vhi = sh ? (v >> (64 - sh)) : (v < 0 ? -1ll : 0ll);
    const unsigned long long lo = a.lo + vlo;
    a.hi += vhi + (lo < a.lo ? 1ll : 0ll);
    a.lo = lo;
}

// Row i of y = H x for FP32 vectors in fixed point: X holds x as int32 (|X| < 2^30); hop
// amplitudes are int32 multiples of 2^emin32 (|m| < 2^24, fewer bits for rows with very many
// hops), so every hop is one 32x32 -> 64-bit product added to an int64 row sum (the host keeps
// max_hops * 2^(bits + 30) below 2^62); diagonal coefficients are int64 multiples of the finer
// 2^emin32d. The row is (diagonal X_i) + (hop sum << (emin32 - emin32d)) in 128 bits, rounded
// once to FP32 with sc = emin32d - F.
template <int CH, bool LIN2>
__device__ __forceinline__ void row_q2_f32x(const DevSector& S, const DevTermsQ2& H, const uint64_t* off_s,
                                            const uint64_t* str_s, uint64_t i, const int* __restrict__ X, int ld,
                                            int col0, int ch, const int* sc, float* __restrict__ y) {
    const uint64_t s = d_unrank(S, off_s, str_s, i);
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
        uint64_t o = (s ^ (s >> H.dist[l])) & H.omask[l];
        if (!o) continue;
        const uint64_t pm = 1ull | (1ull << H.dist[l]);
        if (H.apos[l] < 0) {
            long long sum[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) sum[c] = 0;
            while (o) {
                const int p = __ffsll((long long)o) - 1;
                o &= o - 1;
                const uint64_t j = hop_rank<LIN2>(S, off_s, str_s, i, s, pm << p, p, H.dist[l]);
                const int* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) sum[c] += __ldg(Xj + c);
            }
            const long long MA = __ldg(H.MKA32 + kMaxLayers + l);
#pragma unroll
            for (int c = 0; c < CH; ++c) hs[c] += MA * sum[c];
        } else {
            while (o) {
                const int p = __ffsll((long long)o) - 1;
                o &= o - 1;
                const uint64_t j = hop_rank<LIN2>(S, off_s, str_s, i, s, pm << p, p, H.dist[l]);
                const long long M = __ldg(H.Mpos32 + H.apos[l] + p);
                const int* Xj = X + j * ld + col0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c < ch) hs[c] += M * __ldg(Xj + c);
            }
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
