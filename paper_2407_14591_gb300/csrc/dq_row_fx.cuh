// The row computation of the Q = 2 product for FP64 vectors in exact fixed point, shared by the
// single-sector and the batched kernels.
#pragma once

#include <cstdint>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

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
                const uint64_t j = LIN2 ? d_rank_lin2(S, s ^ (pm << p)) : d_rank(S, off_s, str_s, s ^ (pm << p));
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
                const uint64_t j = LIN2 ? d_rank_lin2(S, s ^ (pm << p)) : d_rank(S, off_s, str_s, s ^ (pm << p));
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

}  // namespace dq
