// Device helpers shared by the product kernels: Eq. (index) (Alg. 2) and Alg. 4 on the device.
#pragma once

#include <cstdint>

#include "dq_internal.h"

namespace dq {

__device__ __forceinline__ int digit_sum(uint32_t f, int nb) {
    switch (nb) {
        case 1: return __popc(f);
        case 2: return __popc(f & 0x55555555u) + 2 * __popc(f & 0xAAAAAAAAu);
        case 3: return __popc(f & 0x49249249u) + 2 * __popc(f & 0x92492492u) + 4 * __popc(f & 0x24924924u);
        default:
            return __popc(f & 0x11111111u) + 2 * __popc(f & 0x22222222u) + 4 * __popc(f & 0x44444444u) +
                   8 * __popc(f & 0x88888888u);
    }
}

// Word types of a basis state: one 64-bit word (L * Nbits <= 64) or a 128-bit pair of words
// (64 < L * Nbits <= 128). The helpers below are templates over the word type; every shift
// count is below the word's width.
using u128 = unsigned __int128;

template <typename W>
__device__ __forceinline__ uint32_t field_of(const DevSector& S, W w, int k) {
    return (uint32_t)(w >> S.shift[k]) & (uint32_t)((1ull << (S.nb * S.Lk[k])) - 1);
}

// Eq. (index) for a valid state. off_s / str_s may live in shared or global memory.
// Checked builds (-DDQ_CHECKED): a rank at or beyond D raises the sector's error word and is
// replaced by 0, so the gather that follows stays inside x. Normal builds compile this away.
__device__ __forceinline__ uint64_t checked_rank(const DevSector& S, uint64_t j) {
#ifdef DQ_CHECKED
    if (j >= S.D) {
        atomicAdd(S.err, 1);
        return 0;
    }
#endif
    return j;
}

template <typename W>
__device__ __forceinline__ uint64_t d_rank(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s, W w) {
    uint64_t idx = 0;
    int lam = 0;
    for (int k = 0; k < S.n_sub; ++k) {
        uint32_t f = field_of(S, w, k);
        uint32_t li = __ldg(S.rank_tab[S.tab[k]] + f);
        int n = digit_sum(f, S.nb);
        int o = S.os_base[k] + lam * S.os_ld[k] + n;
        idx += off_s[o] + str_s[o] * (uint64_t)li;
        lam += n;
    }
    return checked_rank(S, idx);
}

// Lin's two-table form (Sec. 3.3): index = c_0(sigma^(0)) + index_1(sigma^(1)).
template <typename W>
__device__ __forceinline__ uint64_t d_rank_lin2(const DevSector& S, W w) {
    uint32_t f0 = (uint32_t)(w >> S.shift[0]);
    uint32_t f1 = (uint32_t)w & (uint32_t)((1ull << (S.nb * S.Lk[1])) - 1);
    return checked_rank(S, __ldg(S.c0_tab + f0) + (uint64_t)__ldg(S.rank_tab[S.tab[1]] + f1));
}

// Incremental rank (Sec. 3.2): a change of the word inside one subsystem k keeps every n_l and
// lambda_l, so only c_k = offset_k + stride_k index_k changes and the new index is
// i + stride_k (index_k(f') - index_k(f)): one table lookup per side instead of a full Eq. (index).
// Q = 2 only (lambda_k is the popcount of the bits above P_k). w: the row's word, i its index,
// w2: the word after the change.
__device__ __forceinline__ uint64_t d_rank_within(const DevSector& S, const uint64_t* str_s, uint64_t i, uint64_t w,
                                                  uint64_t w2, int k) {
    const uint32_t f = field_of(S, w, k), f2 = field_of(S, w2, k);
    const uint32_t* rt = S.rank_tab[S.tab[k]];
    const int top = S.shift[k] + S.Lk[k];
    const int lam = top >= 64 ? 0 : __popcll(w >> top);
    const uint64_t st = str_s[S.os_base[k] + lam * S.os_ld[k] + __popc(f)];
    const long long delta = (long long)__ldg(rt + f2) - (long long)__ldg(rt + f);
    return checked_rank(S, i + (uint64_t)((long long)st * delta));
}

// Alg. 4 for idx < D.
template <typename W = uint64_t>
__device__ __forceinline__ W d_unrank(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s, uint64_t idx) {
    W w = 0;
    int lam = 0;
    for (int k = 0; k < S.n_sub; ++k) {
        int base = S.os_base[k] + lam * S.os_ld[k];
        int n;
        uint64_t li;
        if (k == S.n_sub - 1) {
            n = S.N - lam;
            li = idx;  // offset 0, stride 1 for the last subsystem
            idx = 0;
        } else {
            n = 0;
            while (n < S.nmax[k] && !(idx < off_s[base + n + 1])) ++n;
            idx -= off_s[base + n];
            uint64_t st = str_s[base + n];
            li = idx / st;
            idx -= li * st;
        }
        int t = S.tab[k];
        uint32_t pat = __ldg(S.unrank_tab[t] + __ldg(S.sec_start[t] + n) + li);
        w |= (W)pat << S.shift[k];
        lam += n;
    }
    return w;
}

// Walk of one lane over the rows i, i + 32, i + 64, ... of a warp (the lanes take consecutive
// rows, so loads and stores stay coalesced). The first row is unranked with Alg. 4. The last
// subsystem has offset 0 and stride 1 in Eq. (index), so consecutive indices run through its
// particle-number sector in its local order: while the last subsystem's local index plus 32 stays
// inside that sector, the next row differs from this one only in the last subsystem's pattern,
// read from the unrank list (Alg. 3 applied 32 times at once); otherwise Alg. 4 again.
template <typename W>
struct RowWalk {
    W s;                   // the row's word
    uint32_t li, len;      // local index of the last subsystem, size of its sector
    const uint32_t* list;  // unrank list of that sector
};

template <typename W>
__device__ __forceinline__ void walk_start(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s,
                                           uint64_t idx, RowWalk<W>& r) {
    W w = 0;
    int lam = 0;
    const int last = S.n_sub - 1;
    for (int k = 0; k < last; ++k) {
        const int base = S.os_base[k] + lam * S.os_ld[k];
        int n = 0;
        while (n < S.nmax[k] && !(idx < off_s[base + n + 1])) ++n;
        idx -= off_s[base + n];
        const uint64_t st = str_s[base + n];
        const uint64_t li = idx / st;
        idx -= li * st;
        const int t = S.tab[k];
        w |= (W)__ldg(S.unrank_tab[t] + __ldg(S.sec_start[t] + n) + li) << S.shift[k];
        lam += n;
    }
    const int t = S.tab[last], n = S.N - lam;
    const uint32_t s0 = __ldg(S.sec_start[t] + n);
    r.list = S.unrank_tab[t] + s0;
    r.len = __ldg(S.sec_start[t] + n + 1) - s0;
    r.li = (uint32_t)idx;
    r.s = w | (W)__ldg(r.list + r.li);  // the last subsystem sits at shift 0
}

template <typename W>
__device__ __forceinline__ void walk_next(const DevSector& S, const uint64_t* off_s, const uint64_t* str_s,
                                          uint64_t idx, RowWalk<W>& r) {
    if (r.li + 32 < r.len) {
        r.li += 32;
        const W lowmask = ((W)1 << (S.nb * S.Lk[S.n_sub - 1])) - 1;
        r.s = (r.s & ~lowmask) | (W)__ldg(r.list + r.li);
    } else {
        walk_start(S, off_s, str_s, idx, r);
    }
}

__device__ __forceinline__ int popc_w(uint64_t v) { return __popcll(v); }
__device__ __forceinline__ int popc_w(u128 v) { return __popcll((uint64_t)v) + __popcll((uint64_t)(v >> 64)); }

template <typename W>
__device__ __forceinline__ bool d_valid(const DevSector& S, W w) {
    constexpr int WB = 8 * (int)sizeof(W);
    int bits = S.L * S.nb;
    if (bits < WB && (w >> bits) != 0) return false;
    if ((S.Q & (S.Q - 1)) == 0) {
        // Q = 2^Nbits: every digit is < Q; the digit sum is a weighted popcount of bit planes
        int n = 0;
        for (int b = 0; b < S.nb; ++b) {
            W plane = 0;
            for (int q = b; q < WB; q += S.nb) plane |= (W)1 << q;
            n += popc_w(w & plane) << b;
        }
        return n == S.N;
    }
    int n = 0;
    unsigned m = (1u << S.nb) - 1;
    for (int i = 0; i < S.L; ++i) {
        int d = (int)((uint32_t)(w >> (S.nb * i)) & m);
        if (d >= S.Q) return false;
        n += d;
    }
    return n == S.N;
}

// Stage the offset / stride tables in shared memory when they fit.
__device__ __forceinline__ void stage_os(const DevSector& S, uint64_t* sm, bool use, const uint64_t*& off_s,
                                         const uint64_t*& str_s) {
    if (use) {
        for (int q = threadIdx.x; q < S.os_total; q += blockDim.x) {
            sm[q] = S.off[q];
            sm[S.os_total + q] = S.str[q];
        }
        __syncthreads();
        off_s = sm;
        str_s = sm + S.os_total;
    } else {
        off_s = S.off;
        str_s = S.str;
    }
}


// Row accumulator: plain FP64 for FP64 vectors; for FP32 vectors FP32 products summed with
// Neumaier's compensated summation (the running error term keeps each row sum within about one
// FP32 rounding of its exact value, however many terms it has).
template <typename T>
struct RowAcc;
template <>
struct RowAcc<double> {
    double s;
    __device__ __forceinline__ void init(double v) { s = v; }
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct RowAcc<float> {
    float s, c;
    __device__ __forceinline__ void init(float v) {
        s = v;
        c = 0.f;
    }
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ float get() const { return s + c; }
};

}  // namespace dq
