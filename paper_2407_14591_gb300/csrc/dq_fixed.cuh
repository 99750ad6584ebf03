// Exact fixed-point arithmetic shared by the product kernels.
//
// FP64 work runs at a small fraction of the integer rate on this GPU, so the FP64 products are
// exact integer sums: x is scaled by 2^F (F from the largest exponent of its column) and rounded
// to int64 with |X| < 2^56 (FP64 input) or to int32 with |X| < 2^30 (FP32 input); the
// coefficients are integers M times 2^e; every row result is formed in 128-bit integers and
// rounded once (ties to even) to the output type.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace dq {

template <typename T>
struct FBits;
template <>
struct FBits<double> {
    using U = unsigned long long;
    static constexpr int MB = 52, EMASK = 0x7ff, BIAS = 1023;
};
template <>
struct FBits<float> {
    using U = unsigned int;
    static constexpr int MB = 23, EMASK = 0xff, BIAS = 127;
};
template <typename XT>
struct XHead;
template <>
struct XHead<long long> {
    static constexpr int HEAD = 56;  // |X| <= 2^56: 64 terms still fit in int64
};
template <>
struct XHead<int> {
    static constexpr int HEAD = 30;
};

// Biased exponent field of one element's bits.
template <typename T>
__device__ __forceinline__ int exp_field(typename FBits<T>::U b) {
    return (int)((b >> FBits<T>::MB) & FBits<T>::EMASK);
}

// x scaled by 2^F and rounded to the integer type XT (round half away from zero).
template <typename T, typename XT>
__device__ __forceinline__ XT to_fixed(typename FBits<T>::U b, int F) {
    using U = typename FBits<T>::U;
    constexpr int MB = FBits<T>::MB, BIAS = FBits<T>::BIAS;
    const int e = exp_field<T>(b);
    unsigned long long m = (unsigned long long)(b & (((U)1 << MB) - 1));
    int ue;
    if (e) {
        m |= 1ull << MB;
        ue = e - BIAS - MB;
    } else {
        ue = 1 - BIAS - MB;
    }
    const int sh = ue + F;  // X = m 2^sh
    unsigned long long v;
    if (sh >= 0)
        v = m << sh;
    else if (sh > -62)
        v = (m + (1ull << (-sh - 1))) >> (-sh);
    else
        v = 0;
    const long long sv = (b >> (sizeof(U) * 8 - 1)) ? -(long long)v : (long long)v;
    return (XT)sv;
}

// ------------------------------------------------------------------ 128-bit helpers ---------

struct I128 {
    long long hi;
    unsigned long long lo;
};

__device__ __forceinline__ void mac(I128& a, long long u, long long v) {
    unsigned long long plo = (unsigned long long)u * (unsigned long long)v;
    long long phi = __mul64hi(u, v);
    unsigned long long lo = a.lo + plo;
    a.hi += phi + (lo < a.lo ? 1 : 0);
    a.lo = lo;
}

// Round the integer a * 2^scale to the nearest double / float (ties to even).
template <typename OUT>
__device__ __forceinline__ OUT i128_to(I128 a, int scale) {
    constexpr int P = sizeof(OUT) == 8 ? 53 : 24;  // mantissa bits
    constexpr int BIAS = sizeof(OUT) == 8 ? 1023 : 127;
    constexpr int EMAXB = sizeof(OUT) == 8 ? 2047 : 255;
    bool neg = a.hi < 0;
    unsigned long long hi = (unsigned long long)a.hi, lo = a.lo;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0 ? 1ull : 0ull);
    }
    if (hi == 0 && lo == 0) return (OUT)0;
    int lz = hi ? __clzll(hi) : 64 + __clzll(lo);
    if (lz >= 64) {
        hi = lo << (lz - 64);
        lo = 0;
    } else if (lz > 0) {
        hi = (hi << lz) | (lo >> (64 - lz));
        lo <<= lz;
    }
    // leading bit at 127 of (hi:lo); keep P bits
    unsigned long long m = hi >> (64 - P);
    unsigned long long rest = hi << P;  // bits below the mantissa in hi, left-aligned
    bool guard = (rest >> 63) & 1ull;
    bool sticky = ((rest << 1) != 0) || lo != 0;
    int e2 = (127 - lz) + scale;  // exponent of the leading bit
    if (guard && (sticky || (m & 1ull))) {
        ++m;
        if (m >> P) {
            m >>= 1;
            ++e2;
        }
    }
    int be = e2 + BIAS;
    if (be <= 0) return neg ? -(OUT)0 : (OUT)0;  // below the normal range (not reached for sane x)
    if (be >= EMAXB) return neg ? -(OUT)INFINITY : (OUT)INFINITY;
    if (sizeof(OUT) == 8) {
        unsigned long long bits =
            ((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1));
        return (OUT)__longlong_as_double((long long)bits);
    } else {
        unsigned int bits = ((unsigned int)neg << 31) | ((unsigned int)be << 23) | (unsigned int)(m & ((1u << 23) - 1));
        return (OUT)__int_as_float((int)bits);
    }
}

// ------------------------------------------------------------------ per-column prepass -------

// Scales of an interleaved block of nrhs <= 64 columns (x[i * nrhs + c]).
constexpr int kMaxCols = 64;
struct ColScale {
    int emax[kMaxCols];  // largest biased exponent of each column
    int F[kMaxCols];     // scale exponent of each column: X = round(x 2^F)
    int bad;             // some column held an Inf or NaN
};
constexpr size_t kColScaleBytes = 1024;  // header size in the scratch area (>= sizeof(ColScale))
static_assert(sizeof(ColScale) <= kColScaleBytes, "column header");

// Threads per block of the column prepass: a multiple of ld, so with a grid-stride loop every
// thread stays on one column.
__host__ __device__ inline int col_block(int ld) { return (256 / ld) * ld; }

template <typename T>
__global__ void k_col_exp_max(const T* __restrict__ x, uint64_t n, int ld, ColScale* h) {
    using U = typename FBits<T>::U;
    __shared__ int m_s[kMaxCols];
    for (int c = threadIdx.x; c < ld; c += blockDim.x) m_s[c] = 0;
    __syncthreads();
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    int m = 0;
    for (uint64_t i = t0; i < n; i += step) m = max(m, exp_field<T>(reinterpret_cast<const U*>(x)[i]));
    if (m) atomicMax(&m_s[(int)(t0 % (uint64_t)ld)], m);
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x)
        if (m_s[c]) atomicMax(&h->emax[c], m_s[c]);
}

template <typename T, typename XT>
__global__ void k_col_to_fixed(const T* __restrict__ x, XT* __restrict__ X, uint64_t n, int ld, ColScale* h) {
    using U = typename FBits<T>::U;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    const int c = (int)(t0 % (uint64_t)ld);
    const int emax = h->emax[c];
    const int F = XHead<XT>::HEAD - (emax - FBits<T>::BIAS + 1);  // |x| < 2^(emax - BIAS + 1)
    if (t0 < (uint64_t)ld) {
        h->F[c] = F;
        if (emax == FBits<T>::EMASK) h->bad = 1;  // Inf or NaN in column c
    }
    if (emax == FBits<T>::EMASK) return;
    for (uint64_t i = t0; i < n; i += step) X[i] = to_fixed<T, XT>(reinterpret_cast<const U*>(x)[i], F);
}

// Host side: the prepass of `rows` rows of `ld` interleaved columns into X, with the header at h.
template <typename T, typename XT>
inline void launch_col_prepass(const T* x, XT* X, uint64_t rows, int ld, ColScale* h, int sms, cudaStream_t st) {
    cudaMemsetAsync(h, 0, sizeof(ColScale), st);
    const int bs = col_block(ld);
    const uint64_t n = rows * (uint64_t)ld;
    uint64_t want = (n + bs - 1) / bs;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 8 ? (want ? want : 1) : (uint64_t)sms * 8);
    k_col_exp_max<T><<<grid, bs, 0, st>>>(x, n, ld, h);
    k_col_to_fixed<T, XT><<<grid, bs, 0, st>>>(x, X, n, ld, h);
}


// ------------------------------------------------------------------ one-column prepass -------

// Scratch of the panel products: this header (first 256 bytes), then X = round(x 2^F).
// Workspace header (first 256 bytes of the scratch area).
struct WsHeader {
    int emax;  // largest biased exponent in x
    int F;     // scale exponent: X = round(x 2^F)
    int bad;   // x held an Inf or NaN
};

// Largest biased exponent in x. 16-byte loads when x is 16-byte aligned (the usual case).
template <typename T>
__global__ void k_exp_max(const T* __restrict__ x, uint64_t n, WsHeader* h) {
    using U = typename FBits<T>::U;
    constexpr int V = 16 / sizeof(T);
    int m = 0;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const uint4* xv = reinterpret_cast<const uint4*>(x);
        const uint64_t nv = n / V;
        for (uint64_t i = t0; i < nv; i += step) {
            const uint4 q = __ldg(xv + i);
            if (sizeof(T) == 8) {  // the exponent sits in the high word of each double
                m = max(m, (int)((q.y >> 20) & 0x7ffu));
                m = max(m, (int)((q.w >> 20) & 0x7ffu));
            } else {
                m = max(m, (int)((q.x >> 23) & 0xffu));
                m = max(m, (int)((q.y >> 23) & 0xffu));
                m = max(m, (int)((q.z >> 23) & 0xffu));
                m = max(m, (int)((q.w >> 23) & 0xffu));
            }
        }
        head = nv * V;
    }
    for (uint64_t i = head + t0; i < n; i += step) m = max(m, exp_field<T>(reinterpret_cast<const U*>(x)[i]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&h->emax, m);
}

// X = round(x 2^F) with F chosen from the largest exponent so that |X| < 2^HEAD. 16-byte loads
// and stores when x is 16-byte aligned (X always is).
template <typename T, typename XT>
__global__ void k_to_fixed(const T* __restrict__ x, XT* __restrict__ X, uint64_t n, WsHeader* h) {
    using U = typename FBits<T>::U;
    constexpr int BIAS = FBits<T>::BIAS;
    const int emax = h->emax;
    if (emax == FBits<T>::EMASK) {  // Inf or NaN in x
        if (blockIdx.x == 0 && threadIdx.x == 0) h->bad = 1;
        return;
    }
    // |x| < 2^(emax - BIAS + 1), so X = x 2^F stays below 2^HEAD
    const int F = XHead<XT>::HEAD - (emax - BIAS + 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) h->F = F;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0 && sizeof(XT) == sizeof(T)) {
        // one 16-byte load of x and one 16-byte store of X per step
        constexpr int V = 16 / sizeof(T);
        const uint64_t nv = n / V;
        for (uint64_t i = t0; i < nv; i += step) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(x) + i);
            uint4 r;
            if (sizeof(T) == 8) {
                const unsigned long long v0 =
                    (unsigned long long)to_fixed<T, XT>((U)(((unsigned long long)q.y << 32) | q.x), F);
                const unsigned long long v1 =
                    (unsigned long long)to_fixed<T, XT>((U)(((unsigned long long)q.w << 32) | q.z), F);
                r = make_uint4((unsigned)v0, (unsigned)(v0 >> 32), (unsigned)v1, (unsigned)(v1 >> 32));
            } else {
                r = make_uint4((unsigned)to_fixed<T, XT>((U)q.x, F), (unsigned)to_fixed<T, XT>((U)q.y, F),
                               (unsigned)to_fixed<T, XT>((U)q.z, F), (unsigned)to_fixed<T, XT>((U)q.w, F));
            }
            reinterpret_cast<uint4*>(X)[i] = r;
        }
        head = nv * V;
    }
    for (uint64_t i = head + t0; i < n; i += step) X[i] = to_fixed<T, XT>(reinterpret_cast<const U*>(x)[i], F);
}


}  // namespace dq
