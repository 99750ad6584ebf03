// Lanczos driver for the ground-state energy (Sec. 4.4; App. D calls a native Lanczos): the
// only use of H is the matrix-free product. The tridiagonal matrix T is solved on the host by
// bisection on its Sturm sequence, and the Ritz vector's coefficients by inverse iteration (own
// implementations).
//
// One step is two launches: the product w = H v_k, then one cooperative kernel (k_lz_step, all
// blocks resident, grid-wide barriers between its phases) that does the rest on the device:
//   alpha_k = <v_k, w>;  r = w - alpha_k v_k - beta_{k-1} v_{k-1}         (rho0 = ||r||^2)
//   with re-orthogonalisation, classical Gram-Schmidt of r against V = [v_0 .. v_k]:
//     h = V^T r; r -= V h; alpha_k += h_k                                  (rho1 = ||r||^2)
//     a second pass only if rho1 < rho0 / 2 (the DGKS criterion; always with reorth = 2)
//   beta_k = ||r||; v_{k+1} = r / beta_k.
// The three-term remainder is formed inside the first tile of the projection pass (from w, v_k
// and v_{k-1}), so it costs no pass of its own. Gram-Schmidt acts on that remainder, not on w:
// applied to w itself, one pass would multiply the basis's loss of orthogonality by
// ||w|| / beta_k at every step.
// Partial sums are reduced in a fixed order (the result does not depend on timing); every block
// derives the same coefficients. alpha_k and beta_k^2 go to device arrays and to mapped pinned
// host memory. The host reads step k's values only after it has queued step k+2, so the GPU
// never waits for the host; a breakdown found late only costs the steps already queued, whose
// results are dropped.
//
// Arithmetic. FP64 runs on this GPU at a small fraction of its FP32 rate, and a pass over V does
// (k + 1) multiply-adds per element, so the passes over V use double-single arithmetic: a value
// is an unevaluated sum of two floats (hi, lo). Products are error-free in their leading part
// (p = a*b and its exact error fma(a, b, -p)), sums use Knuth's TwoSum, and the compensation
// terms are summed in FP32 and folded into a second float pair every kFlush terms: the dot
// product scheme Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005), which returns
// the result as if computed with 48-bit significands and rounded once. Block partials are
// combined in FP64. The basis of FP64 vectors is stored as float pairs (48 significant bits);
// the vector the next product reads is their sum in FP64. FP32 vectors are stored as floats and
// the residual r is kept as a float pair inside a step. Conversions between double and float
// pairs use integer bit operations (no FP64 instruction).

#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

constexpr int kRedThreads = 256;
constexpr int kDotTile = 16;  // basis vectors per pass of the blocked dot kernel
constexpr int kLzThreads = 512;  // threads of a step-kernel block
constexpr int kLzTile = 8;       // basis vectors per tile of the projection pass (one warp each)
constexpr int kFlush = 32;       // terms summed into a float pair before it is folded into the next

// Sum of v over the block; the total is returned in thread 0 only (sh: 32 doubles).
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Called by every block after it wrote its partial result(s): returns true in the one block that
// arrives last (which then sees every block's partials), and resets the counter for the next use.
__device__ __forceinline__ bool last_block(unsigned* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
        if (last) *counter = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// out[j] = <V_j, w> for j < k, V_j = V + j * ldv. Each pass takes kDotTile vectors at once (w is
// read once per tile) over the block's grid-stride rows; partial[b * k + j] holds block b's sums
// and the last block adds them in block order. With `gate` (non-NULL) the kernel does nothing
// unless *gate != 0.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gs_dots(const T* __restrict__ V, size_t ldv, int k,
                                                          const T* __restrict__ w, uint64_t n,
                                                          double* __restrict__ partial, double* __restrict__ out,
                                                          unsigned* counter, const double* gate) {
    if (gate && *gate == 0.0) return;
    __shared__ double sh[kDotTile][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (int j0 = 0; j0 < k; j0 += kDotTile) {
        const int nj = k - j0 < kDotTile ? k - j0 : kDotTile;
        double acc[kDotTile];
#pragma unroll
        for (int q = 0; q < kDotTile; ++q) acc[q] = 0.0;
        const T* Vb = V + (size_t)j0 * ldv;
        if (nj == kDotTile) {
            for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += step) {
                const double wi = (double)w[i];
#pragma unroll
                for (int q = 0; q < kDotTile; ++q) acc[q] += (double)__ldg(Vb + (size_t)q * ldv + i) * wi;
            }
        } else {
            for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += step) {
                const double wi = (double)w[i];
#pragma unroll
                for (int q = 0; q < kDotTile; ++q)
                    if (q < nj) acc[q] += (double)__ldg(Vb + (size_t)q * ldv + i) * wi;
            }
        }
#pragma unroll
        for (int q = 0; q < kDotTile; ++q) {
            double v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[q][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double s = 0.0;
            for (int r = 0; r < kRedThreads / 32; ++r) s += sh[threadIdx.x][r];
            partial[(size_t)blockIdx.x * k + j0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
    if (last_block(counter))
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            double s = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partial + (size_t)b * k + j);
            out[j] = s;
        }
}

// Exact widening of a float to double with integer operations only (the hardware conversion runs
// on the FP64 pipe, and a branch to it would be compiled as a select that always executes it).
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) {  // Inf, NaN
        bits = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (e != 0u) {
        bits = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {
        bits = sign;
    } else {  // subnormal m * 2^-149, leading bit of m at position p: exponent p - 149
        const int p = 31 - __clz(m);
        bits = sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

constexpr unsigned kBarrierLimit = 1u << 24;  // polls of a grid barrier before it gives up

// Grid-wide barrier of a cooperative launch (every block resident): a counter of arrivals and a
// generation word. A block waits at most kBarrierLimit polls; on timeout it raises *fail, and
// every later barrier returns false at once, so the kernel ends with the error recorded.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* fail) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        volatile int* vf = fail;
        ok = !*vf;
        if (ok) {
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0u;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                unsigned it = 0;
                while (*gen == g && !*vf && it < kBarrierLimit) {
                    __nanosleep(64);
                    ++it;
                }
                if (*gen == g) {
                    *vf = 1;
                    ok = 0;
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    return ok != 0;
}

// Sum of part[0 .. nb) in a fixed order, returned to every thread of the block (sh: at least 33
// doubles); every block gets the same value.
__device__ __forceinline__ double reduce_all(const double* part, int nb, double* sh) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += __ldcg(part + b);
    acc = block_sum(acc, sh);  // the total is in thread 0
    if (threadIdx.x == 0) sh[32] = acc;
    __syncthreads();
    acc = sh[32];
    __syncthreads();
    return acc;
}

// ---- double-single arithmetic ---------------------------------------------------------------
// A pair (S, C) stands for S + C. Every operation uses the _rn intrinsics, which the compiler
// never contracts into fused multiply-adds, so each error-free transformation stays exact.

// (S, C) += p: TwoSum gives S + p = s + err exactly; err joins the compensation C.
__device__ __forceinline__ void ff_add(float& S, float& C, float p) {
    const float s = __fadd_rn(S, p);
    const float bp = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    S = s;
    C = __fadd_rn(C, err);
}

// (S, C) += (s, c)
__device__ __forceinline__ void ff_fold(float& S, float& C, float s, float c) {
    ff_add(S, C, s);
    C = __fadd_rn(C, c);
}

// (S, C) += (ah + al)(bh + bl): ah*bh = p + e exactly (e by a fused multiply-add), the cross
// terms join e; al*bl lies below the pair's precision and is dropped.
__device__ __forceinline__ void ff_mac(float& S, float& C, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    ff_add(S, C, p);
    C = __fadd_rn(C, e);
}

// (S, C) += (h + l)^2
__device__ __forceinline__ void ff_sq(float& S, float& C, float h, float l) {
    const float p = __fmul_rn(h, h);
    float e = __fmaf_rn(h, h, -p);
    e = __fmaf_rn(__fadd_rn(h, h), l, e);
    ff_add(S, C, p);
    C = __fadd_rn(C, e);
}

// (rh, rl) = (ah + al) - (bh + bl), renormalised so that |rl| <= ulp(rh) / 2.
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float& rh, float& rl) {
    const float s = __fsub_rn(ah, bh);
    const float bp = __fsub_rn(s, ah);
    const float err = __fsub_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fadd_rn(bh, bp));  // s + err = ah - bh
    const float t = __fadd_rn(err, __fsub_rn(al, bl));
    rh = __fadd_rn(s, t);
    rl = __fsub_rn(t, __fsub_rn(rh, s));
}

// (vh, vl) = (rh + rl)(sh + sl), renormalised.
__device__ __forceinline__ void ff_mul(float rh, float rl, float sh, float sl, float& vh, float& vl) {
    const float p = __fmul_rn(rh, sh);
    float e = __fmaf_rn(rh, sh, -p);
    e = __fmaf_rn(rh, sl, e);
    e = __fmaf_rn(rl, sh, e);
    vh = __fadd_rn(p, e);
    vl = __fsub_rn(e, __fsub_rn(vh, p));
}

// x = hi + lo with hi = x cut to 24 significant bits and lo the remainder rounded to FP32 (48
// significant bits together), by integer operations only. Magnitudes below 2^-126 become zero,
// and below 2^-74 lo is dropped (it would not be a normal float); Inf and NaN give hi = x, lo = 0;
// finite |x| >= 2^128 gives an infinite hi.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if (e >= 897u && e <= 1150u) {
        hi = __uint_as_float(sign | ((e - 896u) << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
        const float scale = __uint_as_float(sign | ((e >= 949u ? e - 948u : 0u) << 23));  // +-2^(e - 1075)
        lo = e >= 949u ? __fmul_rn(__uint2float_rn((unsigned)b & 0x1fffffffu), scale) : 0.f;
    } else if (e < 897u) {
        hi = __uint_as_float(sign);
        lo = 0.f;
    } else {
        const bool nan = e == 0x7ffu && (b & 0xfffffffffffffull) != 0ull;
        hi = __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
        lo = 0.f;
    }
}

// ---- the arithmetic of the passes over the basis ---------------------------------------------
// A policy fixes how an element is held in registers (E), how sums run (Sum), and the basis
// element type S for vectors of type T; a pass loads the raw basis elements (Raw) of a tile or
// round first and converts them afterwards, so that all its loads are in flight together (FP32
// vectors with FP64 passes: a workload-2 pass 1.4x faster than with the conversion behind each
// load).
//   LzF64: FP64 elements and sums (fused multiply-adds on the FP64 pipe); the basis in T.
//   LzDS: double-single elements and sums (above); the basis of FP64 vectors as float pairs,
//         of FP32 vectors as floats.

template <typename T>
struct LzF64 {
    using S = T;
    using E = double;
    struct Sum {
        double s;
    };
    static constexpr bool kXBuffer = false;  // the product reads v_k from the basis itself
    using Raw = T;  // a basis element as loaded, before the conversion to E
    __device__ static Raw ld_raw(const T* p) { return __ldg(p); }
    __device__ static E cvt(Raw r) { return widen(r); }
    __device__ static E ld_basis(const T* p) { return widen(__ldg(p)); }
    __device__ static E ld_w(const T* p) { return widen(__ldg(p)); }
    __device__ static Sum zero() { return {0.0}; }
    __device__ static void mac(Sum& a, E x, E y) { a.s = fma(x, y, a.s); }
    __device__ static void sq(Sum& a, E x) { a.s = fma(x, x, a.s); }
    __device__ static void fold(Sum& a, Sum b) { a.s += b.s; }
    __device__ static Sum shfl_down(Sum a, int o) { return {__shfl_down_sync(0xffffffffu, a.s, o)}; }
    __device__ static double value(Sum a) { return a.s; }
    __device__ static Sum from_double(double x) { return {x}; }
    __device__ static E coef(double c) { return c; }
    __device__ static E sub(E r, Sum a) { return r - a.s; }
    __device__ static E mul(E r, E c) { return r * c; }
    __device__ static void st_basis(T* p, double*, E v) { *p = (T)v; }
    __device__ static void st_out(T* p, Sum a) { *p = (T)a.s; }
};

template <typename T>
struct LzDSBasis;
template <>
struct LzDSBasis<double> {
    using S = float2;
};
template <>
struct LzDSBasis<float> {
    using S = float;
};

template <typename T>
struct LzDS {
    using S = typename LzDSBasis<T>::S;
    using E = float2;
    struct Sum {
        float s, c;
    };
    static constexpr bool kXBuffer = sizeof(T) == 8;  // FP64 vectors: the product reads an FP64 copy
    using Raw = S;
    __device__ static Raw ld_raw(const S* p) { return __ldg(p); }
    __device__ static E cvt(float2 r) { return r; }
    __device__ static E cvt(float r) { return make_float2(r, 0.f); }
    __device__ static E ld_basis(const float2* p) { return __ldg(p); }
    __device__ static E ld_basis(const float* p) { return make_float2(__ldg(p), 0.f); }
    __device__ static E ld_w(const double* p) {
        float h, l;
        split_f64(__ldg(p), h, l);
        return make_float2(h, l);
    }
    __device__ static E ld_w(const float* p) { return make_float2(__ldg(p), 0.f); }
    __device__ static Sum zero() { return {0.f, 0.f}; }
    __device__ static void mac(Sum& a, E x, E y) { ff_mac(a.s, a.c, x.x, x.y, y.x, y.y); }
    __device__ static void sq(Sum& a, E x) { ff_sq(a.s, a.c, x.x, x.y); }
    __device__ static void fold(Sum& a, Sum b) { ff_fold(a.s, a.c, b.s, b.c); }
    __device__ static Sum shfl_down(Sum a, int o) {
        return {__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.c, o)};
    }
    __device__ static double value(Sum a) { return widen(a.s) + widen(a.c); }
    __device__ static Sum from_double(double x) {
        Sum a;
        split_f64(x, a.s, a.c);
        return a;
    }
    __device__ static E coef(double c) {
        float h, l;
        split_f64(c, h, l);
        return make_float2(h, l);
    }
    __device__ static E sub(E r, Sum a) {
        float h, l;
        ff_sub(r.x, r.y, a.s, a.c, h, l);
        return make_float2(h, l);
    }
    __device__ static E mul(E r, E c) {
        float h, l;
        ff_mul(r.x, r.y, c.x, c.y, h, l);
        return make_float2(h, l);
    }
    __device__ static void st_basis(float2* p, double* x, E v) {
        *p = v;
        *x = widen(v.x) + widen(v.y);
    }
    __device__ static void st_basis(float* p, double*, E v) { *p = __fadd_rn(v.x, v.y); }
    __device__ static void st_out(double* p, Sum a) { *p = widen(a.s) + widen(a.c); }
    __device__ static void st_out(float* p, Sum a) { *p = __fadd_rn(a.s, a.c); }
};

template <class P>
__device__ __forceinline__ typename P::Sum warp_sum(typename P::Sum a) {
    for (int o = 16; o > 0; o >>= 1) P::fold(a, P::shfl_down(a, o));
    return a;
}

// Sum over the block, in FP64 in thread 0 (sh: 32 sums).
template <class P>
__device__ __forceinline__ double block_total(typename P::Sum a, typename P::Sum* sh) {
    a = warp_sum<P>(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        typename P::Sum b = lane < (int)(blockDim.x >> 5) ? sh[lane] : P::zero();
        r = P::value(warp_sum<P>(b));
    }
    __syncthreads();
    return r;
}

// Sum of the FP64 block partials part[0 .. nb) in a fixed order, returned to every thread of the
// block; every block gets the same value.
template <class P>
__device__ __forceinline__ double lz_reduce_all(const double* part, int nb, typename P::Sum* sh, double* bc) {
    typename P::Sum a = P::zero();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) P::fold(a, P::from_double(__ldcg(part + b)));
    const double v = block_total<P>(a, sh);
    if (threadIdx.x == 0) *bc = v;
    __syncthreads();
    const double r = *bc;
    __syncthreads();
    return r;
}

template <typename T, class P>
struct LzStep {
    using S = typename P::S;
    using E = typename P::E;
    const S* V;       // basis v_0 .. v_k, stride ldv
    size_t ldv;
    int k;            // step index
    const T* w;       // H v_k (the product's output)
    E* r;             // the residual
    S* vnext;         // v_{k+1} in the basis (NULL at the last step)
    double* xnext;    // v_{k+1} in FP64 for the next product (double-single, FP64 vectors)
    uint64_t n;
    int reorth;       // 0, 1 (DGKS second pass), 2 (second pass always)
    double* part;     // per-block partial sums, gridDim.x * (k + 5) doubles
    double* h;        // projection coefficients, k + 1 doubles
    double* alpha;    // alpha_j, beta_j^2 of every step (device)
    double* beta2;
    volatile double* host;  // mapped pinned host memory: alpha_k, beta_k^2 at [2k], [2k+1]
    unsigned* bar;    // grid barrier (two words)
    int* fail;        // barrier timeout
};

// alpha pass: the block partial of <v_k, w> into pa[b]; w is also stored as the residual r.
// Two elements per iteration, so that each thread has four loads in flight.
template <typename T, class P>
__device__ bool lz_alpha(const LzStep<T, P>& a, const typename P::S* vk, double* pa, typename P::Sum* sh) {
    using Sum = typename P::Sum;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    Sum s1 = P::zero(), s2 = P::zero();
    int cnt = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += 2 * stride) {
        const uint64_t i2 = i + stride;
        const bool two = i2 < a.n;
        const typename P::E w1 = P::ld_w(a.w + i), v1 = P::ld_basis(vk + i);
        const typename P::E w2 = two ? P::ld_w(a.w + i2) : w1, v2 = two ? P::ld_basis(vk + i2) : v1;
        a.r[i] = w1;
        P::mac(s1, v1, w1);
        if (two) {
            a.r[i2] = w2;
            P::mac(s1, v2, w2);
        }
        if (++cnt == kFlush / 2) {
            cnt = 0;
            P::fold(s2, s1);
            s1 = P::zero();
        }
    }
    P::fold(s2, s1);
    const double v = block_total<P>(s2, sh);
    if (threadIdx.x == 0) pa[blockIdx.x] = v;
    return grid_sync(a.bar, a.fail);
}

// The block's slab of elements for the projection: [lo, hi), contiguous, a multiple of 32 long.
__device__ __forceinline__ void lz_slab(uint64_t n, uint64_t& lo, uint64_t& hi) {
    const uint64_t per = ((n + gridDim.x - 1) / gridDim.x + 31) & ~(uint64_t)31;
    lo = per * blockIdx.x;
    hi = lo + per < n ? lo + per : n;
    if (lo > n) lo = n;
}

// Projection pass: block partials pd[b * (k + 1) + j] of h_j = <v_j, r> for j <= k. Block b owns
// a contiguous slab of elements; its warps share the basis vectors in tiles of kLzTile (warp w
// takes tiles w, w + 16, ...), each lane summing its strided elements of the slab (folded every
// kFlush elements into a second sum kept in shared memory, fls, so that registers stay few), and
// a shuffle tree gives the warp's partial for each vector of the tile. No block barrier inside
// the tiles, so they proceed side by side; with fewer tiles than warps, several warps share a
// tile (wp: their sums). first: before the tiles, the block replaces r (holding w) on its slab by
// the three-term remainder r - alpha v_k - beta v_{k-1} and puts ||r||^2 into pw[b].
template <typename T, class P>
__device__ bool lz_project(const LzStep<T, P>& a, typename P::E al, typename P::E be, bool first, double* pd,
                           double* pw, typename P::Sum* sh, typename P::Sum* wp, typename P::Sum* fls) {
    using S = typename P::S;
    using E = typename P::E;
    using Sum = typename P::Sum;
    const int nj = a.k + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t lo, hi;
    lz_slab(a.n, lo, hi);
    if (first) {
        const S* vk = a.V + (size_t)a.k * a.ldv;
        const S* vp = a.k ? vk - a.ldv : nullptr;
        Sum n1 = P::zero(), n2 = P::zero();
        int cnt = 0;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            Sum t = P::zero();
            P::mac(t, P::ld_basis(vk + i), al);
            if (vp) P::mac(t, P::ld_basis(vp + i), be);
            const E w = P::sub(a.r[i], t);
            a.r[i] = w;
            P::sq(n1, w);
            if (++cnt == kFlush) {
                cnt = 0;
                P::fold(n2, n1);
                n1 = P::zero();
            }
        }
        P::fold(n2, n1);
        const double v = block_total<P>(n2, sh);  // also orders the writes to r above
        if (threadIdx.x == 0) pw[blockIdx.x] = v;
    }
    // P warps per tile when there are fewer tiles than warps (each takes every Pw-th 32-element
    // chunk of the slab; their sums are combined through shared memory in part order)
    const int ntile = (nj + kLzTile - 1) / kLzTile;
    const int Pw = ntile >= nw ? 1 : nw / ntile;
    const int part = wid % Pw;
    for (int t0 = (wid / Pw) * kLzTile; t0 < nj; t0 += (nw / Pw) * kLzTile) {
        const int nt = nj - t0 < kLzTile ? nj - t0 : kLzTile;
        const S* Vb = a.V + (size_t)t0 * a.ldv;
        Sum s1[kLzTile];
        Sum* fl = fls + wid * kLzTile * 32 + lane;  // this lane's second-level sums
#pragma unroll
        for (int q = 0; q < kLzTile; ++q) {
            s1[q] = P::zero();
            fl[q * 32] = P::zero();
        }
        int cnt = 0;
        for (uint64_t i = lo + 32 * part + lane; i < hi; i += 32 * Pw) {
            const E rv = a.r[i];
            typename P::Raw v[kLzTile];  // all loads of the tile first, then the conversions
#pragma unroll
            for (int q = 0; q < kLzTile; ++q) {
                v[q] = typename P::Raw{};
                if (q < nt) v[q] = P::ld_raw(Vb + (size_t)q * a.ldv + i);
            }
#pragma unroll
            for (int q = 0; q < kLzTile; ++q) P::mac(s1[q], P::cvt(v[q]), rv);
            if (++cnt == kFlush) {
                cnt = 0;
#pragma unroll
                for (int q = 0; q < kLzTile; ++q) {
                    Sum m = fl[q * 32];
                    P::fold(m, s1[q]);
                    fl[q * 32] = m;
                    s1[q] = P::zero();
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kLzTile; ++q) {
            Sum m = fl[q * 32];
            P::fold(m, s1[q]);
            m = warp_sum<P>(m);
            if (lane == 0 && q < nt) {
                if (Pw == 1)
                    pd[(size_t)blockIdx.x * nj + t0 + q] = P::value(m);
                else
                    wp[wid * kLzTile + q] = m;
            }
        }
    }
    if (Pw > 1) {
        __syncthreads();
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            const int w0 = (j / kLzTile) * Pw, q = j % kLzTile;
            Sum m = P::zero();
            for (int p = 0; p < Pw; ++p) P::fold(m, wp[(w0 + p) * kLzTile + q]);
            pd[(size_t)blockIdx.x * nj + j] = P::value(m);
        }
    }
    return grid_sync(a.bar, a.fail);
}

// h_j for j <= k from the block partials: one warp per vector sums the blocks' partials in a
// fixed order (lane l takes blocks l, l + 32, ..., then a shuffle tree). With at most as many
// vectors as a block has warps every block does this for all of them into hd (no grid barrier);
// otherwise the warps of the grid share the vectors, write a.h, and after a barrier each block
// copies a.h into hd. Either way every block holds the same values.
template <typename T, class P>
__device__ bool lz_reduce(const LzStep<T, P>& a, const double* pd, double* hd) {
    const int nj = a.k + 1, nb = gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto column = [&](int j) {
        typename P::Sum m = P::zero();
        for (int b = lane; b < nb; b += 32) P::fold(m, P::from_double(__ldcg(pd + (size_t)b * nj + j)));
        return P::value(warp_sum<P>(m));
    };
    if (nj <= nw) {
        if (wid < nj) {
            const double v = column(wid);
            if (lane == 0) hd[wid] = v;
        }
        __syncthreads();
        return true;
    }
    for (int j = blockIdx.x * nw + wid; j < nj; j += nb * nw) {
        const double v = column(j);
        if (lane == 0) a.h[j] = v;
    }
    if (!grid_sync(a.bar, a.fail)) return false;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) hd[j] = __ldcg(a.h + j);
    __syncthreads();
    return true;
}

// Update pass: r -= sum_{j in [u0, k]} c_j v_j over the thread's elements (coefficients in cf),
// kG basis loads in flight per round (padded rounds load zeros) and two independent sums over j,
// folded into one every 4 kFlush terms; then the block partial of ||r||^2 into pr[b].
template <typename T, class P>
__device__ bool lz_update(const LzStep<T, P>& a, int u0, const typename P::E* cf, double* pr,
                          typename P::Sum* sh) {
    using E = typename P::E;
    using Sum = typename P::Sum;
    constexpr int kG = 10;  // loads per round (registers)
    const int kk = a.k + 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    Sum n1 = P::zero(), n2 = P::zero();
    int cnt = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += stride) {
        Sum s0 = P::zero(), s1 = P::zero(), fs = P::zero();
        for (int j0 = u0; j0 < kk; j0 += 4 * kFlush) {
            const int je = kk - j0 < 4 * kFlush ? kk : j0 + 4 * kFlush;
            for (int j = j0; j < je; j += kG) {
                typename P::Raw v[kG];  // all loads of the round first, then the conversions
#pragma unroll
                for (int q = 0; q < kG; ++q) {
                    v[q] = typename P::Raw{};
                    if (j + q < je) v[q] = P::ld_raw(a.V + (size_t)(j + q) * a.ldv + i);
                }
                // a padded term multiplies a zero by the last (finite) coefficient
#pragma unroll
                for (int q = 0; q < kG; q += 2) {
                    P::mac(s0, P::cvt(v[q]), cf[j + q < je ? j + q : je - 1]);
                    P::mac(s1, P::cvt(v[q + 1]), cf[j + q + 1 < je ? j + q + 1 : je - 1]);
                }
            }
            P::fold(fs, s0);
            P::fold(fs, s1);
            s0 = s1 = P::zero();
        }
        const E rn = P::sub(a.r[i], fs);
        a.r[i] = rn;
        P::sq(n1, rn);
        if (++cnt == kFlush) {
            cnt = 0;
            P::fold(n2, n1);
            n1 = P::zero();
        }
    }
    P::fold(n2, n1);
    const double v = block_total<P>(n2, sh);
    if (threadIdx.x == 0) pr[blockIdx.x] = v;
    return grid_sync(a.bar, a.fail);
}

// One Lanczos step after the product (see the file comment). Cooperative launch; dynamic shared
// memory: k + 1 doubles (the coefficients) and k + 1 elements E (the coefficients converted).
template <typename T, class P>
__global__ void __launch_bounds__(kLzThreads, 2) k_lz_step(LzStep<T, P> a) {
    using E = typename P::E;
    using Sum = typename P::Sum;
    extern __shared__ __align__(16) unsigned char lz_smem[];
    double* hd = reinterpret_cast<double*>(lz_smem);
    E* cf = reinterpret_cast<E*>(hd + a.k + 1);
    __shared__ Sum sh[32];
    __shared__ double bcast;
    __shared__ Sum wp[kLzThreads / 32 * kLzTile];        // the projection's per-warp sums
    __shared__ Sum fls[kLzThreads / 32 * kLzTile * 32];  // its per-lane second-level sums
    const int nb = gridDim.x, kk = a.k + 1;
    double* pa = a.part;   // <v_k, w>
    double* pw = pa + nb;  // ||r||^2 after the three-term step
    double* pr1 = pw + nb; // after the first Gram-Schmidt pass (or the three-term update)
    double* pr2 = pr1 + nb;
    double* pd = pr2 + nb; // projection partials, nb * (k + 1)
    if (!lz_alpha(a, a.V + (size_t)a.k * a.ldv, pa, sh)) return;
    double al = lz_reduce_all<P>(pa, nb, sh, &bcast);
    const double be = a.k ? sqrt(__ldcg(a.beta2 + a.k - 1)) : 0.0;
    double b2;
    if (!a.reorth) {  // r -= alpha_k v_k + beta_{k-1} v_{k-1}
        if (threadIdx.x < 2 && (threadIdx.x == 0 || a.k)) cf[a.k - threadIdx.x] = P::coef(threadIdx.x ? be : al);
        __syncthreads();
        if (!lz_update(a, a.k ? a.k - 1 : 0, cf, pr1, sh)) return;
        b2 = lz_reduce_all<P>(pr1, nb, sh, &bcast);
    } else {
        const E ale = P::coef(al), bee = P::coef(be);
        if (!lz_project(a, ale, bee, true, pd, pw, sh, wp, fls)) return;
        if (!lz_reduce(a, pd, hd)) return;
        al += hd[a.k];
        for (int j = threadIdx.x; j < kk; j += blockDim.x) cf[j] = P::coef(hd[j]);
        __syncthreads();
        if (!lz_update(a, 0, cf, pr1, sh)) return;
        b2 = lz_reduce_all<P>(pr1, nb, sh, &bcast);
        const double rho0 = lz_reduce_all<P>(pw, nb, sh, &bcast);
        if (a.reorth == 2 || b2 < 0.5 * rho0) {
            if (!lz_project(a, ale, bee, false, pd, nullptr, sh, wp, fls)) return;
            if (!lz_reduce(a, pd, hd)) return;
            al += hd[a.k];
            for (int j = threadIdx.x; j < kk; j += blockDim.x) cf[j] = P::coef(hd[j]);
            __syncthreads();
            if (!lz_update(a, 0, cf, pr2, sh)) return;
            b2 = lz_reduce_all<P>(pr2, nb, sh, &bcast);
        }
    }
    // beta_k, v_{k+1}
    if (a.vnext) {
        const E sc = P::coef(b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0);
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += 2 * stride) {
            const uint64_t i2 = i + stride;
            const E r1 = a.r[i];
            const E r2 = i2 < a.n ? a.r[i2] : r1;
            P::st_basis(a.vnext + i, a.xnext + i, P::mul(r1, sc));
            if (i2 < a.n) P::st_basis(a.vnext + i2, a.xnext + i2, P::mul(r2, sc));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.alpha[a.k] = al;
        a.beta2[a.k] = b2;
        a.host[2 * a.k] = al;
        a.host[2 * a.k + 1] = b2;
        __threadfence_system();
    }
}

// v_0 = v0 / sqrt(*nrm2) into the basis (and, with an FP64 copy, into the product input x0).
template <typename T, class P>
__global__ void k_lz_start(typename P::S* V0, double* x0, const T* __restrict__ v0, const double* __restrict__ nrm2,
                           uint64_t n) {
    const double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        P::st_basis(V0 + i, x0 + i, P::coef(s * widen(v0[i])));
}

// psi[i] = sum_{j<m} c[j] v_j[i] (c converted in shared memory).
template <typename T, class P>
__global__ void k_combination(T* __restrict__ psi, const typename P::S* V, size_t ldv, int m,
                              const double* __restrict__ c, uint64_t n) {
    using E = typename P::E;
    extern __shared__ __align__(16) unsigned char cmb_smem[];
    E* cs = reinterpret_cast<E*>(cmb_smem);
    for (int q = threadIdx.x; q < m; q += blockDim.x) cs[q] = P::coef(c[q]);
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        typename P::Sum s1 = P::zero(), s2 = P::zero();
        for (int j = 0; j < m; ++j) {
            P::mac(s1, P::ld_basis(V + (size_t)j * ldv + i), cs[j]);
            if ((j + 1) % kFlush == 0) {
                P::fold(s2, s1);
                s1 = P::zero();
            }
        }
        P::fold(s2, s1);
        P::st_out(psi + i, s2);
    }
}

// Number of eigenvalues of the symmetric tridiagonal T (diagonal a, off-diagonal b) below x.
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        double bb = i ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest eigenvalue of T by bisection inside its Gershgorin interval.
double tridiag_min_eig(const std::vector<double>& a, const std::vector<double>& b) {
    size_t m = a.size();
    double lo = a[0], hi = a[0];
    for (size_t i = 0; i < m; ++i) {
        double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::fmin(lo, a[i] - r);
        hi = std::fmax(hi, a[i] + r);
    }
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, mid) >= 1)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Unit eigenvector of T for the eigenvalue lam by inverse iteration: three solves of
// (T - lam I) z = z_prev with Gaussian elimination and partial pivoting on the tridiagonal
// system (a zero pivot is replaced by a tiny one, the usual device for a shift that is an
// eigenvalue to working precision).
static std::vector<double> tridiag_eigvec(const std::vector<double>& a, const std::vector<double>& b, double lam) {
    const size_t m = a.size();
    std::vector<double> z(m, 1.0 / std::sqrt((double)m));
    if (m == 1) return {1.0};
    double tn = 0.0;
    for (size_t i = 0; i < m; ++i) tn = std::fmax(tn, std::fabs(a[i]) + (i + 1 < m ? std::fabs(b[i]) : 0.0));
    const double eps = (tn > 0.0 ? tn : 1.0) * 2.2e-16;  // stands in for an exactly zero pivot
    for (int it = 0; it < 3; ++it) {
        // rows of the banded LU: d (diagonal), du (first superdiagonal), du2 (second, from pivoting)
        std::vector<double> d(m), du(m, 0.0), du2(m, 0.0), dl(m, 0.0), rhs = z;
        for (size_t i = 0; i < m; ++i) d[i] = a[i] - lam;
        for (size_t i = 0; i + 1 < m; ++i) {
            du[i] = b[i];
            dl[i] = b[i];
        }
        for (size_t i = 0; i + 1 < m; ++i) {
            if (std::fabs(d[i]) >= std::fabs(dl[i])) {
                if (d[i] == 0.0) d[i] = eps;
                const double f = dl[i] / d[i];
                d[i + 1] -= f * du[i];
                rhs[i + 1] -= f * rhs[i];
                dl[i] = 0.0;
            } else {  // swap rows i and i + 1
                const double f = d[i] / dl[i];
                d[i] = dl[i];
                const double t = d[i + 1];
                d[i + 1] = du[i] - f * t;
                du[i] = t;
                if (i + 2 < m) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du2[i];
                }
                std::swap(rhs[i], rhs[i + 1]);
                rhs[i + 1] -= f * rhs[i];
            }
        }
        if (d[m - 1] == 0.0) d[m - 1] = eps;
        z[m - 1] = rhs[m - 1] / d[m - 1];
        z[m - 2] = (rhs[m - 2] - du[m - 2] * z[m - 1]) / d[m - 2];
        for (size_t q = m - 2; q-- > 0;) z[q] = (rhs[q] - du[q] * z[q + 1] - du2[q] * z[q + 2]) / d[q];
        double nz = 0.0;
        for (double v : z) nz += v * v;
        nz = std::sqrt(nz);
        if (!(nz > 0.0) || !std::isfinite(nz)) break;
        for (double& v : z) v /= nz;
    }
    // sign convention: the largest component positive
    size_t imax = 0;
    for (size_t i = 1; i < m; ++i)
        if (std::fabs(z[i]) > std::fabs(z[imax])) imax = i;
    if (z[imax] < 0.0)
        for (double& v : z) v = -v;
    return z;
}

struct Work {
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;
    std::vector<cudaEvent_t> events;
    ~Work() {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (void* p : host_allocs) cudaFreeHost(p);
        for (void* p : allocs) cudaFree(p);
    }
    void* get(size_t bytes, int& rc) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            rc = set_error(DQ_ENOMEM, "Lanczos workspace cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    }
    void* get_host(size_t bytes, int& rc) {
        void* p = nullptr;
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e != cudaSuccess) {
            rc = set_error(DQ_ENOMEM, "Lanczos cudaMallocHost(%zu): %s", bytes, cudaGetErrorString(e));
            return nullptr;
        }
        host_allocs.push_back(p);
        return p;
    }
};

template <typename T, class P>
static int run_lanczos(const dq_sector* s, const dq_terms* t, const T* v0, int steps, int reorth, double* E0,
                       double* alpha_out, double* beta_out, int* steps_done, T* psi, cudaStream_t st) {
    using S = typename P::S;
    using E = typename P::E;
    const uint64_t D = s->D;
    const size_t ldv = (D + 31) & ~(size_t)31;
    const int sms = sm_count_cached();
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return set_error(DQ_ECUDA, "Lanczos: the device does not support cooperative launches");
    const size_t smem_max = (size_t)(steps + 1) * (sizeof(double) + sizeof(E));
    auto kern = k_lz_step<T, P>;
    if (smem_max > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) != cudaSuccess)
        return set_error(DQ_ECUDA, "Lanczos: shared memory for %d coefficients", steps + 1);
    int per_sm = occupancy_cached(reinterpret_cast<const void*>(kern), kLzThreads, smem_max);
    // blocks per SM: two, or one for sectors below 4 M elements (fewer arrivals at each grid
    // barrier and fewer partials to reduce; FP32 vectors with FP64 passes are the exception, they
    // measured faster with two)
    const int per_sm_max = D < (1ull << 22) && !std::is_same<P, LzF64<float>>::value ? 1 : 2;
    if (per_sm > per_sm_max) per_sm = per_sm_max;
    if (per_sm < 1) return set_error(DQ_ECUDA, "Lanczos: the step kernel does not fit on an SM");
    const int nb = per_sm * sms;  // blocks of the cooperative step kernel (all resident)
    const int nbd = 2 * sms;      // blocks of the start-vector reduction
    int rc = DQ_OK;
    Work ws;
    S* V = (S*)ws.get((size_t)(steps + 1) * ldv * sizeof(S), rc);
    if (!V) return rc;
    T* w = (T*)ws.get(ldv * sizeof(T), rc);
    if (!w) return rc;
    E* r = (E*)ws.get(ldv * sizeof(E), rc);
    if (!r) return rc;
    double* x = nullptr;  // v_k in FP64, the product's input, when the basis holds float pairs
    if (P::kXBuffer && !(x = (double*)ws.get(ldv * sizeof(double), rc))) return rc;
    const size_t npart = (size_t)nb * (steps + 4) > (size_t)nbd ? (size_t)nb * (steps + 4) : (size_t)nbd;
    double* part = (double*)ws.get(npart * sizeof(double), rc);
    if (!part) return rc;
    // device doubles: h[0 .. steps], alpha[0 .. steps), beta2[0 .. steps), ||v0||^2
    double* dd = (double*)ws.get((size_t)(3 * steps + 4) * sizeof(double), rc);
    if (!dd) return rc;
    double* hv = dd;
    double* alpha_d = dd + (steps + 1);
    double* beta2_d = alpha_d + steps;
    double* v0n = beta2_d + steps;
    int* ictl = (int*)ws.get(8 * sizeof(int), rc);  // barrier (2 words), fail flag, start-vector counter
    if (!ictl) return rc;
    // alpha_k, beta_k^2 of every step, written by the step kernel into mapped pinned memory
    double* hst = nullptr;
    {
        cudaError_t e = cudaHostAlloc((void**)&hst, (size_t)2 * steps * sizeof(double), cudaHostAllocMapped);
        if (e != cudaSuccess) return set_error(DQ_ENOMEM, "Lanczos cudaHostAlloc: %s", cudaGetErrorString(e));
        ws.host_allocs.push_back(hst);
    }
    double* hst_dev = nullptr;
    if (cudaHostGetDevicePointer((void**)&hst_dev, hst, 0) != cudaSuccess)
        return set_error(DQ_ECUDA, "Lanczos: no device address for mapped host memory");
    for (int q = 0; q < 3; ++q) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return set_error(DQ_ECUDA, "Lanczos: cudaEventCreate failed");
        ws.events.push_back(e);
    }
    cudaMemsetAsync(ictl, 0, 8 * sizeof(int), st);
    const int dtype = sizeof(T) == 8 ? DQ_F64 : DQ_F32;
    auto cuda_fail = [&](const char* what) -> int {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos %s: %s", what, cudaGetErrorString(e));
        return DQ_OK;
    };

    // v_0 = v0 / ||v0|| (last-block reduction; its counter is ictl[4])
    k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(v0, ldv, 1, v0, D, part, v0n, (unsigned*)(ictl + 4), nullptr);
    double nrm2 = 0.0;
    cudaError_t e = cudaMemcpyAsync(&nrm2, v0n, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos start vector: %s", cudaGetErrorString(e));
    if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) return set_error(DQ_EINVAL, "v0 has zero or non-finite norm");
    k_lz_start<T, P><<<8 * sms, kRedThreads, 0, st>>>(V, x, v0, v0n, D);

    LzStep<T, P> arg;
    arg.ldv = ldv;
    arg.V = V;
    arg.w = w;
    arg.r = r;
    arg.n = D;
    arg.reorth = reorth;
    arg.part = part;
    arg.h = hv;
    arg.alpha = alpha_d;
    arg.beta2 = beta2_d;
    arg.host = hst_dev;
    arg.bar = (unsigned*)ictl;
    arg.fail = ictl + 2;

    std::vector<double> a, b;
    double tnorm = 0.0, bprev = 0.0;
    int m = 0;
    bool stop = false;
    // host side of step q: its event has completed, so its coefficients are in hst
    auto consume = [&](int q) -> int {
        cudaError_t ee = cudaEventSynchronize(ws.events[q % 3]);
        if (ee != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos step: %s", cudaGetErrorString(ee));
        if (stop) return DQ_OK;
        const double al = ((volatile double*)hst)[2 * q], be = std::sqrt(((volatile double*)hst)[2 * q + 1]);
        if (!std::isfinite(al) || !std::isfinite(be)) return set_error(DQ_ECUDA, "Lanczos: non-finite coefficient");
        a.push_back(al);
        b.push_back(be);
        m = q + 1;
        tnorm = std::fmax(tnorm, std::fmax(std::fabs(al), std::fmax(be, bprev)));
        bprev = be;
        // an invariant subspace: the residual is at the level of the 48-bit arithmetic
        if (be < 1e-12 * tnorm) stop = true;
        return DQ_OK;
    };
    int queued = 0;
    for (int k = 0; k < steps; ++k) {
        if (k >= 2) {  // step k-2 is done; the GPU still has step k-1 queued
            if ((rc = consume(k - 2))) return rc;
            if (stop) break;
        }
        const T* xk = P::kXBuffer ? (const T*)x : (const T*)(V + (size_t)k * ldv);
        int le = launch_matvec(s, t, xk, w, dtype, 1, st);
        if (le) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)le));
        arg.k = k;
        arg.vnext = k + 1 < steps ? V + (size_t)(k + 1) * ldv : nullptr;
        arg.xnext = x;
        void* args[] = {&arg};
        const size_t smem = (size_t)(k + 1) * (sizeof(double) + sizeof(E));
        e = cudaLaunchCooperativeKernel((const void*)kern, dim3(nb), dim3(kLzThreads), args, smem, st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos step launch: %s", cudaGetErrorString(e));
        cudaEventRecord(ws.events[k % 3], st);
        if ((rc = cuda_fail("step"))) return rc;
        queued = k + 1;
    }
    for (int q = (queued >= 2 ? queued - 2 : 0); q < queued && !stop; ++q) {
        if (q < m) continue;
        if ((rc = consume(q))) return rc;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos: %s", cudaGetErrorString(e));
    int ctl[4] = {0, 0, 0, 0};
    cudaMemcpy(ctl, ictl, sizeof ctl, cudaMemcpyDeviceToHost);
    if (ctl[2]) return set_error(DQ_ECUDA, "Lanczos: a grid barrier of the step kernel timed out");
    if (m == 0) return set_error(DQ_ECUDA, "Lanczos: no step completed");
    std::vector<double> off(b.begin(), b.begin() + (m - 1));
    const double e0 = m == 1 ? a[0] : tridiag_min_eig(a, off);
    *E0 = e0;
    if (psi) {
        std::vector<double> y = m == 1 ? std::vector<double>{1.0} : tridiag_eigvec(a, off, e0);
        e = cudaMemcpyAsync(hv, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos Ritz vector: %s", cudaGetErrorString(e));
        k_combination<T, P><<<8 * sms, kRedThreads, (size_t)m * sizeof(E), st>>>(psi, V, ldv, m, hv, D);
        if ((rc = cuda_fail("Ritz vector"))) return rc;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos: %s", cudaGetErrorString(e));
    }
    if (alpha_out)
        for (int k = 0; k < m; ++k) alpha_out[k] = a[k];
    if (beta_out)
        for (int k = 0; k < m; ++k) beta_out[k] = b[k];
    if (steps_done) *steps_done = m;
    return DQ_OK;
}

}  // namespace dq

using namespace dq;

extern "C" int dq_lanczos(const dq_sector* s, const dq_terms* t, const void* v0, int steps, int dtype, int reorth,
                          double* E0, double* alpha, double* beta, int* steps_done, void* psi, void* stream) {
    clear_error();
    if (!s || !t || !v0 || !E0) return set_error(DQ_EINVAL, "NULL argument");
    if (t->sector != s) return set_error(DQ_EINVAL, "terms were compiled for another sector");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    if (steps < 1 || steps > 4096) return set_error(DQ_EINVAL, "steps must be in [1, 4096]");
    const bool ds = (reorth & DQ_LZ_DOUBLE_SINGLE) != 0;
    reorth &= ~DQ_LZ_DOUBLE_SINGLE;
    if (reorth < 0 || reorth > 2) return set_error(DQ_EINVAL, "reorth must be 0, 1 or 2 (optionally | DQ_LZ_DOUBLE_SINGLE)");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64) {
        const double* v = (const double*)v0;
        double* p = (double*)psi;
        return ds ? run_lanczos<double, LzDS<double>>(s, t, v, steps, reorth, E0, alpha, beta, steps_done, p, st)
                  : run_lanczos<double, LzF64<double>>(s, t, v, steps, reorth, E0, alpha, beta, steps_done, p, st);
    }
    const float* v = (const float*)v0;
    float* p = (float*)psi;
    return ds ? run_lanczos<float, LzDS<float>>(s, t, v, steps, reorth, E0, alpha, beta, steps_done, p, st)
              : run_lanczos<float, LzF64<float>>(s, t, v, steps, reorth, E0, alpha, beta, steps_done, p, st);
}
