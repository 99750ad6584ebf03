// Lanczos driver for the ground-state energy (Sec. 4.4; App. D calls a native Lanczos): the
// only use of H is the matrix-free product. Vectors live on the device in the caller's dtype;
// every dot product and norm accumulates in FP64 with a fixed reduction order (the result does
// not depend on timing). The tridiagonal matrix T is solved on the host by bisection on its
// Sturm sequence, and the Ritz vector's coefficients by inverse iteration (own
// implementations).
//
// One step is two launches: the product w = H v_k, then one cooperative kernel (k_lz_step, all
// blocks resident, grid-wide barriers between its phases) that does the rest on the device:
//   alpha_k = <v_k, w>;  w -= alpha_k v_k + beta_{k-1} v_{k-1}      (rho0 = ||w||)
//   with re-orthogonalisation, classical Gram-Schmidt against V = [v_0 .. v_k]:
//     h = V^T w; w -= V h                                           (rho1 = ||w||)
//     a second pass only if rho1 < rho0 / sqrt(2) (the DGKS criterion; always with reorth = 2)
//   beta_k = ||w||; v_{k+1} = w / beta_k
// Every block reduces the partial sums itself in the same fixed order, so all blocks hold the
// same coefficients without another barrier. alpha_k and beta_k^2 go to device arrays and to
// mapped pinned host memory. The host reads step k's values only after it has queued step k+2,
// so the GPU never waits for the host; a breakdown found late only costs the steps already
// queued, whose results are dropped.
// Arithmetic: FP64 for dot products, norms, the three-term step and (FP64 vectors) the
// Gram-Schmidt updates; FP32 vectors are widened to FP64 with integer bit operations (exact)
// and take their Gram-Schmidt updates, whose coefficients are at the level of the vectors' own
// rounding, as FP32 multiply-adds. The FP64 multiply-adds of the passes over V (2 D (k+1) per
// step) bound a step on this GPU, whose FP64 rate is a small fraction of its integer rate.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

constexpr int kRedThreads = 256;
constexpr int kDotTile = 16;  // basis vectors per pass of the blocked dot kernel

// Device scalars of the driver (one array of doubles in the workspace).
enum : int {
    kAlpha = 0,    // alpha_k
    kRho0 = 1,     // ||w||^2 after the three-term step
    kRho1 = 2,     // ||w||^2 after the first Gram-Schmidt pass
    kBeta2 = 3,    // ||w||^2 at the end of the step: beta_k^2
    kPass2 = 4,    // 1.0 if the second pass runs
    kV0 = 5,       // ||v0||^2
    kNScal = 8,
};

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

// Exact widening of a float to double with integer operations (the hardware conversion runs on
// the FP64 pipe); zero, subnormals, Inf and NaN take the hardware path.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
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

template <typename T>
struct LzStep {
    const T* V;       // v_0 .. v_k, stride ldv
    size_t ldv;
    int k;            // step index
    T* w;             // H v_k on entry; the new residual on exit
    T* vnext;         // v_{k+1} (NULL at the last step)
    uint64_t n;
    int reorth;       // 0, 1 (DGKS second pass), 2 (second pass always)
    double* part;     // per-block partial sums, gridDim.x * (2 (k+1) + 8) doubles
    double* h;        // projection coefficients, k+1 doubles
    double* alpha;    // alpha_j, beta_j^2 of every step (device)
    double* beta2;
    volatile double* host;  // mapped pinned host memory: alpha_k, beta_k^2 at [2k], [2k+1]
    unsigned* bar;    // grid barrier (two words)
    int* fail;        // barrier timeout
};

// h = V^T w over j <= k (partials per block and vector, then block b reduces the vectors
// j = b, b + nb, ... in block order), followed by w -= V h and the block partials of ||w||^2.
template <typename T>
__device__ __forceinline__ bool lz_gram_schmidt(const LzStep<T>& a, double* pd, double* pn, double* hs,
                                                double* red) {
    __shared__ double sh[kDotTile][kRedThreads / 32];
    const int kk = a.k + 1, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (int j0 = 0; j0 < kk; j0 += kDotTile) {
        const int nj = kk - j0 < kDotTile ? kk - j0 : kDotTile;
        double acc[kDotTile];
#pragma unroll
        for (int q = 0; q < kDotTile; ++q) acc[q] = 0.0;
        const T* Vb = a.V + (size_t)j0 * a.ldv;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += step) {
            const double wi = widen(a.w[i]);
#pragma unroll
            for (int q = 0; q < kDotTile; ++q)
                if (q < nj) acc[q] += widen(__ldg(Vb + (size_t)q * a.ldv + i)) * wi;
        }
#pragma unroll
        for (int q = 0; q < kDotTile; ++q) {
            double v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[q][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < nj) {
            double sum = 0.0;
            for (int r = 0; r < kRedThreads / 32; ++r) sum += sh[threadIdx.x][r];
            pd[(size_t)blockIdx.x * kk + j0 + threadIdx.x] = sum;
        }
        __syncthreads();
    }
    if (!grid_sync(a.bar, a.fail)) return false;
    for (int j = blockIdx.x; j < kk; j += gridDim.x) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc += __ldcg(pd + (size_t)b * kk + j);
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) a.h[j] = acc;
    }
    if (!grid_sync(a.bar, a.fail)) return false;
    for (int q = threadIdx.x; q < kk; q += blockDim.x) hs[q] = __ldcg(a.h + q);
    __syncthreads();
    double nacc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += step) {
        T r;
        if constexpr (sizeof(T) == 8) {
            double acc = a.w[i];
            int j = 0;
            for (; j + 8 <= kk; j += 8) {
                double v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = __ldg(a.V + (size_t)(j + q) * a.ldv + i);
#pragma unroll
                for (int q = 0; q < 8; ++q) acc -= hs[j + q] * v[q];
            }
            for (; j < kk; ++j) acc -= hs[j] * __ldg(a.V + (size_t)j * a.ldv + i);
            r = acc;
        } else {
            float corr = 0.f;
            int j = 0;
            for (; j + 8 <= kk; j += 8) {
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = __ldg(a.V + (size_t)(j + q) * a.ldv + i);
#pragma unroll
                for (int q = 0; q < 8; ++q) corr = fmaf((float)hs[j + q], v[q], corr);
            }
            for (; j < kk; ++j) corr = fmaf((float)hs[j], __ldg(a.V + (size_t)j * a.ldv + i), corr);
            r = a.w[i] - corr;
        }
        a.w[i] = r;
        const double rd = widen(r);
        nacc += rd * rd;
    }
    nacc = block_sum(nacc, red);
    if (threadIdx.x == 0) pn[blockIdx.x] = nacc;
    return grid_sync(a.bar, a.fail);
}

// One Lanczos step after the product (see the file comment). Cooperative launch; dynamic shared
// memory: k + 1 doubles (the projection coefficients).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_lz_step(LzStep<T> a) {
    extern __shared__ double hs[];
    __shared__ double red[33];
    const int nb = gridDim.x;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    double* p_alpha = a.part;
    double* p_rho0 = a.part + nb;
    double* p_rho1 = a.part + 2 * nb;
    double* p_rho2 = a.part + 3 * nb;
    double* p_dots = a.part + 4 * nb;  // nb * kk
    const T* vk = a.V + (size_t)a.k * a.ldv;
    const T* vp = a.k ? a.V + (size_t)(a.k - 1) * a.ldv : nullptr;
    // alpha_k = <v_k, w>
    double acc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += step)
        acc += widen(__ldg(vk + i)) * widen(a.w[i]);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) p_alpha[blockIdx.x] = acc;
    if (!grid_sync(a.bar, a.fail)) return;
    const double al = reduce_all(p_alpha, nb, red);
    const double be = vp ? sqrt(__ldcg(a.beta2 + a.k - 1)) : 0.0;
    // three-term step, rho0^2
    acc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += step) {
        double r = widen(a.w[i]) - al * widen(__ldg(vk + i));
        if (vp) r -= be * widen(__ldg(vp + i));
        const T rt = (T)r;
        a.w[i] = rt;
        const double rd = widen(rt);
        acc += rd * rd;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) p_rho0[blockIdx.x] = acc;
    if (!grid_sync(a.bar, a.fail)) return;
    double b2 = reduce_all(p_rho0, nb, red);
    if (a.reorth) {
        const double rho0 = b2;
        if (!lz_gram_schmidt(a, p_dots, p_rho1, hs, red)) return;
        b2 = reduce_all(p_rho1, nb, red);
        if (a.reorth == 2 || b2 < 0.5 * rho0) {
            if (!lz_gram_schmidt(a, p_dots, p_rho2, hs, red)) return;
            b2 = reduce_all(p_rho2, nb, red);
        }
    }
    // beta_k, v_{k+1}
    if (a.vnext) {
        const double sc = b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += step)
            a.vnext[i] = (T)(sc * widen(a.w[i]));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.alpha[a.k] = al;
        a.beta2[a.k] = b2;
        a.host[2 * a.k] = al;
        a.host[2 * a.k + 1] = b2;
        __threadfence_system();
    }
}

// dst = src / sqrt(*nrm2) (the norm squared read from device memory); a zero norm (an exact
// invariant subspace) gives a zero vector.
template <typename T>
__global__ void k_normalise(T* __restrict__ dst, const T* __restrict__ src, const double* __restrict__ nrm2,
                            uint64_t n) {
    const double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (T)(s * (double)src[i]);
}

// psi[i] = sum_{j<k} c[j] V_j[i] (FP64 arithmetic, stored in T); c staged in shared memory.
template <typename T>
__global__ void k_combination(T* __restrict__ psi, const T* __restrict__ V, size_t ldv, int k,
                              const double* __restrict__ c, uint64_t n) {
    extern __shared__ double cs[];
    for (int q = threadIdx.x; q < k; q += blockDim.x) cs[q] = c[q];
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc += cs[j] * (double)__ldg(V + (size_t)j * ldv + i);
        psi[i] = (T)acc;
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

template <typename T>
static int run_lanczos(const dq_sector* s, const dq_terms* t, const T* v0, int steps, int reorth, double* E0,
                       double* alpha_out, double* beta_out, int* steps_done, T* psi, cudaStream_t st) {
    const uint64_t D = s->D;
    const size_t ldv = (D + 31) & ~(size_t)31;
    const int sms = sm_count_cached();
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return set_error(DQ_ECUDA, "Lanczos: the device does not support cooperative launches");
    const size_t hsm = (size_t)(steps + 1) * sizeof(double);
    auto kern = k_lz_step<T>;
    if (hsm > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm) != cudaSuccess)
        return set_error(DQ_ECUDA, "Lanczos: shared memory for %d coefficients", steps + 1);
    int per_sm = occupancy_cached(reinterpret_cast<const void*>(kern), kRedThreads, hsm);
    if (per_sm > 4) per_sm = 4;
    const int nb = per_sm * sms;  // blocks of the cooperative step kernel (all resident)
    const int nbd = 2 * sms;      // blocks of the start-vector reduction
    int rc = DQ_OK;
    Work ws;
    T* V = (T*)ws.get((size_t)(steps + 1) * ldv * sizeof(T), rc);
    if (!V) return rc;
    T* w = (T*)ws.get(ldv * sizeof(T), rc);
    if (!w) return rc;
    const size_t npart = (size_t)nb * (steps + 6) > (size_t)nbd ? (size_t)nb * (steps + 6) : (size_t)nbd;
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
    k_normalise<T><<<8 * sms, kRedThreads, 0, st>>>(V, v0, v0n, D);

    LzStep<T> arg;
    arg.ldv = ldv;
    arg.V = V;
    arg.w = w;
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
        if (be < 1e-14 * tnorm) stop = true;
        return DQ_OK;
    };
    int queued = 0;
    for (int k = 0; k < steps; ++k) {
        if (k >= 2) {  // step k-2 is done; the GPU still has step k-1 queued
            if ((rc = consume(k - 2))) return rc;
            if (stop) break;
        }
        T* vk = V + (size_t)k * ldv;
        int le = launch_matvec(s, t, vk, w, dtype, 1, st);
        if (le) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)le));
        arg.k = k;
        arg.vnext = k + 1 < steps ? V + (size_t)(k + 1) * ldv : nullptr;
        void* args[] = {&arg};
        e = cudaLaunchCooperativeKernel((const void*)kern, dim3(nb), dim3(kRedThreads), args, (size_t)(k + 1) * 8, st);
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
        k_combination<T><<<8 * sms, kRedThreads, (size_t)m * sizeof(double), st>>>(psi, V, ldv, m, hv, D);
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
    if (reorth < 0 || reorth > 2) return set_error(DQ_EINVAL, "reorth must be 0, 1 or 2");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64)
        return run_lanczos<double>(s, t, (const double*)v0, steps, reorth, E0, alpha, beta, steps_done, (double*)psi,
                                   st);
    return run_lanczos<float>(s, t, (const float*)v0, steps, reorth, E0, alpha, beta, steps_done, (float*)psi, st);
}
