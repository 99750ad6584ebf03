// Lanczos driver for the ground-state energy (Sec. 4.4; App. D calls a native Lanczos): the
// only use of H is the matrix-free product. Vectors live on the device in the caller's dtype;
// every dot product and norm accumulates in FP64 with a fixed reduction tree (the result does
// not depend on timing). The tridiagonal matrix T is solved on the host by bisection on its
// Sturm sequence, and the Ritz vector's coefficients by inverse iteration (own implementations).
//
// Data movement per step, with full re-orthogonalisation (classical Gram-Schmidt, twice):
//   dots   h1 = V^T w            one pass over V, one pass over w per tile of kDotTile vectors
//   update w -= V h1             one pass over V
//   dots   h2 = V^T w            one pass over V
//   update w -= V h2, ||w||^2    one pass over V
//   scale  v_{k+1} = w / ||w||
// The coefficients stay on the device (each kernel reads them from device memory); the host
// reads alpha_k and ||w||^2 once per step, for T and for the breakdown test.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

constexpr int kRedThreads = 256;
constexpr int kDotTile = 16;  // basis vectors per pass of the blocked dot kernel

static int sm_count_now() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

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

// partial[j * gridDim.x + block] = sum over the block's rows of V_j[i] * w[i], for j < k.
// The rows of a block are a grid stride; each pass takes kDotTile vectors at once, so w is read
// once per tile instead of once per vector, and one block reduction serves the whole tile.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gs_dots(const T* __restrict__ V, size_t ldv, int k,
                                                          const T* __restrict__ w, uint64_t n,
                                                          double* __restrict__ partial) {
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
            partial[(size_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[j] = sum_b partial[j * nb + b], one block per j.
__global__ void k_finish(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[(size_t)blockIdx.x * nb + b];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// w[i] = w[i] - sum_{j<k} h[j] V_j[i] (FP64 arithmetic, stored in T); with NORM, also the
// block's partial sum of the new w[i]^2 into norm_partial[block]. h is a device array of k
// doubles, staged in shared memory.
template <typename T, bool NORM>
__global__ void __launch_bounds__(kRedThreads) k_gs_update(T* __restrict__ w, const T* __restrict__ V, size_t ldv,
                                                            int k, const double* __restrict__ h, uint64_t n,
                                                            double* __restrict__ norm_partial) {
    extern __shared__ double hs[];
    __shared__ double red[32];
    for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
    __syncthreads();
    double nacc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = (double)w[i];
        int j = 0;
        for (; j + 8 <= k; j += 8) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (double)__ldg(V + (size_t)(j + q) * ldv + i);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc -= hs[j + q] * v[q];
        }
        for (; j < k; ++j) acc -= hs[j] * (double)__ldg(V + (size_t)j * ldv + i);
        const T r = (T)acc;
        w[i] = r;
        if (NORM) nacc += (double)r * (double)r;
    }
    if (NORM) {
        nacc = block_sum(nacc, red);
        if (threadIdx.x == 0) norm_partial[blockIdx.x] = nacc;
    }
}

// Plain three-term step without re-orthogonalisation: w -= alpha v + beta u (u may be NULL),
// with alpha = *a and beta = sqrt(*bb) read from device memory, and the block's partial sum of
// the new w^2.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_three_term(T* __restrict__ w, const T* __restrict__ v,
                                                             const T* __restrict__ u, const double* __restrict__ a,
                                                             const double* __restrict__ bb, uint64_t n,
                                                             double* __restrict__ norm_partial) {
    __shared__ double red[32];
    const double al = *a, be = u ? sqrt(*bb) : 0.0;
    double nacc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = (double)w[i] - al * (double)v[i];
        if (u) acc -= be * (double)u[i];
        const T r = (T)acc;
        w[i] = r;
        nacc += (double)r * (double)r;
    }
    nacc = block_sum(nacc, red);
    if (threadIdx.x == 0) norm_partial[blockIdx.x] = nacc;
}

// dst = src / sqrt(*nrm2) (the norm squared read from device memory).
template <typename T>
__global__ void k_normalise(T* __restrict__ dst, const T* __restrict__ src, const double* __restrict__ nrm2,
                            uint64_t n) {
    const double s = 1.0 / sqrt(*nrm2);
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
    ~Work() {
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
};

template <typename T>
static int run_lanczos(const dq_sector* s, const dq_terms* t, const T* v0, int steps, int reorth, double* E0,
                       double* alpha_out, double* beta_out, int* steps_done, T* psi, cudaStream_t st) {
    const uint64_t D = s->D;
    const size_t ldv = (D + 31) & ~(size_t)31;
    const int sms = sm_count_now();
    const int nbd = 4 * sms;  // blocks of the dot kernels (one partial each)
    const int nbu = 8 * sms;  // blocks of the streaming kernels
    int rc = DQ_OK;
    Work ws;
    T* V = (T*)ws.get((size_t)(steps + 1) * ldv * sizeof(T), rc);
    if (!V) return rc;
    T* w = (T*)ws.get(ldv * sizeof(T), rc);
    if (!w) return rc;
    const int nbmax = nbd > nbu ? nbd : nbu;
    double* partial = (double*)ws.get((size_t)(steps + 2) * nbmax * sizeof(double), rc);
    if (!partial) return rc;
    // device scalars: h1[0..steps], h2[0..steps], then [alpha, ||w||^2, ||v0||^2]
    double* dres = (double*)ws.get((size_t)(2 * (steps + 1) + 8) * sizeof(double), rc);
    if (!dres) return rc;
    double* h1 = dres;
    double* h2 = dres + (steps + 1);
    double* dsc = dres + 2 * (steps + 1);
    const int dtype = sizeof(T) == 8 ? DQ_F64 : DQ_F32;
    auto cuda_fail = [&](const char* what) -> int {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos %s: %s", what, cudaGetErrorString(e));
        return DQ_OK;
    };

    // v_0 = v0 / ||v0||
    k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(v0, ldv, 1, v0, D, partial);
    k_finish<<<1, kRedThreads, 0, st>>>(partial, nbd, dsc + 2);
    double nrm2 = 0.0;
    cudaError_t e = cudaMemcpyAsync(&nrm2, dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos start vector: %s", cudaGetErrorString(e));
    if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) return set_error(DQ_EINVAL, "v0 has zero or non-finite norm");
    k_normalise<T><<<nbu, kRedThreads, 0, st>>>(V, v0, dsc + 2, D);

    std::vector<double> a, b;
    double bprev = 0.0, tnorm = 0.0;
    int m = 0;
    for (int k = 0; k < steps; ++k) {
        T* vk = V + (size_t)k * ldv;
        int le = launch_matvec(s, t, vk, w, dtype, 1, st);
        if (le) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)le));
        if (reorth) {
            // h1 = V^T w (h1[k] = alpha_k), w -= V h1; h2 = V^T w, w -= V h2 with ||w||^2
            const int kk = k + 1;
            const size_t hsm = (size_t)kk * sizeof(double);
            k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(V, ldv, kk, w, D, partial);
            k_finish<<<kk, kRedThreads, 0, st>>>(partial, nbd, h1);
            k_gs_update<T, false><<<nbu, kRedThreads, hsm, st>>>(w, V, ldv, kk, h1, D, nullptr);
            k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(V, ldv, kk, w, D, partial);
            k_finish<<<kk, kRedThreads, 0, st>>>(partial, nbd, h2);
            k_gs_update<T, true><<<nbu, kRedThreads, hsm, st>>>(w, V, ldv, kk, h2, D, partial);
            k_finish<<<1, kRedThreads, 0, st>>>(partial, nbu, dsc + 1);
            cudaMemcpyAsync(dsc, h1 + k, sizeof(double), cudaMemcpyDeviceToDevice, st);
        } else {
            // alpha_k = <v_k, w>; w -= alpha_k v_k + beta_{k-1} v_{k-1} with ||w||^2
            k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(vk, ldv, 1, w, D, partial);
            k_finish<<<1, kRedThreads, 0, st>>>(partial, nbd, dsc);
            // dsc[1] still holds ||w_{k-1}||^2 = beta_{k-1}^2 when k > 0
            k_three_term<T><<<nbu, kRedThreads, 0, st>>>(w, vk, k ? V + (size_t)(k - 1) * ldv : nullptr, dsc, dsc + 1,
                                                        D, partial);
            k_finish<<<1, kRedThreads, 0, st>>>(partial, nbu, dsc + 1);
        }
        if (k + 1 < steps) k_normalise<T><<<nbu, kRedThreads, 0, st>>>(V + (size_t)(k + 1) * ldv, w, dsc + 1, D);
        if ((rc = cuda_fail("step"))) return rc;
        double hs2[2];
        e = cudaMemcpyAsync(hs2, dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos step: %s", cudaGetErrorString(e));
        const double al = hs2[0], be = std::sqrt(hs2[1]);
        a.push_back(al);
        b.push_back(be);
        m = k + 1;
        tnorm = std::fmax(tnorm, std::fmax(std::fabs(al), std::fmax(be, bprev)));
        if (k == steps - 1 || be < 1e-14 * tnorm) break;
        bprev = be;
    }
    std::vector<double> off(b.begin(), b.begin() + (m - 1));
    const double e0 = m == 1 ? a[0] : tridiag_min_eig(a, off);
    *E0 = e0;
    if (psi) {
        std::vector<double> y = m == 1 ? std::vector<double>{1.0} : tridiag_eigvec(a, off, e0);
        e = cudaMemcpyAsync(h1, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos Ritz vector: %s", cudaGetErrorString(e));
        k_combination<T><<<nbu, kRedThreads, (size_t)m * sizeof(double), st>>>(psi, V, ldv, m, h1, D);
        if ((rc = cuda_fail("Ritz vector"))) return rc;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos: %s", cudaGetErrorString(e));
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
    if (steps < 1) return set_error(DQ_EINVAL, "steps must be >= 1");
    if (steps > 4096) return set_error(DQ_EINVAL, "steps must be <= 4096");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64)
        return run_lanczos<double>(s, t, (const double*)v0, steps, reorth, E0, alpha, beta, steps_done, (double*)psi,
                                   st);
    return run_lanczos<float>(s, t, (const float*)v0, steps, reorth, E0, alpha, beta, steps_done, (float*)psi, st);
}
