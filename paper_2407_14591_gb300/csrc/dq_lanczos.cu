// Lanczos driver for the ground-state energy (Sec. 4.4; App. D calls a native Lanczos): the
// only use of H is the matrix-free product. Vectors live on the device in the caller's dtype;
// every dot product, norm and vector update is computed in FP64 with a fixed reduction order (the
// result does not depend on timing). The tridiagonal matrix T is solved on the host by bisection
// on its Sturm sequence, and the Ritz vector's coefficients by inverse iteration (own
// implementations).
//
// One step, all on the device:
//   w = H v_k                                     (the product)
//   alpha_k = <v_k, w>                            (k_gs_dots over one vector)
//   w -= alpha_k v_k + beta_{k-1} v_{k-1}         (k_three_term, with rho0 = ||w||)
//   with re-orthogonalisation, classical Gram-Schmidt against v_0 .. v_k:
//     h = V^T w; w -= V h                         (k_gs_dots, k_gs_update, with rho1 = ||w||)
//     a second pass only if rho1 < rho0 / sqrt(2) (the DGKS criterion; always with reorth = 2):
//     the kernels of that pass read the decision from device memory and return at once when
//     it is not needed
//   beta_k = ||w||; v_{k+1} = w / beta_k           (k_normalise)
// The reductions finish in the last block of each kernel (fixed order), the coefficients stay in
// device memory, and each step copies alpha_k and beta_k^2 into pinned host memory. The host
// reads step k's values only after it has queued step k+2 (two events in flight), so the GPU
// never waits for the host; a breakdown found late only costs the steps already queued, whose
// results are dropped.
// Work per step: the product, one pass over v_k and v_{k-1}, and with re-orthogonalisation two
// passes over V = [v_0 .. v_k] (dots, update), four when the second pass runs. The FP64 multiply-
// adds of those passes (2 D (k+1)) are what bounds a step on this GPU, where FP64 runs at a small
// fraction of the integer and FP32 rate.
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

// Sum of partial[0 .. nb) in a fixed order (strided per thread, then the block tree).
__device__ __forceinline__ double sum_partials(const double* partial, int nb, double* sh) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += __ldcg(partial + b);
    return block_sum(acc, sh);
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

// w[i] -= sum_{j<k} h[j] V_j[i] (FP64 arithmetic, stored in T) and the new ||w||^2 into
// scal[norm_slot]; the first pass (pass2 == false) also decides whether the second one runs
// (scal[kPass2]: always with `always2`, else when the norm fell below 1/sqrt(2) of rho0), the
// second (pass2 == true) does nothing unless scal[kPass2] is set. Both leave the step's final
// ||w||^2 in scal[kBeta2].
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gs_update(T* __restrict__ w, const T* __restrict__ V, size_t ldv,
                                                            int k, const double* __restrict__ h, uint64_t n,
                                                            double* __restrict__ partial, double* scal,
                                                            unsigned* counter, bool pass2, bool always2) {
    if (pass2 && scal[kPass2] == 0.0) return;
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
        nacc += (double)r * (double)r;
    }
    nacc = block_sum(nacc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = nacc;
    if (last_block(counter)) {
        const double r2 = sum_partials(partial, gridDim.x, red);
        if (threadIdx.x == 0) {
            if (!pass2) {
                scal[kRho1] = r2;
                scal[kPass2] = (always2 || r2 < 0.5 * scal[kRho0]) ? 1.0 : 0.0;
            }
            scal[kBeta2] = r2;
        }
    }
}

// w -= alpha v + beta u (u may be NULL; alpha = scal[kAlpha], beta^2 = beta2_prev), the new
// ||w||^2 into scal[kRho0] and scal[kBeta2].
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_three_term(T* __restrict__ w, const T* __restrict__ v,
                                                             const T* __restrict__ u, double* scal,
                                                             const double* __restrict__ beta2_prev, uint64_t n,
                                                             double* __restrict__ partial, unsigned* counter) {
    __shared__ double red[32];
    const double al = scal[kAlpha], be = u ? sqrt(*beta2_prev) : 0.0;
    double nacc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = (double)w[i] - al * (double)v[i];
        if (u) acc -= be * (double)u[i];
        const T r = (T)acc;
        w[i] = r;
        nacc += (double)r * (double)r;
    }
    nacc = block_sum(nacc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = nacc;
    if (last_block(counter)) {
        const double r2 = sum_partials(partial, gridDim.x, red);
        if (threadIdx.x == 0) {
            scal[kRho0] = r2;
            scal[kBeta2] = r2;
        }
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
    const int nbd = 2 * sms;  // blocks of the dot kernel (one partial per vector each)
    const int nbu = 8 * sms;  // blocks of the streaming kernels
    int rc = DQ_OK;
    Work ws;
    T* V = (T*)ws.get((size_t)(steps + 1) * ldv * sizeof(T), rc);
    if (!V) return rc;
    T* w = (T*)ws.get(ldv * sizeof(T), rc);
    if (!w) return rc;
    double* partial = (double*)ws.get((size_t)((steps + 1) * nbd + nbu) * sizeof(double), rc);
    if (!partial) return rc;
    // device doubles: h[0 .. steps], then the scalars; counters of the last-block reductions
    double* dd = (double*)ws.get((size_t)(steps + 1 + kNScal) * sizeof(double), rc);
    if (!dd) return rc;
    double* hv = dd;
    double* scal = dd + (steps + 1);
    unsigned* counter = (unsigned*)ws.get(4 * sizeof(unsigned), rc);
    if (!counter) return rc;
    double* beta2_prev = (double*)ws.get(sizeof(double), rc);  // beta_{k-1}^2 for the three-term step
    if (!beta2_prev) return rc;
    double* hst = (double*)ws.get_host((size_t)2 * steps * sizeof(double), rc);  // alpha_k, beta_k^2
    if (!hst) return rc;
    const int nev = 3;
    for (int q = 0; q < nev; ++q) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return set_error(DQ_ECUDA, "Lanczos: cudaEventCreate failed");
        ws.events.push_back(e);
    }
    cudaMemsetAsync(counter, 0, 4 * sizeof(unsigned), st);
    const int dtype = sizeof(T) == 8 ? DQ_F64 : DQ_F32;
    auto cuda_fail = [&](const char* what) -> int {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos %s: %s", what, cudaGetErrorString(e));
        return DQ_OK;
    };

    // v_0 = v0 / ||v0||
    k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(v0, ldv, 1, v0, D, partial, scal + kV0, counter, nullptr);
    double nrm2 = 0.0;
    cudaError_t e = cudaMemcpyAsync(&nrm2, scal + kV0, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos start vector: %s", cudaGetErrorString(e));
    if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) return set_error(DQ_EINVAL, "v0 has zero or non-finite norm");
    k_normalise<T><<<nbu, kRedThreads, 0, st>>>(V, v0, scal + kV0, D);
    cudaMemsetAsync(beta2_prev, 0, sizeof(double), st);

    std::vector<double> a, b;
    double tnorm = 0.0, bprev = 0.0;
    int m = 0;
    bool stop = false;
    // host side of step q: read its coefficients (its event has completed) and test for breakdown
    auto consume = [&](int q) -> int {
        cudaError_t ee = cudaEventSynchronize(ws.events[q % nev]);
        if (ee != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos step: %s", cudaGetErrorString(ee));
        if (stop) return DQ_OK;
        const double al = hst[2 * q], be = std::sqrt(hst[2 * q + 1]);
        a.push_back(al);
        b.push_back(be);
        m = q + 1;
        tnorm = std::fmax(tnorm, std::fmax(std::fabs(al), std::fmax(be, bprev)));
        bprev = be;
        if (!std::isfinite(al) || !std::isfinite(be)) return set_error(DQ_ECUDA, "Lanczos: non-finite coefficient");
        if (be < 1e-14 * tnorm) stop = true;
        return DQ_OK;
    };
    int queued = 0;
    for (int k = 0; k < steps; ++k) {
        if (k >= 2) {  // step k-2 done: the GPU still has step k-1 queued
            if ((rc = consume(k - 2))) return rc;
            if (stop) break;
        }
        T* vk = V + (size_t)k * ldv;
        int le = launch_matvec(s, t, vk, w, dtype, 1, st);
        if (le) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)le));
        k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(vk, ldv, 1, w, D, partial, scal + kAlpha, counter, nullptr);
        k_three_term<T><<<nbu, kRedThreads, 0, st>>>(w, vk, k ? V + (size_t)(k - 1) * ldv : nullptr, scal,
                                                    beta2_prev, D, partial, counter + 1);
        if (reorth) {
            const int kk = k + 1;
            const size_t hsm = (size_t)kk * sizeof(double);
            for (int pass = 0; pass < 2; ++pass) {
                k_gs_dots<T><<<nbd, kRedThreads, 0, st>>>(V, ldv, kk, w, D, partial, hv, counter + 2,
                                                         pass ? scal + kPass2 : nullptr);
                k_gs_update<T><<<nbu, kRedThreads, hsm, st>>>(w, V, ldv, kk, hv, D, partial + (size_t)kk * nbd, scal,
                                                             counter + 3, pass == 1, reorth == 2);
            }
        }
        if (k + 1 < steps) k_normalise<T><<<nbu, kRedThreads, 0, st>>>(V + (size_t)(k + 1) * ldv, w, scal + kBeta2, D);
        cudaMemcpyAsync(beta2_prev, scal + kBeta2, sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(hst + 2 * k, scal + kAlpha, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hst + 2 * k + 1, scal + kBeta2, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaEventRecord(ws.events[k % nev], st);
        if ((rc = cuda_fail("step"))) return rc;
        queued = k + 1;
    }
    for (int q = (queued >= 2 ? queued - 2 : 0); q < queued && !stop; ++q) {
        if (q < m) continue;
        if ((rc = consume(q))) return rc;
    }
    if (m == 0) return set_error(DQ_ECUDA, "Lanczos: no step completed");
    std::vector<double> off(b.begin(), b.begin() + (m - 1));
    const double e0 = m == 1 ? a[0] : tridiag_min_eig(a, off);
    *E0 = e0;
    if (psi) {
        std::vector<double> y = m == 1 ? std::vector<double>{1.0} : tridiag_eigvec(a, off, e0);
        e = cudaMemcpyAsync(hv, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos Ritz vector: %s", cudaGetErrorString(e));
        k_combination<T><<<nbu, kRedThreads, (size_t)m * sizeof(double), st>>>(psi, V, ldv, m, hv, D);
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
    if (steps < 1 || steps > 4096) return set_error(DQ_EINVAL, "steps must be in [1, 4096]");
    if (reorth < 0 || reorth > 2) return set_error(DQ_EINVAL, "reorth must be 0, 1 or 2");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64)
        return run_lanczos<double>(s, t, (const double*)v0, steps, reorth, E0, alpha, beta, steps_done, (double*)psi,
                                   st);
    return run_lanczos<float>(s, t, (const float*)v0, steps, reorth, E0, alpha, beta, steps_done, (float*)psi, st);
}
