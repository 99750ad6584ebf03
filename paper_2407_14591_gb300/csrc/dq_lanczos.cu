// Lanczos driver for the ground-state energy (Sec. 4.4; App. D calls a native Lanczos): the
// only use of H is the matrix-free product. Vectors live on the device in the caller's dtype;
// every dot product and norm accumulates in FP64 with a fixed two-pass reduction tree (the
// result does not depend on timing). The tridiagonal matrix T is solved on the host by
// bisection on its Sturm sequence (own implementation).
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

constexpr int kRedThreads = 256;

static int red_blocks() {
    static int b = 0;
    if (!b) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        b = 2 * (sms > 0 ? sms : 1);
    }
    return b;
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

// partial[j * gridDim.x + block] = sum over the block's rows of V_j[i] * w[i], j < k.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_multi_dot(const T* __restrict__ V, size_t ldv, int k,
                                                            const T* __restrict__ w, uint64_t n,
                                                            double* __restrict__ partial) {
    __shared__ double sh[32];
    for (int j = 0; j < k; ++j) {
        const T* v = V + (size_t)j * ldv;
        double acc = 0.0;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
            acc += (double)v[i] * (double)w[i];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = acc;
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

// w[i] -= sum_{j<k} h[j] V_j[i]
template <typename T>
__global__ void k_sub_combination(T* __restrict__ w, const T* __restrict__ V, size_t ldv, int k,
                                  const double* __restrict__ h, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = (double)w[i];
        for (int j = 0; j < k; ++j) acc -= h[j] * (double)V[(size_t)j * ldv + i];
        w[i] = (T)acc;
    }
}

// w -= a v + b u   (u may be NULL)
template <typename T>
__global__ void k_three_term(T* __restrict__ w, const T* __restrict__ v, const T* __restrict__ u, double a, double b,
                             uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = (double)w[i] - a * (double)v[i];
        if (u) acc -= b * (double)u[i];
        w[i] = (T)acc;
    }
}

template <typename T>
__global__ void k_scale_copy(T* __restrict__ dst, const T* __restrict__ src, double s, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (T)(s * (double)src[i]);
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
                       double* alpha_out, double* beta_out, int* steps_done, cudaStream_t st) {
    const uint64_t D = s->D;
    const size_t ldv = (D + 31) & ~(size_t)31;
    const int nb = red_blocks();
    int rc = DQ_OK;
    Work ws;
    T* V = (T*)ws.get((size_t)(steps + 1) * ldv * sizeof(T), rc);
    if (!V) return rc;
    T* w = (T*)ws.get(ldv * sizeof(T), rc);
    if (!w) return rc;
    double* partial = (double*)ws.get((size_t)(steps + 1) * nb * sizeof(double), rc);
    if (!partial) return rc;
    double* dres = (double*)ws.get((size_t)(steps + 1) * sizeof(double), rc);
    if (!dres) return rc;
    std::vector<double> h(steps + 1);
    const unsigned grid = (unsigned)nb;
    const int dtype = sizeof(T) == 8 ? DQ_F64 : DQ_F32;

    auto dots = [&](const T* Vb, int k, const T* x, double* out) -> int {
        k_multi_dot<T><<<grid, kRedThreads, 0, st>>>(Vb, ldv, k, x, D, partial);
        k_finish<<<k, kRedThreads, 0, st>>>(partial, nb, dres);
        cudaError_t e = cudaMemcpyAsync(out, dres, k * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos reduction: %s", cudaGetErrorString(e));
        return DQ_OK;
    };

    double nrm2;
    if ((rc = dots(v0, 1, v0, &nrm2))) return rc;
    if (!(nrm2 > 0.0)) return set_error(DQ_EINVAL, "v0 has zero norm");
    k_scale_copy<T><<<grid, 256, 0, st>>>(V, v0, 1.0 / std::sqrt(nrm2), D);
    std::vector<double> a, b;
    double bprev = 0.0, tnorm = 0.0;
    int m = 0;
    for (int k = 0; k < steps; ++k) {
        T* vk = V + (size_t)k * ldv;
        int e = launch_matvec(s, t, vk, w, dtype, 1, st);
        if (e) return set_error(DQ_ECUDA, "matvec launch: %s", cudaGetErrorString((cudaError_t)e));
        double al;
        if ((rc = dots(vk, 1, w, &al))) return rc;
        k_three_term<T><<<grid, 256, 0, st>>>(w, vk, k ? V + (size_t)(k - 1) * ldv : nullptr, al, bprev, D);
        if (reorth) {
            for (int pass = 0; pass < 2; ++pass) {
                if ((rc = dots(V, k + 1, w, h.data()))) return rc;
                cudaMemcpyAsync(dres, h.data(), (k + 1) * sizeof(double), cudaMemcpyHostToDevice, st);
                k_sub_combination<T><<<grid, 256, 0, st>>>(w, V, ldv, k + 1, dres, D);
            }
        }
        double bb;
        if ((rc = dots(w, 1, w, &bb))) return rc;
        double be = std::sqrt(bb);
        a.push_back(al);
        b.push_back(be);
        m = k + 1;
        tnorm = std::fmax(tnorm, std::fmax(std::fabs(al), std::fmax(be, bprev)));
        if (k == steps - 1 || be < 1e-14 * tnorm) break;
        k_scale_copy<T><<<grid, 256, 0, st>>>(V + (size_t)(k + 1) * ldv, w, 1.0 / be, D);
        bprev = be;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "Lanczos: %s", cudaGetErrorString(e));
    std::vector<double> off(b.begin(), b.begin() + (m - 1));
    *E0 = m == 1 ? a[0] : tridiag_min_eig(a, off);
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
                          double* E0, double* alpha, double* beta, int* steps_done, void* stream) {
    clear_error();
    if (!s || !t || !v0 || !E0) return set_error(DQ_EINVAL, "NULL argument");
    if (t->sector != s) return set_error(DQ_EINVAL, "terms were compiled for another sector");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    if (steps < 1) return set_error(DQ_EINVAL, "steps must be >= 1");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64)
        return run_lanczos<double>(s, t, (const double*)v0, steps, reorth, E0, alpha, beta, steps_done, st);
    return run_lanczos<float>(s, t, (const float*)v0, steps, reorth, E0, alpha, beta, steps_done, st);
}
