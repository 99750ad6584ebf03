// Batched product: y_k = H_k x_k for up to 64 sectors of uneven dimension (different L, N and
// disorder), each with nrhs right-hand sides, in ONE persistent launch.
//
// The rows of all sectors are cut into tiles; tile t belongs to the sector k with
// prefix[k] <= t < prefix[k+1]. CTAs pull tiles from an atomic queue (a counter cleared before
// each launch), copy the descriptor of the tile's sector into shared memory when the sector
// changes, and run the general Q = 2 row computation (bond layers, rank by Eq. (index) or Lin's
// two tables, gather of the nrhs values of x[j], one store of y[i]). Two row mappings:
//   rows    -- the threads of the CTA take the tile's rows with a block stride, each row
//              unranked with Alg. 4;
//   walk    -- each warp takes 32 R consecutive rows, lane l the rows l, l + 32, ..., the next
//              row of a lane from the last subsystem's unrank list (RowWalk: one Alg. 4 per
//              lane and tile).
// The autotuner times every (mapping, threads, CTAs per SM, tile) candidate on the caller's
// vectors and keeps the fastest.
//
// Arithmetic: FP64 vectors accumulate in FP64. FP32 vectors use the FP32 copies of the
// coefficients, form products in FP32 and sum them with Neumaier's compensated summation, so the
// error of each row sum stays at about one FP32 rounding instead of growing with its length.
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "dq_device.cuh"
#include "dq_internal.h"

namespace dq {

constexpr int kBatchMax = 64;
constexpr int kBatchMaxRhs = 8;

struct BatchItem {
    DevSector S;
    DevTermsQ2 H;
};

struct BatchParams {
    int n, nrhs, rows_per_tile, R;  // R: rows per lane of the walk mapping
    unsigned long long total_tiles;
    unsigned long long* queue;      // next tile (cleared before the launch)
    unsigned long long prefix[kBatchMax + 1];  // first tile of each sector
    const BatchItem* items;
    const void* x[kBatchMax];
    void* y[kBatchMax];
};

// Coefficient in the vectors' precision (FP64 vectors: the FP64 value; FP32: its FP32 copy).
template <typename T>
__device__ __forceinline__ T bcf(double d, float f) {
    if constexpr (sizeof(T) == 8)
        return d;
    else
        return f;
}

template <typename T>
__device__ __forceinline__ void load_rhs(const T* p, int nr, T* v) {
#pragma unroll
    for (int c = 0; c < kBatchMaxRhs; ++c) v[c] = c < nr ? __ldg(p + c) : (T)0;
}

// Row i (word s) of sector (S, H): y[i, :] = sum_j H_ij x[j, :] for the nr right-hand sides.
template <typename T>
__device__ __forceinline__ void batch_row(const DevSector& S, const DevTermsQ2& H, const T* __restrict__ x,
                                          T* __restrict__ y, int nr, uint64_t i, uint64_t s) {
    const bool lin2 = S.n_sub == 2;
    const T* posT = sizeof(T) == 8 ? (const T*)H.pos : (const T*)H.posf;
    // diagonal: FP64 vectors in FP64; FP32 vectors with FP32 coefficients, compensated
    T dv;
    if constexpr (sizeof(T) == 8) {
        double d = H.C;
        if (H.lin) {
            uint64_t m = s;
            while (m) {
                int p = __ffsll((long long)m) - 1;
                m &= m - 1;
                d += __ldg(H.lin + p);
            }
        }
        for (int l = 0; l < H.nl; ++l) {
            uint64_t a = (s ^ (s >> H.dist[l])) & H.dmask[l];
            if (H.kpos[l] < 0) {
                d += __ldg(H.KA + l) * (double)__popcll(a);
            } else {
                while (a) {
                    int p = __ffsll((long long)a) - 1;
                    a &= a - 1;
                    d += __ldg(H.pos + H.kpos[l] + p);
                }
            }
        }
        dv = d;
    } else {
        RowAcc<float> d;
        d.init(H.Cf);
        if (H.linf) {
            uint64_t m = s;
            while (m) {
                int p = __ffsll((long long)m) - 1;
                m &= m - 1;
                d.add(__ldg(H.linf + p));
            }
        }
        for (int l = 0; l < H.nl; ++l) {
            uint64_t a = (s ^ (s >> H.dist[l])) & H.dmask[l];
            if (H.kpos[l] < 0) {
                if (a) d.add(__ldg(H.KAf + l) * (float)__popcll(a));
            } else {
                while (a) {
                    int p = __ffsll((long long)a) - 1;
                    a &= a - 1;
                    d.add(__ldg(H.posf + H.kpos[l] + p));
                }
            }
        }
        dv = d.get();
    }
    T xv[kBatchMaxRhs];
    load_rhs(x + i * nr, nr, xv);
    RowAcc<T> acc[kBatchMaxRhs];
#pragma unroll
    for (int c = 0; c < kBatchMaxRhs; ++c) acc[c].init(c < nr ? dv * xv[c] : (T)0);
    for (int l = 0; l < H.nl; ++l) {
        uint64_t o = (s ^ (s >> H.dist[l])) & H.omask[l];
        const uint64_t pm = 1ull | (1ull << H.dist[l]);
        const T au = bcf<T>(__ldg(H.KA + kMaxLayers + l), __ldg(H.KAf + kMaxLayers + l));
        while (o) {
            int p = __ffsll((long long)o) - 1;
            o &= o - 1;
            const uint64_t s2 = s ^ (pm << p);
            const uint64_t j = lin2 ? d_rank_lin2(S, s2) : d_rank(S, S.off, S.str, s2);
            const T amp = H.apos[l] < 0 ? au : __ldg(posT + H.apos[l] + p);
            load_rhs(x + j * nr, nr, xv);
#pragma unroll
            for (int c = 0; c < kBatchMaxRhs; ++c)
                if (c < nr) acc[c].add(amp * xv[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kBatchMaxRhs; ++c)
        if (c < nr) y[i * nr + c] = acc[c].get();
}

template <typename T, bool WALK>
__global__ void __launch_bounds__(512) k_batch(BatchParams bp) {
    __shared__ BatchItem it;
    __shared__ unsigned long long s_tile;
    int cur = -1;  // sector whose descriptor is in `it` (same value in every thread)
    const int nr = bp.nrhs;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(bp.queue, 1ull);
        __syncthreads();
        const unsigned long long tile = s_tile;
        if (tile >= bp.total_tiles) break;
        int k = 0;
        while (k + 1 < bp.n && bp.prefix[k + 1] <= tile) ++k;
        if (k != cur) {  // uniform across the CTA
            const uint32_t* src = reinterpret_cast<const uint32_t*>(bp.items + k);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&it);
            for (int q = threadIdx.x; q < (int)(sizeof(BatchItem) / 4); q += blockDim.x) dst[q] = src[q];
            __syncthreads();
            cur = k;
        }
        const DevSector& S = it.S;
        const DevTermsQ2& H = it.H;
        const T* x = reinterpret_cast<const T*>(bp.x[k]);
        T* y = reinterpret_cast<T*>(bp.y[k]);
        const unsigned long long r0 = (tile - bp.prefix[k]) * (unsigned long long)bp.rows_per_tile;
        const unsigned long long r1 = min(r0 + (unsigned long long)bp.rows_per_tile, (unsigned long long)S.D);
        if (WALK) {
            const unsigned long long w0 = r0 + (unsigned long long)(threadIdx.x >> 5) * 32ull * bp.R;
            RowWalk<uint64_t> rw;
            unsigned long long i = w0 + (threadIdx.x & 31);
            for (int r = 0; r < bp.R && i < r1; ++r, i += 32) {
                if (r == 0)
                    walk_start(S, S.off, S.str, i, rw);
                else
                    walk_next(S, S.off, S.str, i, rw);
                batch_row<T>(S, H, x, y, nr, i, rw.s);
            }
        } else {
            for (unsigned long long i = r0 + threadIdx.x; i < r1; i += blockDim.x)
                batch_row<T>(S, H, x, y, nr, i, d_unrank(S, S.off, S.str, i));
        }
        __syncthreads();  // everyone is done with `it` and s_tile before they change
    }
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Candidates of the autotuner: (mapping 0 = rows, 1 = walk; threads; CTAs per SM; rows per
// tile; rows per lane R of the walk mapping, tile = threads * R).
struct Shape {
    int walk, threads, per_sm, tile, R;
};
static const Shape kShapes[] = {{0, 128, 8, 2048, 0}, {0, 256, 4, 4096, 0}, {0, 256, 8, 2048, 0},
                                {0, 512, 2, 8192, 0}, {0, 512, 4, 4096, 0}, {0, 256, 4, 16384, 0},
                                {1, 128, 8, 1024, 8}, {1, 256, 4, 2048, 8}, {1, 256, 8, 1024, 4},
                                {1, 512, 2, 8192, 16}, {1, 256, 4, 4096, 16}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

}  // namespace dq

struct dq_batch {
    int n, nrhs, dtype, shape;
    std::vector<unsigned long long> dims;
    void* items;  // device array of BatchItem, then the tile counter of the work queue
    int device;
};

using namespace dq;

static int batch_launch(dq_batch* b, const void* const* x, void* const* y, cudaStream_t st, int shape) {
    const Shape& sh = kShapes[shape];
    BatchParams bp;
    std::memset(&bp, 0, sizeof bp);
    bp.n = b->n;
    bp.nrhs = b->nrhs;
    bp.rows_per_tile = sh.tile;
    bp.R = sh.R;
    bp.items = reinterpret_cast<const BatchItem*>(b->items);
    bp.queue = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(b->items) + sizeof(BatchItem) * b->n);
    unsigned long long t = 0;
    for (int k = 0; k < b->n; ++k) {
        bp.prefix[k] = t;
        t += (b->dims[k] + sh.tile - 1) / sh.tile;
        bp.x[k] = x[k];
        bp.y[k] = y[k];
    }
    bp.prefix[b->n] = t;
    bp.total_tiles = t;
    unsigned long long cap = (unsigned long long)sm_count() * sh.per_sm;
    unsigned grid = (unsigned)(t < cap ? (t ? t : 1) : cap);
    cudaMemsetAsync(bp.queue, 0, sizeof(unsigned long long), st);
    const int tslot = timing_start(st);
    if (b->dtype == DQ_F64) {
        if (sh.walk)
            k_batch<double, true><<<grid, sh.threads, 0, st>>>(bp);
        else
            k_batch<double, false><<<grid, sh.threads, 0, st>>>(bp);
    } else {
        if (sh.walk)
            k_batch<float, true><<<grid, sh.threads, 0, st>>>(bp);
        else
            k_batch<float, false><<<grid, sh.threads, 0, st>>>(bp);
    }
    timing_stop(tslot, st, 1);
    return (int)cudaGetLastError();
}

extern "C" {

int dq_batch_make(int n, const dq_sector* const* sectors, const dq_terms* const* terms, int nrhs, int dtype,
                  dq_batch** out) {
    clear_error();
    if (!out || !sectors || !terms) return set_error(DQ_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1 || n > kBatchMax) return set_error(DQ_EINVAL, "n must be in [1, %d]", kBatchMax);
    if (nrhs < 1 || nrhs > kBatchMaxRhs) return set_error(DQ_EINVAL, "nrhs must be in [1, %d]", kBatchMaxRhs);
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    std::vector<BatchItem> host(n);
    dq_batch* b = new (std::nothrow) dq_batch();
    if (!b) return set_error(DQ_ENOMEM, "host allocation");
    b->n = n;
    b->nrhs = nrhs;
    b->dtype = dtype;
    b->shape = 1;
    b->items = nullptr;
    for (int k = 0; k < n; ++k) {
        const dq_sector* s = sectors[k];
        const dq_terms* t = terms[k];
        if (!s || !t || t->sector != s) {
            delete b;
            return set_error(DQ_EINVAL, "item %d: NULL or terms of another sector", k);
        }
        if (!s->has_device) {
            delete b;
            return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
        }
        if (!t->q2) {
            delete b;
            return set_error(DQ_EINVAL, "item %d: the batched product serves Q = 2 sectors of one-word states", k);
        }
        host[k].S = s->dev;
        host[k].H = t->q2v;
        b->dims.push_back(s->D);
    }
    cudaError_t e = cudaMalloc(&b->items, sizeof(BatchItem) * n + sizeof(unsigned long long));
    if (e != cudaSuccess) {
        delete b;
        return set_error(DQ_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(b->items, host.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->items);
        delete b;
        return set_error(DQ_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    cudaGetDevice(&b->device);
    *out = b;
    return DQ_OK;
}

void dq_batch_free(dq_batch* b) {
    if (!b) return;
    cudaFree(b->items);
    delete b;
}

int dq_batch_matvec(dq_batch* b, const void* const* x, void* const* y, void* stream) {
    clear_error();
    if (!b || !x || !y) return set_error(DQ_EINVAL, "NULL argument");
    for (int k = 0; k < b->n; ++k)
        if (!x[k] || !y[k]) return set_error(DQ_EINVAL, "item %d: NULL vector", k);
    int e = batch_launch(b, x, y, (cudaStream_t)stream, b->shape);
    if (e) return set_error(DQ_ECUDA, "batch launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}

int dq_batch_shape(dq_batch* b, int shape, int* n_shapes) {
    clear_error();
    if (!b) return set_error(DQ_EINVAL, "NULL argument");
    if (n_shapes) *n_shapes = kNumShapes;
    if (shape < 0) return DQ_OK;
    if (shape >= kNumShapes) return set_error(DQ_EINVAL, "shape must be in [0, %d)", kNumShapes);
    b->shape = shape;
    return DQ_OK;
}

int dq_batch_tune(dq_batch* b, const void* const* x, void* const* y, void* stream, int* choice) {
    clear_error();
    if (!b || !x || !y) return set_error(DQ_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_i = b->shape;
    for (int i = 0; i < kNumShapes; ++i) {
        int rc = batch_launch(b, x, y, st, i);  // warm-up
        if (rc) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return set_error(DQ_ECUDA, "batch launch: %s", cudaGetErrorString((cudaError_t)rc));
        }
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) batch_launch(b, x, y, st, i);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape = best_i;
    if (choice) *choice = best_i;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "batch tune: %s", cudaGetErrorString(e));
    return DQ_OK;
}

}  // extern "C"
