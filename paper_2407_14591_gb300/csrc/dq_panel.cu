// Panel product y = H x for Q = 2 and two subsystems (plan in dq_panel.cpp).
//
// Arithmetic. FP64 work runs at a small fraction of the integer rate on this GPU, so the sums
// are exact integer sums: a prepass scales x by 2^F (F from the largest exponent in x) and
// rounds it to int64 (FP64 input, |X| < 2^56) or int32 (FP32 input, |X| < 2^30); every hop adds
// an integer; the row result sum_k M_k T_k (coefficients M_k = c_k / 2^emin, integers) is formed
// in 128-bit integers and rounded once to the output type. The only error is the rounding of
// x to 2^-F, at most 2^-57 (FP64) or 2^-31 (FP32) of max|x| per term.
//
// Data movement. One CTA per panel (all rows with one P_0 pattern s0, contiguous in the
// canonical order), persistent over panels. The panel of x is loaded into shared memory; hops
// inside P_1 are shared-memory gathers through the P_1 rank table (also in shared memory); hops
// inside P_0 read the partner panel element by element (coalesced); hops across the cut read the
// panel s0 ^ bit_a of the neighbouring block from a ring of shared-memory slots filled by bulk
// (TMA) copies, two in flight for FP64 and five for FP32. The last warp done with a slot starts
// its next copy, so the warps never wait for each other inside a panel. Gathers of inactive hops
// are not skipped but pointed at a slot that holds zero: no branches, and all such lanes read one
// address. Every y element is written once, by one thread.
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "dq_fixed.cuh"
#include "dq_internal.h"


namespace dq {

// threads per panel CTA: 1024 (one CTA per SM) for panels of more than 1024 rows, else 512 (two
// CTAs per SM, each thread on at most two rows)
constexpr int kPT = 1024;
constexpr int kPTSmall = 512;
constexpr unsigned kWaitLimit = 1u << 22;

// ------------------------------------------------------------------ mbarrier / bulk copy -----

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Bulk copy of `bytes` (multiple of 16) from 16-byte aligned global memory into shared memory,
// completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of `bar`. On timeout it raises the block's abort flag, after
// which every wait of the block returns false at once: a lost copy costs one time limit, not one
// per wait.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (*abort_flag) return false;
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        if (bar_try(bar, parity)) return true;
        if ((it & 63u) == 63u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// Copy the panel of `len` elements starting at global index `start` into `buf`; returns the
// offset of element 0 inside `buf` (the copy starts at the 16-byte boundary below `start`).
template <typename XT>
__device__ __forceinline__ int stage(XT* buf, const XT* X, uint64_t start, int len, uint64_t* bar) {
    constexpr int per16 = 16 / sizeof(XT);
    uint64_t a0 = start & ~(uint64_t)(per16 - 1);
    int off = (int)(start - a0);
    uint32_t bytes = (uint32_t)(((off + len) * sizeof(XT) + 15) & ~(size_t)15);
    bulk_load(buf, X + a0, bytes, bar);
    return off;
}

// ------------------------------------------------------------------ panel kernel -------------

// Shared-memory layout of the panel kernel:
//   [0, kT1Bytes)  the P_1 rank table (local index of every pattern, as a byte offset) and, at
//                  kZeroSlot, one entry that points at a zero element;
//   kOwn + s * bstride, s < R: R slots of cap + 8 elements. Slot 0 holds the panel's own x, slots
//                  1 .. R-1 are the ring of cut partners. Elements cap - 1 .. cap + 6 of every
//                  slot stay zero (no copy reaches them).
//   then R mbarriers and the panel's source list.
// A table entry is a byte offset into a slot, so a gather is two loads with no address arithmetic.
constexpr int kT1Entries = 1 << 15;
constexpr uint32_t kZeroSlot = 2 * kT1Entries;  // byte offset of the zero-slot entry
constexpr int kT1Bytes = 2 * kT1Entries + 128;
constexpr int kOwn = kT1Bytes;
constexpr int kZeroPad = 8;
template <typename XT>
struct PanelSmem {
    static __host__ __device__ size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
    static __host__ __device__ size_t buf_bytes(int cap) { return al((size_t)(cap + kZeroPad) * sizeof(XT)); }
    static __host__ __device__ size_t total(int cap, int nslots) {
        return kT1Bytes + (size_t)nslots * buf_bytes(cap) + 128 + 8 * kPanelMaxList;
    }
};

template <typename XT>
__device__ __forceinline__ long long lds_x(const unsigned char* sm, uint32_t off) {
    return (long long)*reinterpret_cast<const XT*>(sm + off);
}
__device__ __forceinline__ uint32_t lds_u16(const unsigned char* sm, uint32_t off) {
    return (uint32_t)*reinterpret_cast<const uint16_t*>(sm + off);
}

struct PanelCtx {
    uint32_t s0;
    uint64_t start;
    int n1, C, ncls0, np0, nx;
};

// Block-shared bookkeeping of the copy ring.
template <int R>
struct Ring {
    int done[R];   // warps finished with each slot's current contents
    int issued[R]; // copies started into each slot (for the drain after a timeout)
    int abort;     // a wait timed out
};

// Start the copy of cut partner j (entry np0 + j of the source list) into slot s.
template <typename XT, int R>
__device__ __forceinline__ void issue_cut(int j, int s, const PanelPlan& P, const PanelCtx& pc, const XT* X,
                                          unsigned char* smem, size_t bstride, uint64_t* bar, const uint64_t* lst,
                                          Ring<R>& rg) {
    const uint64_t ent = lst[pc.np0 + j];
    const int g = (int)(ent >> 48);
    const int len = (int)P.t1len[pc.n1 + ((pc.s0 & P.xg_abit[g]) ? 1 : -1)];
    stage(reinterpret_cast<XT*>(smem + kOwn + s * bstride), X, ent & ((1ull << 48) - 1), len, &bar[s]);
    rg.issued[s] += 1;
}

// Every warp calls this when it has finished reading slot s; the last of the block's warps
// starts the copy of cut partner jn into it (if there is one). No block-wide barrier: the other
// warps go on with their next slot.
template <typename XT, int R, int NT>
__device__ __forceinline__ void release_slot(int s, int jn, const PanelPlan& P, const PanelCtx& pc, const XT* X,
                                             unsigned char* smem, size_t bstride, uint64_t* bar, const uint64_t* lst,
                                             Ring<R>& rg) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();  // this warp's reads of the slot happen before the count
        if (atomicAdd(&rg.done[s], 1) == NT / 32 - 1) {
            rg.done[s] = 0;
            __threadfence_block();
            if (jn < pc.nx && !rg.abort) issue_cut<XT, R>(jn, s, P, pc, X, smem, bstride, bar, lst, rg);
        }
    }
}

// All the work of one panel for rows tid + e * NT, e < E. Rows past the panel hold s = 0: their
// gathers read in-range entries, and they are never stored.
template <typename XT, typename OUT, int NA, int R, int E, int NT>
__device__ __forceinline__ void panel_rows(const PanelPlan& P, const XT* __restrict__ X, OUT* __restrict__ y,
                                           unsigned char* smem, uint64_t* bar, const uint64_t* lst, const PanelDiag& dg,
                                           const PanelCtx& pc, size_t bstride, uint32_t& ph, int scale, int& fail,
                                           Ring<R>& rg) {
    const int tid = threadIdx.x;
    const unsigned char* own = smem + kOwn;
    uint32_t s2[E];  // P_1 pattern of each row, shifted left by one (rank-table byte offset)
    long long acc[NA][E];
    const uint16_t* st = P.t1states + P.t1start[pc.n1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int c = tid + e * NT;
        s2[e] = c < pc.C ? ((uint32_t)__ldg(st + c) << 1) : 0u;
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k][e] = 0;
    }
    // The work of the panel in units that need no copy: P_0 partner panels two at a time (per
    // amplitude class), and P_1 bond layers. They are interleaved with the cross partners of
    // the copy ring, so that each bulk copy lands while the warps work on units.
    // P_0 partner panels per unit: two, or four when a thread has at most two rows (more loads
    // in flight per thread)
    constexpr int kP0 = NT == kPT ? 2 : 4;
    const int n0a = (pc.ncls0 + kP0 - 1) / kP0;                  // class-0 P_0 units
    const int n0u = n0a + (pc.np0 - pc.ncls0 + kP0 - 1) / kP0;  // all P_0 units
    const int nu = n0u + P.n_p1l;
    auto p0_unit = [&](auto kc, int l, int l1) {
        constexpr int k = decltype(kc)::value;
        if constexpr (kP0 != 2) {
            if (l + kP0 <= l1) {
                const XT* src[kP0];
#pragma unroll
                for (int q = 0; q < kP0; ++q) src[q] = X + lst[l + q];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int c = tid + e * NT;
                    if (c < pc.C) {
                        long long a = 0;
#pragma unroll
                        for (int q = 0; q < kP0; ++q) a += (long long)__ldg(src[q] + c);
                        acc[k][e] += a;
                    }
                }
            } else {
                for (; l < l1; ++l) {
                    const XT* src = X + lst[l];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int c = tid + e * NT;
                        if (c < pc.C) acc[k][e] += (long long)__ldg(src + c);
                    }
                }
            }
        } else if (l + 1 < l1) {
            const XT* src = X + lst[l];
            const XT* src2 = X + lst[l + 1];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = tid + e * NT;
                if (c < pc.C) acc[k][e] += (long long)__ldg(src + c) + (long long)__ldg(src2 + c);
            }
        } else {
            const XT* src = X + lst[l];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = tid + e * NT;
                if (c < pc.C) acc[k][e] += (long long)__ldg(src + c);
            }
        }
    };
    // hops inside P_1, one bond layer of distance d: s ^ (s >> d) marks the active pairs; rows
    // whose pair is not active read the zero slot (one address for all of them, so no bank
    // conflicts and no branch)
    auto run_unit = [&](int u) {
        if (u < n0a) {
            p0_unit(std::integral_constant<int, 0>(), kP0 * u, pc.ncls0);
        } else if (u < n0u) {
            if constexpr (NA > 1) p0_unit(std::integral_constant<int, NA - 1>(), pc.ncls0 + kP0 * (u - n0a), pc.np0);
        } else {
            const int l = u - n0u, d = P.p1l_d[l];
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const int q0 = k ? P.p1l_cut[l] : P.p1l_first[l], q1 = k ? P.p1l_end[l] : P.p1l_cut[l];
                for (int q = q0; q < q1; ++q) {
                    const uint32_t lb = P.p1b_lobit[q] << 1, pm2 = P.p1b_pm2[q];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const uint32_t t = ((s2[e] ^ (s2[e] >> d)) & lb) ? (s2[e] ^ pm2) : kZeroSlot;
                        acc[k][e] += lds_x<XT>(own, lds_u16(smem, t));
                    }
                }
            }
        }
    };
    int u = 0;
    const int lead = pc.nx ? (nu < 2 ? nu : 2) : nu;  // units before the first cross partner
    for (; u < lead; ++u) run_unit(u);
    int target = lead, frac = 0;
    // hops across the cut: panel s0 ^ bit_a of the neighbouring block, in the copy ring
    for (int j = 0; j < pc.nx; ++j) {
        const int s = 1 + j % (R - 1);
        if (!bar_wait(&bar[s], (ph >> s) & 1u, &rg.abort)) fail = 1;
        ph ^= 1u << s;
        const uint64_t ent = lst[pc.np0 + j];
        const int g = (int)(ent >> 48);
        const unsigned char* sp = smem + kOwn + s * bstride + (ent & (16 / sizeof(XT) - 1)) * sizeof(XT);
        // a hop needs s_b != s_a: with s_a = 1 the particle moves a -> b (b empty); rows whose
        // pair is not active read the zero slot
        const uint32_t flip = (pc.s0 & P.xg_abit[g]) ? ~0u : 0u;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int b0 = k ? P.xg_cut[g] : P.xg_first[g];
            const int b1 = k ? P.xg_end[g] : P.xg_cut[g];
            for (int q = b0; q < b1; ++q) {
                const uint32_t bb2 = P.xb_bit[q] << 1;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t t = ((s2[e] ^ flip) & bb2) ? (s2[e] ^ bb2) : kZeroSlot;
                    acc[k][e] += lds_x<XT>(sp, lds_u16(smem, t));
                }
            }
        }
        release_slot<XT, R, NT>(s, j + R - 1, P, pc, X, smem, bstride, bar, lst, rg);
        // target = lead + floor((nu - lead) (j + 1) / nx), kept incrementally
        frac += nu - lead;
        while (frac >= pc.nx) {
            frac -= pc.nx;
            ++target;
        }
        for (; u < target; ++u) run_unit(u);
    }
    for (; u < nu; ++u) run_unit(u);
    // the row result: (C + sum_k K_k n_k) x_i + sum_k A_k S_k, exactly, rounded once
    const uint32_t m1 = (1u << P.L1) - 1u;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int c = tid + e * NT;
        if (c >= pc.C) continue;
        const uint32_t s = s2[e] >> 1;
        long long md = P.MC;
#pragma unroll
        for (int k = 0; k < kPanelMaxK; ++k) {
            if (k >= P.nK) break;
            long long n = dg.cnt0[k];
            for (int l = (k ? P.p1z_end[k - 1] : 0); l < P.p1z_end[k]; ++l)
                n += __popc((s ^ (s >> P.p1z_d[l])) & P.p1z_mask[l]);
#pragma unroll
            for (int q = 0; q < 3; ++q) n += (long long)(__popc(s & dg.w0[k][q]) + __popc(~s & m1 & dg.w1[k][q])) << q;
            md += P.MK[k] * n;
        }
        I128 r = {0, 0};
        mac(r, md, lds_x<XT>(own, (uint32_t)(c * sizeof(XT))));
#pragma unroll
        for (int k = 0; k < NA; ++k) mac(r, P.MA[k], acc[k][e]);
        y[pc.start + c] = i128_to<OUT>(r, scale);
    }
}

template <typename XT, typename OUT, int NA, int R, int NT>
__global__ void __launch_bounds__(NT, kPT / NT)
    k_panel(PanelPlan P, const XT* __restrict__ X, OUT* __restrict__ y, const WsHeader* __restrict__ h, int* err,
            int cap) {
    extern __shared__ __align__(128) unsigned char smem[];
    using SL = PanelSmem<XT>;
    const int tid = threadIdx.x;
    uint16_t* t1 = reinterpret_cast<uint16_t*>(smem);
    XT* own = reinterpret_cast<XT*>(smem + kOwn);
    const size_t bstride = SL::buf_bytes(cap);
    unsigned char* tail = smem + kOwn + (size_t)R * bstride;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tail);  // [s]: copy slot s
    uint64_t* lst = reinterpret_cast<uint64_t*>(tail + 128);
    __shared__ uint32_t s_hdr;
    __shared__ int s_fail;
    __shared__ PanelDiag dg;
    __shared__ Ring<R> rg;
    const uint16_t zoff = (uint16_t)((cap - 1) * sizeof(XT));  // byte offset of a zero element

    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            bar_init(&bar[s]);
            rg.done[s] = 0;
            rg.issued[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        rg.abort = 0;
        s_fail = 0;
        t1[kT1Entries] = zoff;
    }
    if (tid < kZeroPad * R) reinterpret_cast<XT*>(smem + kOwn + (tid / kZeroPad) * bstride)[cap - 1 + tid % kZeroPad] = 0;
    for (int q = tid; q < (1 << P.L1); q += NT) t1[q] = (uint16_t)(__ldg(P.t1rank + q) * sizeof(XT));
    __syncthreads();
    if (h->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint32_t pi = blockIdx.x; pi < P.npanels; pi += gridDim.x) {
            const uint64_t st = P.panel_start[pi];
            const int C = (int)P.t1len[P.N - __popc(P.panel_s0[pi])];
            for (int c = tid; c < C; c += NT) y[st + c] = (OUT)NAN;
        }
        if (blockIdx.x == 0 && tid == 0) atomicAdd(err, 1);
        return;
    }
    const int scale = P.emin - h->F;
    uint32_t ph = 0u;  // mbarrier parity of each slot (bit s)
    int fail = 0;

    for (uint32_t pi = blockIdx.x; pi < P.npanels; pi += gridDim.x) {
        PanelCtx pc;
        pc.s0 = P.panel_s0[pi];
        pc.start = P.panel_start[pi];
        pc.n1 = P.N - __popc(pc.s0);
        pc.C = (int)P.t1len[pc.n1];
        // warp 0: source list into shared memory and the first copies; warp 1: diagonal counters
        if (tid < 32) {
            const uint32_t lo = __ldg(P.list_off + pi), hi = __ldg(P.list_off + pi + 1);
            for (uint32_t q = lo + tid; q < hi; q += 32) lst[q - lo] = __ldg(P.list + q);
            if (tid == 0) s_hdr = __ldg(P.list_hdr + pi);
            __syncwarp();
            if (tid == 0) {
                const uint32_t hd = s_hdr;
                PanelCtx pq = pc;
                pq.np0 = (int)(hd & 255u) + (int)((hd >> 8) & 255u);
                pq.nx = (int)((hd >> 16) & 255u);
                for (int j = 0; j < pq.nx && j < R - 1; ++j)
                    issue_cut<XT, R>(j, 1 + j, P, pq, X, smem, bstride, bar, lst, rg);
            }
        } else if (tid < 32 + (int)(sizeof(PanelDiag) / 4)) {
            // the panel's diagonal counters, built on the host
            reinterpret_cast<uint32_t*>(&dg)[tid - 32] = __ldg(reinterpret_cast<const uint32_t*>(P.diag + pi) + tid - 32);
        }
        // the panel's own x: plain coalesced loads into slot 0 (element c at kOwn + c*size)
        {
            const XT* src = X + pc.start;
            for (int c = tid; c < pc.C; c += NT) own[c] = __ldg(src + c);
        }
        __syncthreads();
        const uint32_t hd = s_hdr;
        pc.ncls0 = (int)(hd & 255u);
        pc.np0 = pc.ncls0 + (int)((hd >> 8) & 255u);
        pc.nx = (int)((hd >> 16) & 255u);
        // rows per thread: the smallest E with E * NT >= C (every E from 1 to 7 is compiled for
        // 1024 threads; 512-thread CTAs take panels of at most 1024 rows)
        if constexpr (NT == kPT) {
            switch ((pc.C + NT - 1) / NT) {
                case 7: panel_rows<XT, OUT, NA, R, 7, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                case 6: panel_rows<XT, OUT, NA, R, 6, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                case 5: panel_rows<XT, OUT, NA, R, 5, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                case 4: panel_rows<XT, OUT, NA, R, 4, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                case 3: panel_rows<XT, OUT, NA, R, 3, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                case 2: panel_rows<XT, OUT, NA, R, 2, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg); break;
                default: panel_rows<XT, OUT, NA, R, 1, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg);
            }
        } else {
            if (pc.C > NT)
                panel_rows<XT, OUT, NA, R, 2, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg);
            else
                panel_rows<XT, OUT, NA, R, 1, NT>(P, X, y, smem, bar, lst, dg, pc, bstride, ph, scale, fail, rg);
        }
        __syncthreads();
    }
    if (fail) s_fail = 1;
    __syncthreads();
    if (tid == 0 && (s_fail || rg.abort)) {
        atomicAdd(err, 1);
        // after a timeout, wait (bounded) for the copies still in flight before the block exits
        for (int s = 0; s < R; ++s)
            if (rg.issued[s] > 0)
                for (unsigned it = 0; it < kWaitLimit && !bar_try(&bar[s], (uint32_t)(rg.issued[s] - 1) & 1u); ++it) {
                }
    }
}

// ------------------------------------------------------------------ launch -------------------

size_t panel_scratch_bytes(const dq_sector* s, int dtype) {
    size_t es = dtype == DQ_F64 ? 8 : 4;
    return 256 + ((size_t)(s->D + 8) * es + 255) / 256 * 256;
}

static int sms_count() { return sm_count_cached(); }

template <typename T, typename XT, int NA, int R, int NT>
static int run_panel(const dq_sector* s, const dq_terms* t, const T* x, T* y, void* ws, cudaStream_t st) {
    const PanelPlan& P = t->pp;
    WsHeader* h = reinterpret_cast<WsHeader*>(ws);
    XT* X = reinterpret_cast<XT*>(reinterpret_cast<char*>(ws) + 256);
    cudaMemsetAsync(h, 0, sizeof(WsHeader), st);
    const int sms = sms_count();
    k_exp_max<T><<<sms * 8, 256, 0, st>>>(x, s->D, h);
    k_to_fixed<T, XT><<<sms * 8, 256, 0, st>>>(x, X, s->D, h);
    const int cap = P.cmax + 16 / (int)sizeof(XT) + 4;
    size_t sm = PanelSmem<XT>::total(cap, R);
    auto kern = k_panel<XT, T, NA, R, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 1;
    if (NT != kPT && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm)) != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    const uint32_t slots = (uint32_t)sms * (uint32_t)per_sm;
    unsigned grid = (unsigned)(P.npanels < slots ? P.npanels : slots);
    const int tslot = timing_start(st);
    kern<<<grid, NT, sm, st>>>(P, X, y, h, s->dev.err, cap);
    timing_stop(tslot, st, 3);
    return (int)cudaGetLastError();
}

template <typename T, typename XT, int NA>
static int run_panel_n(const dq_sector* s, const dq_terms* t, const T* x, T* y, void* ws, cudaStream_t st) {
    // copy slots (the panel's own buffer and the staging buffers) that fit next to the rank
    // table in 227 KB of shared memory; panels of at most 1024 rows run two 512-thread CTAs per
    // SM, with six slots when two such CTAs still fit in one SM's shared memory
    if (t->pp.cmax <= 2 * kPTSmall) {
        const int cap = t->pp.cmax + 16 / (int)sizeof(XT) + 4;
        if (2 * (PanelSmem<XT>::total(cap, 6) + 2048) <= 232448)
            return run_panel<T, XT, NA, 6, kPTSmall>(s, t, x, y, ws, st);
        return run_panel<T, XT, NA, 3, kPTSmall>(s, t, x, y, ws, st);
    }
    return run_panel<T, XT, NA, sizeof(XT) == 8 ? 3 : 6, kPT>(s, t, x, y, ws, st);
}

int launch_panel_matvec_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* ws,
                           void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int na = t->pp.nA;
    if (dtype == DQ_F64) {
        if (na <= 1) return run_panel_n<double, long long, 1>(s, t, (const double*)x, (double*)y, ws, st);
        return run_panel_n<double, long long, 2>(s, t, (const double*)x, (double*)y, ws, st);
    }
    if (na <= 1) return run_panel_n<float, int, 1>(s, t, (const float*)x, (float*)y, ws, st);
    return run_panel_n<float, int, 2>(s, t, (const float*)x, (float*)y, ws, st);
}

int launch_panel_matvec(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream) {
    size_t need = panel_scratch_bytes(s, dtype);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    return launch_panel_matvec_ws(s, t, x, y, dtype, t->scratch, stream);
}

}  // namespace dq
