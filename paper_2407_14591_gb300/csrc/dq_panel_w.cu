// Warp-panel product y = H x for Q = 2 and three or more subsystems (plan in dq_panel.cpp).
//
// Eq. (index) gives the last subsystem P_1 offset 0 and stride 1 inside the block of its particle
// number, so the rows that share the pattern s0 of all other subsystems (the prefix P_0) form a
// contiguous panel of D_2(L_1, N - |s0|) rows in P_1's local order, as with two subsystems. With
// P_1 of 8 to 10 sites a panel has at most 252 rows and there are many of them, so each warp takes
// one panel at a time (8 warps per CTA, persistent over the panel list), and the partner panels
// are ranked on the device, once per panel, by Eq. (index) over the prefix subsystems:
//   - the warp stages its panel of x (fixed point) in its own shared-memory slot;
//   - its lanes test the prefix bonds and the cut groups, rank the partner panels and compact
//     them into a list (warp ballots), and build the panel's diagonal counters;
//   - hops inside P_0 read the partner panel element by element (coalesced global loads);
//   - hops inside P_1 are gathers through the shared rank table (byte offsets into a slot);
//   - hops across the cut stage the partner panel s0 ^ bit_a in the warp's second slot;
//   - inactive pairs read an element that holds zero, so the lanes never branch;
//   - the row result (C + sum_k K_k n_k) X_i + sum_k A_k S_k is formed in 128-bit integers and
//     rounded once, as in the two-subsystem panel kernel.
// No block barrier after the set-up: the warps of a CTA never wait for each other.
#include <cstdint>

#include <cuda_runtime.h>

#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

constexpr int kPWT = 256;                        // threads per CTA (eight warps)
constexpr int kPWWarps = kPWT / 32;
constexpr int kPWCap = 256;                      // rows of the longest panel (P_1 <= 10 sites)
constexpr int kPWTab = 1 << 10;                  // rank-table entries
constexpr uint32_t kPWZero = 2 * kPWTab;         // byte offset of the entry that points at a zero
constexpr int kPWSlot = kPWCap + 8;              // elements per slot; [kPWCap, kPWCap + 8) stay zero

template <typename XT>
struct PWSmem {
    static __host__ __device__ size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
    static __host__ __device__ size_t table() { return al(2 * kPWTab + 16); }
    static __host__ __device__ size_t tables(int os_total) { return al((size_t)os_total * 16); }
    static __host__ __device__ size_t slot() { return al((size_t)kPWSlot * sizeof(XT)); }
    // per warp: two slots, the partner list and the panel's diagonal counters
    static __host__ __device__ size_t warp() { return 2 * slot() + al((size_t)kPanelMaxList * 8) + al(sizeof(PanelDiag)); }
    static __host__ __device__ size_t total(int os_total) { return table() + tables(os_total) + kPWWarps * warp(); }
};

template <typename XT>
__device__ __forceinline__ long long pw_lds(const unsigned char* base, uint32_t off) {
    return (long long)*reinterpret_cast<const XT*>(base + off);
}

// First index of the panel with prefix pattern s0 (its row of local index 0): Eq. (index) over the
// prefix subsystems, plus the offset of the last subsystem's block.
__device__ __forceinline__ uint64_t pw_start(const PWRank& R, const uint64_t* off_s, const uint64_t* str_s,
                                             uint32_t s0) {
    const uint64_t w = (uint64_t)s0 << R.L1;
    uint64_t idx = 0;
    int lam = 0;
    for (int k = 0; k < R.n_sub - 1; ++k) {
        const uint32_t f = (uint32_t)(w >> R.shift[k]) & R.fmask[k];
        const int n = __popc(f);
        const int o = R.os_base[k] + lam * R.os_ld[k] + n;
        idx += off_s[o] + str_s[o] * (uint64_t)__ldg(R.rank[k] + f);
        lam += n;
    }
    const int last = R.n_sub - 1;
    return idx + off_s[R.os_base[last] + lam * R.os_ld[last] + (R.N - lam)];
}

// Per-panel values of one warp (registers, the same in every lane); the diagonal counters
// (PanelDiag) sit in the warp's shared memory.
struct PWPanel {
    uint32_t s0;
    uint64_t start;
    int n1, C;
    int np0[kPanelMaxA];  // P_0 partners of each amplitude class (list entries, in class order)
    uint32_t xvalid;      // cut groups whose partner panel exists (bit g)
};

// The warp's set-up of panel pi: list of partner starts (P_0 partners compacted by class, then one
// entry per cut group) and the diagonal counters (written by lane 0 into dg).
__device__ __forceinline__ void pw_setup(const PanelPlan& P, const PWRank& R, const uint64_t* off_s,
                                         const uint64_t* str_s, uint64_t* lst, PanelDiag* dg, PWPanel& pp, int* err) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t s0 = pp.s0;
    int pos = 0;
#pragma unroll
    for (int k = 0; k < kPanelMaxA; ++k) {
        const int lo = k ? P.p0_end[k - 1] : 0, hi = P.p0_end[k];
        const int before = pos;
        for (int base = lo; base < hi; base += 32) {
            const int l = base + lane;
            const uint32_t m = l < hi ? P.p0_mask[l] : 0u;
            const bool act = l < hi && __popc(s0 & m) == 1;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) {
                uint64_t st = pw_start(R, off_s, str_s, s0 ^ m);
#ifdef DQ_CHECKED
                if (st + (uint64_t)pp.C > R.D) {
                    atomicAdd(err, 1);
                    st = pp.start;
                }
#endif
                lst[pos + __popc(bal & lt)] = st;
            }
            pos += __popc(bal);
        }
        pp.np0[k] = pos - before;
    }
    // cut groups: partner s0 ^ bit_a, one list entry per group
    {
        const int g = lane;
        bool ok = false;
        if (g < P.n_xg) {
            const uint32_t s0p = s0 ^ P.xg_abit[g];
            const int n1p = R.N - __popc(s0p);
            ok = n1p >= 0 && n1p <= R.L1;
            if (ok) {
                uint64_t st = pw_start(R, off_s, str_s, s0p);
#ifdef DQ_CHECKED
                if (st + (uint64_t)P.t1len[n1p] > R.D) {
                    atomicAdd(err, 1);
                    ok = false;
                }
#endif
                lst[pos + g] = st;
            }
        }
        pp.xvalid = __ballot_sync(0xffffffffu, ok);
    }
    // diagonal counters: Sz Sz bonds inside P_0 per class, and per position b of P_1 the cut
    // bonds with s_a = 0 (w0) and s_a = 1 (w1) in three bit planes
#pragma unroll
    for (int k = 0; k < kPanelMaxK; ++k) {
        int c = 0;
        if (k < P.nK) {
            const int lo = k ? P.p0z_end[k - 1] : 0, hi = P.p0z_end[k];
            for (int base = lo; base < hi; base += 32) {
                const int l = base + lane;
                c += __popc(__ballot_sync(0xffffffffu, l < hi && __popc(s0 & P.p0z_mask[l]) == 1));
            }
        }
        const uint32_t am = lane < R.L1 && k < P.nK ? P.xzA[k][lane] : 0u;
        const int c0 = __popc(~s0 & am), c1 = __popc(s0 & am);
        uint32_t b0[3], b1[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            b0[q] = __ballot_sync(0xffffffffu, (c0 >> q) & 1);
            b1[q] = __ballot_sync(0xffffffffu, (c1 >> q) & 1);
        }
        if (lane == 0) {
            dg->cnt0[k] = c;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dg->w0[k][q] = b0[q];
                dg->w1[k][q] = b1[q];
            }
        }
    }
}

// The rows of one panel, rows lane + 32 e (e < E) of the warp.
template <typename XT, typename OUT, int NA, int E>
__device__ __forceinline__ void pw_rows(const PanelPlan& P, const XT* __restrict__ X, OUT* __restrict__ y,
                                        const unsigned char* tab, const unsigned char* own, unsigned char* slot,
                                        const uint64_t* lst, const PanelDiag* dg, const PWPanel& pp, int scale) {
    const int lane = threadIdx.x & 31;
    const int C = pp.C;
    uint32_t s2[E];  // P_1 pattern of each row, shifted left by one (rank-table byte offset)
    long long acc[NA][E];
    const uint16_t* st = P.t1states + P.t1start[pp.n1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        s2[e] = c < C ? ((uint32_t)__ldg(st + c) << 1) : 0u;
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k][e] = 0;
    }
    // hops inside P_0: partner panels element by element, by amplitude class (two partners per
    // round with int32 elements; int64 elements would need more registers than four CTAs per SM
    // leave)
    {
        constexpr int kU = sizeof(XT) == 4 ? 2 : 1;
        int l = 0;
#pragma unroll
        for (int k = 0; k < NA; ++k)
#pragma unroll(kU)
            for (int r = 0; r < pp.np0[k]; ++r, ++l) {
                const XT* src = X + lst[l];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int c = lane + 32 * e;
                    if (c < C) acc[k][e] += (long long)__ldg(src + c);
                }
            }
    }
    // hops inside P_1, one bond layer of distance d at a time
    for (int ly = 0; ly < P.n_p1l; ++ly) {
        const int d = P.p1l_d[ly];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int q0 = k ? P.p1l_cut[ly] : P.p1l_first[ly], q1 = k ? P.p1l_end[ly] : P.p1l_cut[ly];
            for (int q = q0; q < q1; ++q) {
                const uint32_t lb = P.p1b_lobit[q] << 1, pm2 = P.p1b_pm2[q];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t t = ((s2[e] ^ (s2[e] >> d)) & lb) ? (s2[e] ^ pm2) : kPWZero;
                    acc[k][e] += pw_lds<XT>(own, *reinterpret_cast<const uint16_t*>(tab + t));
                }
            }
        }
    }
    // hops across the cut: the partner panel s0 ^ bit_a staged in the warp's second slot
    const int np0 = pp.np0[0] + (NA > 1 ? pp.np0[NA - 1] : 0);
    for (int g = 0; g < P.n_xg; ++g) {
        if (!((pp.xvalid >> g) & 1u)) continue;
        const bool sa = (pp.s0 & P.xg_abit[g]) != 0;
        const int len = (int)P.t1len[sa ? pp.n1 + 1 : pp.n1 - 1];
        const XT* src = X + lst[np0 + g];
        __syncwarp();  // the slot's previous partner is no longer read
        for (int c = lane; c < len; c += 32) reinterpret_cast<XT*>(slot)[c] = __ldg(src + c);
        __syncwarp();
        // a hop needs s_b != s_a: rows whose pair is not active read the zero element
        const uint32_t flip = sa ? ~0u : 0u;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int b0 = k ? P.xg_cut[g] : P.xg_first[g];
            const int b1 = k ? P.xg_end[g] : P.xg_cut[g];
            for (int q = b0; q < b1; ++q) {
                const uint32_t bb2 = P.xb_bit[q] << 1;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t t = ((s2[e] ^ flip) & bb2) ? (s2[e] ^ bb2) : kPWZero;
                    acc[k][e] += pw_lds<XT>(slot, *reinterpret_cast<const uint16_t*>(tab + t));
                }
            }
        }
    }
    // the row result: (C + sum_k K_k n_k) x_i + sum_k A_k S_k, exactly, rounded once
    const uint32_t m1 = (1u << P.L1) - 1u;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        if (c >= C) continue;
        const uint32_t s = s2[e] >> 1;
        long long md = P.MC;
#pragma unroll
        for (int k = 0; k < kPanelMaxK; ++k) {
            if (k >= P.nK) break;
            long long n = dg->cnt0[k];
            for (int l = (k ? P.p1z_end[k - 1] : 0); l < P.p1z_end[k]; ++l)
                n += __popc((s ^ (s >> P.p1z_d[l])) & P.p1z_mask[l]);
#pragma unroll
            for (int q = 0; q < 3; ++q) n += (long long)(__popc(s & dg->w0[k][q]) + __popc(~s & m1 & dg->w1[k][q])) << q;
            md += P.MK[k] * n;
        }
        I128 r = {0, 0};
        mac(r, md, pw_lds<XT>(own, (uint32_t)(c * sizeof(XT))));
#pragma unroll
        for (int k = 0; k < NA; ++k) mac(r, P.MA[k], acc[k][e]);
        y[pp.start + c] = i128_to<OUT>(r, scale);
    }
}

// Four CTAs (32 warps) per SM: at most 64 registers per thread.
template <typename XT, typename OUT, int NA>
__global__ void __launch_bounds__(kPWT, 4) k_panel_w(PanelPlan P, PWRank R, const XT* __restrict__ X, OUT* __restrict__ y,
                                                  const WsHeader* __restrict__ h, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    using SL = PWSmem<XT>;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint16_t* t1 = reinterpret_cast<uint16_t*>(smem);
    uint64_t* off_s = reinterpret_cast<uint64_t*>(smem + SL::table());
    uint64_t* str_s = off_s + R.os_total;
    unsigned char* wbase = smem + SL::table() + SL::tables(R.os_total) + (size_t)wid * SL::warp();
    unsigned char* own = wbase;
    unsigned char* slot = wbase + SL::slot();
    uint64_t* lst = reinterpret_cast<uint64_t*>(wbase + 2 * SL::slot());
    PanelDiag* dg = reinterpret_cast<PanelDiag*>(wbase + 2 * SL::slot() + SL::al((size_t)kPanelMaxList * 8));
    for (int q = tid; q < (1 << P.L1); q += kPWT) t1[q] = (uint16_t)(__ldg(P.t1rank + q) * sizeof(XT));
    if (tid == 0) t1[kPWTab] = (uint16_t)(kPWCap * sizeof(XT));
    for (int q = tid; q < R.os_total; q += kPWT) {
        off_s[q] = __ldg(R.off + q);
        str_s[q] = __ldg(R.str + q);
    }
    if (lane < 8) {
        reinterpret_cast<XT*>(own)[kPWCap + lane] = 0;
        reinterpret_cast<XT*>(slot)[kPWCap + lane] = 0;
    }
    __syncthreads();
    const uint32_t nwarps = gridDim.x * kPWWarps;
    if (h->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint32_t pi = blockIdx.x * kPWWarps + wid; pi < P.npanels; pi += nwarps) {
            const uint64_t st = P.panel_start[pi];
            const int C = (int)P.t1len[P.N - __popc(P.panel_s0[pi])];
            for (int c = lane; c < C; c += 32) y[st + c] = (OUT)NAN;
        }
        if (blockIdx.x == 0 && tid == 0) atomicAdd(err, 1);
        return;
    }
    const int scale = P.emin - h->F;
    for (uint32_t pi = blockIdx.x * kPWWarps + wid; pi < P.npanels; pi += nwarps) {
        PWPanel pp;
        pp.s0 = __ldg(P.panel_s0 + pi);
        pp.start = __ldg(P.panel_start + pi);
        pp.n1 = P.N - __popc(pp.s0);
        pp.C = (int)P.t1len[pp.n1];
        __syncwarp();  // the previous panel's reads of the slots and the list are done
        const XT* src = X + pp.start;
        for (int c = lane; c < pp.C; c += 32) reinterpret_cast<XT*>(own)[c] = __ldg(src + c);
        pw_setup(P, R, off_s, str_s, lst, dg, pp, err);
        __syncwarp();
        switch ((pp.C + 31) >> 5) {
            case 8: pw_rows<XT, OUT, NA, 8>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 7: pw_rows<XT, OUT, NA, 7>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 6: pw_rows<XT, OUT, NA, 6>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 5: pw_rows<XT, OUT, NA, 5>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 4: pw_rows<XT, OUT, NA, 4>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 3: pw_rows<XT, OUT, NA, 3>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            case 2: pw_rows<XT, OUT, NA, 2>(P, X, y, smem, own, slot, lst, dg, pp, scale); break;
            default: pw_rows<XT, OUT, NA, 1>(P, X, y, smem, own, slot, lst, dg, pp, scale);
        }
    }
}

// ws: the fixed-point scratch (header and X, panel_scratch_bytes).
template <typename T, typename XT, int NA>
static int run_pw(const dq_sector* s, const dq_terms* t, const T* x, T* y, void* ws, cudaStream_t st) {
    const PanelPlan& P = t->pp;
    WsHeader* h = reinterpret_cast<WsHeader*>(ws);
    XT* X = reinterpret_cast<XT*>(reinterpret_cast<char*>(ws) + 256);
    cudaMemsetAsync(h, 0, sizeof(WsHeader), st);
    const int sms = sm_count_cached();
    k_exp_max<T><<<sms * 8, 256, 0, st>>>(x, s->D, h);
    k_to_fixed<T, XT><<<sms * 8, 256, 0, st>>>(x, X, s->D, h);
    const size_t sm = PWSmem<XT>::total(t->pwr.os_total);
    auto kern = k_panel_w<XT, T, NA>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
    }
    const int per_sm = occupancy_cached(reinterpret_cast<const void*>(kern), kPWT, sm);
    const uint64_t want = ((uint64_t)P.npanels + kPWWarps - 1) / kPWWarps;
    const uint64_t cap_blocks = (uint64_t)sms * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(want < cap_blocks ? (want ? want : 1) : cap_blocks);
    const int tslot = timing_start(st);
    kern<<<grid, kPWT, sm, st>>>(P, t->pwr, X, y, h, s->dev.err);
    timing_stop(tslot, st, 3);
    return (int)cudaGetLastError();
}

int launch_panel_w_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* ws,
                      void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const bool two = t->pp.nA > 1;
    if (dtype == DQ_F64)
        return two ? run_pw<double, long long, 2>(s, t, (const double*)x, (double*)y, ws, st)
                   : run_pw<double, long long, 1>(s, t, (const double*)x, (double*)y, ws, st);
    return two ? run_pw<float, int, 2>(s, t, (const float*)x, (float*)y, ws, st)
               : run_pw<float, int, 1>(s, t, (const float*)x, (float*)y, ws, st);
}

int launch_panel_w(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream) {
    const size_t need = panel_scratch_bytes(s, dtype);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    return launch_panel_w_ws(s, t, x, y, dtype, t->scratch, stream);
}

}  // namespace dq
