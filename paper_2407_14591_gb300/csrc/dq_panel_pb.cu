// Per-bond panel product: the structural rank of the panel product (dq_panel.cu) for operators
// whose couplings and fields differ from bond to bond and from site to site (disordered chains
// and lattices), Q = 2, two subsystems, P_1 of at most 13 sites.
//
// With index = c_0(s0) + index_1(s1) (Sec. 3.3, Lin's two tables) the rows sharing a P_0 pattern
// s0 form a contiguous panel of C(L_1, n_1) rows. Per panel (one CTA of 256 threads, several
// CTAs per SM):
//   - the panel's x (fixed point, from the one-column prepass) is loaded into shared memory,
//     next to the P_1 rank table (byte offsets of the local index of every P_1 pattern);
//   - hops inside P_0 map the panel onto a partner panel element by element: coalesced loads,
//     one 128-bit multiply-add of the bond's amplitude per element;
//   - hops inside P_1 are shared-memory gathers through the rank table; a pair whose bits are
//     equal reads a slot that holds zero, so the lanes never branch;
//   - hops across the cut read the partner panel s0 ^ bit_a (the neighbouring particle-number
//     block), loaded cooperatively into a second shared-memory slot, through the same table;
//   - the diagonal is a per-panel constant (P_0 fields and P_0 Sz Sz bonds, built on the host)
//     plus, per row, the P_1 fields, the P_1 and cut Sz Sz bonds.
// Every coefficient is an integer on one grid 2^emin (at least 55 significant bits relative to
// the largest), every row result a 128-bit integer sum rounded once, as in the general kernels.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

constexpr int kPBT = 256;  // threads per CTA

int build_panel_pb(const dq_sector* s, double C, const double* lin,
                   const std::vector<std::pair<std::pair<int, int>, std::pair<double, double>>>& pairs, dq_terms* t) {
    t->pb_ok = false;
    if (s->Q != 2 || s->n_sub != 2 || s->wide) return DQ_OK;
    const int L0 = s->Lk[0], L1 = s->Lk[1], N = s->N, L = s->L;
    if (L1 < 1 || L1 > kPBMaxL1 || L0 > 16) return DQ_OK;
    PanelPB& P = t->pbp;
    std::memset(&P, 0, sizeof P);
    P.L0 = L0;
    P.L1 = L1;
    P.N = N;
    std::vector<std::pair<uint32_t, double>> p0hop, p0zz;  // (s0 pair mask, coefficient)
    std::vector<double> p1A, p1K, xA, xK;
    std::map<uint32_t, std::vector<std::pair<uint32_t, double>>> xh;  // P_0 bit a -> (P_1 bit b, A)
    double cmax = std::fabs(C);
    int nzz = 0;
    for (auto& e : pairs) {
        const int lo = e.first.first, hi = lo + e.first.second;
        const double K = e.second.first, A = e.second.second;
        if (K == 0.0 && A == 0.0) continue;
        cmax = std::max(cmax, std::max(std::fabs(K), std::fabs(A)));
        if (K != 0.0) ++nzz;
        if (hi < L1) {
            if (P.n1b == kPBMaxBonds) return DQ_OK;
            P.p1_lo[P.n1b] = 1u << lo;
            P.p1_hi[P.n1b++] = 1u << hi;
            p1A.push_back(A);
            p1K.push_back(K);
        } else if (lo >= L1) {
            const uint32_t m = (1u << (lo - L1)) | (1u << (hi - L1));
            if (A != 0.0) p0hop.push_back({m, A});
            if (K != 0.0) p0zz.push_back({m, K});
        } else {
            const uint32_t abit = 1u << (hi - L1), bbit = 1u << lo;
            if (A != 0.0) xh[abit].push_back({bbit, A});
            if (K != 0.0) {
                if (P.nxz == kPBMaxBonds) return DQ_OK;
                P.xz_abit[P.nxz] = abit;
                P.xz_bbit[P.nxz++] = bbit;
                xK.push_back(K);
            }
        }
    }
    if ((int)xh.size() > kPBMaxGroups || p0hop.size() > 200) return DQ_OK;
    for (int p = 0; p < L; ++p) cmax = std::max(cmax, std::fabs(lin[p]));
    // one grid 2^emin for all coefficients; a row's diagonal (1 + L + nzz unit terms) stays
    // below 2^62, each hop product below 2^111 in the 128-bit row sum
    long long tdiag = 1 + L + nzz;
    int lg = 0;
    while ((1ll << lg) < tdiag) ++lg;
    const int mbits = std::min(55, 62 - lg);
    P.emin = cmax > 0.0 ? std::ilogb(cmax) + 1 - mbits : 0;
    auto M = [&](double c) { return (long long)std::llrint(std::ldexp(c, -P.emin)); };
    int nxb = 0;
    for (auto& g : xh) {
        P.xg_abit[P.nxg] = g.first;
        P.xg_first[P.nxg] = nxb;
        for (auto& e : g.second) {
            if (nxb == kPBMaxBonds) return DQ_OK;
            P.xb_bit[nxb++] = e.first;
            xA.push_back(e.second);
        }
        P.xg_end[P.nxg++] = nxb;
    }
    // P_1 tables (local index within its particle-number sector, the states per sector)
    const auto& rt = s->h.rank_tab[s->dev.tab[1]];
    const auto& ut = s->h.unrank_tab[s->dev.tab[1]];
    const auto& ss = s->h.sec_start[s->dev.tab[1]];
    std::vector<uint16_t> t1rank(rt.size()), t1states(ut.size());
    for (size_t q = 0; q < rt.size(); ++q) t1rank[q] = (uint16_t)(rt[q] == 0xffffffffu ? 0 : rt[q]);
    for (size_t q = 0; q < ut.size(); ++q) t1states[q] = (uint16_t)ut[q];
    for (int n = 0; n <= L1 + 1; ++n) {
        P.t1start[n] = ss[n <= L1 ? n : L1 + 1];
        P.t1len[n] = n <= L1 ? ss[n + 1] - ss[n] : 0;
    }
    // panels in canonical order, their diagonal constants and sources
    const auto& u0 = s->h.unrank_tab[s->dev.tab[0]];
    const auto& s0s = s->h.sec_start[s->dev.tab[0]];
    std::vector<uint32_t> ps0;
    std::vector<uint64_t> pst, lst;
    std::vector<long long> pdiag;
    std::vector<uint32_t> loff, lhdr;
    const long long MC = M(C);
    for (int n0 = 0; n0 <= L0; ++n0) {
        const int n1 = N - n0;
        if (n1 < 0 || n1 > L1) continue;
        P.cmax = std::max(P.cmax, (int)P.t1len[n1]);
        for (uint32_t q = s0s[n0]; q < s0s[n0 + 1]; ++q) {
            const uint32_t s0 = u0[q];
            const uint64_t start = s->h.c0_tab[s0];
            if (start >> 48) return DQ_OK;
            ps0.push_back(s0);
            pst.push_back(start);
            long long d = MC;
            for (int k = 0; k < L0; ++k)
                if ((s0 >> k) & 1u) d += M(lin[L1 + k]);
            for (auto& e : p0zz) d += (__builtin_popcount(s0 & e.first) == 1) ? M(e.second) : 0;
            pdiag.push_back(d);
            loff.push_back((uint32_t)lst.size());
            uint32_t n0p = 0, nx = 0;
            for (size_t b = 0; b < p0hop.size(); ++b)
                if (__builtin_popcount(s0 & p0hop[b].first) == 1) {
                    lst.push_back(s->h.c0_tab[s0 ^ p0hop[b].first] | ((uint64_t)b << 48));
                    ++n0p;
                }
            for (int g = 0; g < P.nxg; ++g) {
                const uint64_t src = s->h.c0_tab[s0 ^ P.xg_abit[g]];
                if (src == UINT64_MAX) continue;  // no partner sector: no row of the panel hops here
                lst.push_back(src | ((uint64_t)g << 48));
                ++nx;
            }
            lhdr.push_back(n0p | (nx << 8));
        }
    }
    loff.push_back((uint32_t)lst.size());
    P.npanels = (uint32_t)ps0.size();
    std::vector<long long> mp1A(p1A.size()), mp1K(p1K.size()), mxA(xA.size()), mxK(xK.size()), mf1(L1), mp0A(p0hop.size());
    for (size_t q = 0; q < p1A.size(); ++q) {
        mp1A[q] = M(p1A[q]);
        mp1K[q] = M(p1K[q]);
    }
    for (size_t q = 0; q < xA.size(); ++q) mxA[q] = M(xA[q]);
    for (size_t q = 0; q < xK.size(); ++q) mxK[q] = M(xK[q]);
    for (int b = 0; b < L1; ++b) mf1[b] = M(lin[b]);
    for (size_t b = 0; b < p0hop.size(); ++b) mp0A[b] = M(p0hop[b].second);
    int rc;
    void* p;
#define DQ_UP(vec, field, type)                                                                   \
    if ((rc = dev_upload(t->dev_allocs, vec.data(), vec.size() * sizeof(vec[0]), &p))) return rc; \
    P.field = (const type*)p;
    DQ_UP(ps0, panel_s0, uint32_t)
    DQ_UP(pst, panel_start, uint64_t)
    DQ_UP(t1rank, t1rank, uint16_t)
    DQ_UP(t1states, t1states, uint16_t)
    DQ_UP(mp1A, p1_A, long long)
    DQ_UP(mp1K, p1_K, long long)
    DQ_UP(mxA, xb_A, long long)
    DQ_UP(mxK, xz_K, long long)
    DQ_UP(mf1, f1, long long)
    DQ_UP(pdiag, pdiag, long long)
    DQ_UP(mp0A, p0_A, long long)
    DQ_UP(loff, list_off, uint32_t)
    DQ_UP(lhdr, list_hdr, uint32_t)
    DQ_UP(lst, list, uint64_t)
#undef DQ_UP
    t->pb_ok = true;
    return DQ_OK;
}

// ------------------------------------------------------------------ device ------------------

template <typename XT>
__device__ __forceinline__ long long pb_lds(const unsigned char* base, uint32_t off) {
    return (long long)*reinterpret_cast<const XT*>(base + off);
}

// Shared memory: [rank table: 2^L1 + 8 u16 byte offsets, entry 2^L1 points at a zero element]
// [own panel: cap + 8 elements] [partner slot: cap + 8 elements] [source list]
template <typename XT>
struct PBSmem {
    static __host__ __device__ size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
    static __host__ __device__ size_t table(int L1) { return al(((size_t)1 << L1) * 2 + 16); }
    static __host__ __device__ size_t buf(int cap) { return al((size_t)(cap + 8) * sizeof(XT)); }
    static __host__ __device__ size_t total(int L1, int cap) { return table(L1) + 2 * buf(cap) + 8 * 256; }
};

template <typename XT, typename OUT, int E>
__device__ __forceinline__ void pb_rows(const PanelPB& P, const XT* __restrict__ X, OUT* __restrict__ y,
                                        const uint16_t* t1, const unsigned char* own, unsigned char* slot,
                                        const uint64_t* lst, uint32_t s0, uint64_t start, int n1, int C, int np0,
                                        int nx, long long d0, uint32_t zoff, int scale) {
    const int tid = threadIdx.x;
    const uint16_t* states = P.t1states + P.t1start[n1];
    uint32_t sv[E];
    long long md[E];
    I128 acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = tid + e * kPBT;
        sv[e] = c < C ? (uint32_t)__ldg(states + c) : 0u;
        md[e] = d0;
        acc[e] = {0, 0};
    }
    // hops inside P_0: partner panels element by element
    for (int l = 0; l < np0; ++l) {
        const uint64_t ent = lst[l];
        const long long A = __ldg(P.p0_A + (ent >> 48));
        const XT* src = X + (ent & ((1ull << 48) - 1));
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = tid + e * kPBT;
            if (c < C) mac(acc[e], A, (long long)__ldg(src + c));
        }
    }
    // bonds inside P_1: hop through the rank table, Sz Sz by the pair's bits
    for (int q = 0; q < P.n1b; ++q) {
        const uint32_t lo = P.p1_lo[q], hi = P.p1_hi[q], pm = lo | hi;
        const long long A = __ldg(P.p1_A + q), K = __ldg(P.p1_K + q);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const bool act = ((sv[e] & lo) != 0) != ((sv[e] & hi) != 0);
            if (A) mac(acc[e], A, pb_lds<XT>(own, act ? (uint32_t)t1[sv[e] ^ pm] : zoff));
            if (act) md[e] += K;
        }
    }
    // P_1 fields and the Sz Sz bonds across the cut
    for (int b = 0; b < P.L1; ++b) {
        const long long f = __ldg(P.f1 + b);
        if (f == 0) continue;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if ((sv[e] >> b) & 1u) md[e] += f;
    }
    for (int z = 0; z < P.nxz; ++z) {
        const bool sa = (s0 & P.xz_abit[z]) != 0;
        const uint32_t bb = P.xz_bbit[z];
        const long long K = __ldg(P.xz_K + z);
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (((sv[e] & bb) != 0) != sa) md[e] += K;
    }
    // hops across the cut: the partner panel in the second slot
    for (int j = 0; j < nx; ++j) {
        const uint64_t ent = lst[np0 + j];
        const int g = (int)(ent >> 48);
        const bool sa = (s0 & P.xg_abit[g]) != 0;
        const int nn = sa ? n1 + 1 : n1 - 1;  // the partner's P_1 particle number
        const int len = (nn < 0 || nn > P.L1) ? 0 : (int)P.t1len[nn];
        const XT* src = X + (ent & ((1ull << 48) - 1));
        __syncthreads();  // the slot's previous partner is no longer read
        for (int c = tid; c < len; c += kPBT) reinterpret_cast<XT*>(slot)[c] = __ldg(src + c);
        __syncthreads();
        for (int q = P.xg_first[g]; q < P.xg_end[g]; ++q) {
            const uint32_t bb = P.xb_bit[q];
            const long long A = __ldg(P.xb_A + q);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool act = ((sv[e] & bb) != 0) != sa;
                mac(acc[e], A, pb_lds<XT>(slot, act ? (uint32_t)t1[sv[e] ^ bb] : zoff));
            }
        }
    }
    // the row result: d x_i + sum of the hops, exactly, rounded once
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = tid + e * kPBT;
        if (c >= C) continue;
        I128 r = acc[e];
        mac(r, md[e], pb_lds<XT>(own, (uint32_t)(c * sizeof(XT))));
        y[start + c] = i128_to<OUT>(r, scale);
    }
}

// Four CTAs per SM (at most 64 registers per thread): the kernel waits on its partner loads, so
// the extra warps pay for the few spilled registers (0.200 -> 0.178 ms on workload 5).
template <typename XT, typename OUT>
__global__ void __launch_bounds__(kPBT, 4) k_panel_pb(PanelPB P, const XT* __restrict__ X, OUT* __restrict__ y,
                                                   const WsHeader* __restrict__ h, int* err, int cap) {
    extern __shared__ __align__(128) unsigned char smem[];
    using SL = PBSmem<XT>;
    const int tid = threadIdx.x;
    uint16_t* t1 = reinterpret_cast<uint16_t*>(smem);
    unsigned char* own = smem + SL::table(P.L1);
    unsigned char* slot = own + SL::buf(cap);
    uint64_t* lst = reinterpret_cast<uint64_t*>(slot + SL::buf(cap));
    __shared__ uint32_t s_hdr;
    const uint32_t ntab = 1u << P.L1;
    const uint32_t zoff = (uint32_t)((cap + 1) * sizeof(XT));  // an element that stays zero
    for (uint32_t q = tid; q < ntab; q += kPBT) t1[q] = (uint16_t)(__ldg(P.t1rank + q) * sizeof(XT));
    for (int q = tid; q < 8; q += kPBT) {
        reinterpret_cast<XT*>(own)[cap + q] = 0;
        reinterpret_cast<XT*>(slot)[cap + q] = 0;
    }
    __syncthreads();
    if (h->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint32_t pi = blockIdx.x; pi < P.npanels; pi += gridDim.x) {
            const uint64_t st = P.panel_start[pi];
            const int C = (int)P.t1len[P.N - __popc(P.panel_s0[pi])];
            for (int c = tid; c < C; c += kPBT) y[st + c] = (OUT)NAN;
        }
        if (blockIdx.x == 0 && tid == 0) atomicAdd(err, 1);
        return;
    }
    const int scale = P.emin - h->F;
    for (uint32_t pi = blockIdx.x; pi < P.npanels; pi += gridDim.x) {
        const uint32_t s0 = __ldg(P.panel_s0 + pi);
        const uint64_t start = __ldg(P.panel_start + pi);
        const int n1 = P.N - __popc(s0);
        const int C = (int)P.t1len[n1];
        const uint32_t lo = __ldg(P.list_off + pi), hi = __ldg(P.list_off + pi + 1);
        for (uint32_t q = lo + tid; q < hi; q += kPBT) lst[q - lo] = __ldg(P.list + q);
        if (tid == 0) s_hdr = __ldg(P.list_hdr + pi);
        const XT* src = X + start;
        for (int c = tid; c < C; c += kPBT) reinterpret_cast<XT*>(own)[c] = __ldg(src + c);
        __syncthreads();
        const int np0 = (int)(s_hdr & 255u), nx = (int)((s_hdr >> 8) & 255u);
        const long long d0 = __ldg(P.pdiag + pi);
        switch ((C + kPBT - 1) / kPBT) {
            case 7: pb_rows<XT, OUT, 7>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            case 6: pb_rows<XT, OUT, 6>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            case 5: pb_rows<XT, OUT, 5>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            case 4: pb_rows<XT, OUT, 4>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            case 3: pb_rows<XT, OUT, 3>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            case 2: pb_rows<XT, OUT, 2>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale); break;
            default: pb_rows<XT, OUT, 1>(P, X, y, t1, own, slot, lst, s0, start, n1, C, np0, nx, d0, zoff, scale);
        }
        __syncthreads();
    }
}

template <typename T, typename XT>
static int run_pb(const dq_sector* s, dq_terms* t, const T* x, T* y, cudaStream_t st) {
    const PanelPB& P = t->pbp;
    const size_t need = panel_scratch_bytes(s, sizeof(T) == 8 ? DQ_F64 : DQ_F32);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    WsHeader* h = reinterpret_cast<WsHeader*>(t->scratch);
    XT* X = reinterpret_cast<XT*>(reinterpret_cast<char*>(t->scratch) + 256);
    cudaMemsetAsync(h, 0, sizeof(WsHeader), st);
    const int sms = sm_count_cached();
    k_exp_max<T><<<sms * 8, 256, 0, st>>>(x, s->D, h);
    k_to_fixed<T, XT><<<sms * 8, 256, 0, st>>>(x, X, s->D, h);
    const int cap = P.cmax + 16 / (int)sizeof(XT);
    const size_t sm = PBSmem<XT>::total(P.L1, cap);
    auto kern = k_panel_pb<XT, T>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
    }
    const int per_sm = occupancy_cached(reinterpret_cast<const void*>(kern), kPBT, sm);
    const uint64_t cap_blocks = (uint64_t)sms * per_sm;
    const unsigned grid = (unsigned)(P.npanels < cap_blocks ? (P.npanels ? P.npanels : 1) : cap_blocks);
    const int tslot = timing_start(st);
    kern<<<grid, kPBT, sm, st>>>(P, X, y, h, s->dev.err, cap);
    timing_stop(tslot, st, 3);
    return (int)cudaGetLastError();
}

int launch_panel_pb(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64) return run_pb<double, long long>(s, t, (const double*)x, (double*)y, st);
    return run_pb<float, int>(s, t, (const float*)x, (float*)y, st);
}

}  // namespace dq
