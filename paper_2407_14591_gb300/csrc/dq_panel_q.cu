// Boson panel product y = H x for Q > 2 and two subsystems: the plan (host) and the kernel.
//
// With two subsystems the canonical index is c_0(s0) + index_1(s1) (Sec. 3.3, Lin's two tables),
// so the rows sharing one P_0 pattern s0 form a contiguous panel of D_Q(L_1, N - n_0) rows in
// P_1's local order, for any Q. The operator is the per-term form of the general kernel (site
// functions f_i(n_i), hops -t_q (b+_a b_b + h.c.) with amplitude -t_q sqrt((n_up + 1) n_dn)),
// its coefficients already integers on one grid 2^emin. A hop b+_up b_dn acts on a panel in one
// of three ways:
//   both sites in P_1:  s1 -> s1 + e_up - e_dn inside the panel, the same for every panel of a
//                       particle-number block: a per-pattern list of partner rows and amplitude
//                       entries (host), gathers from the panel's own x (L1);
//   both sites in P_0:  panel s0 receives panel s0 + e_up - e_dn element by element, with one
//                       amplitude for the whole panel: a coalesced stream of the partner panel;
//   across the cut:     panel s0 receives panel s0 +- e_a (one particle more or less in P_0) at
//                       the local index of s1 -+ e_b: the panel fixes the partner panel and the
//                       P_0 digit, a per-pattern table the partner row and the P_1 digit.
// The diagonal is a per-panel constant (the constant and the P_0 site functions) plus a
// per-pattern value (the P_1 site functions), both from the host. The kernel thus does no digit
// arithmetic at all: per hop it reads a table entry, an amplitude and an x element, and adds
// four 32 x 32 -> 64-bit products (below). Every row is one exact integer sum rounded once; the
// coefficients are those of the general kernel, so on FP64 vectors the two give the same y.
//
// One warp per panel: the warps of persistent 512-thread CTAs take panels from an atomic counter,
// longest panels first, and never wait for each other; a warp's lanes take the panel's rows.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

constexpr uint64_t kPQStart = (1ull << 40) - 1;

// ------------------------------------------------------------------ plan (host) -------------

int build_panel_q(const dq_sector* s, const std::vector<int>& site_sh, const std::vector<long long>& msite,
                  const std::vector<int>& hop_sh, const std::vector<long long>& mhop, long long MC, int emin,
                  int npair, dq_terms* t) {
    t->pq_ok = false;
    const int Q = s->Q, nb = s->nb;
    if (Q <= 2 || s->wide || s->n_sub != 2 || npair != 0 || !s->has_device) return DQ_OK;
    const int L1 = s->Lk[1], L0 = s->Lk[0], N = s->N;
    const int B = nb * L1, B0 = nb * L0;
    const int nhop = (int)hop_sh.size() / 2, nsite = (int)site_sh.size();
    if (B < 1 || B > kPQMaxBits || B0 > 24 || (Q - 1) * L1 + 1 > kPQMaxN) return DQ_OK;
    // at most 63 hops per row (the kernel's int64 partial sums), 4096 amplitude entries
    if (2 * nhop > 63 || (size_t)nhop * Q * Q > 4096 || s->D >= (1ull << 40)) return DQ_OK;
    PanelQ& P = t->pqp;
    std::memset(&P, 0, sizeof P);
    P.Q = Q;
    P.nb = nb;
    P.L1 = L1;
    P.N = N;
    P.emin = emin;
    P.nM = nhop * Q * Q;
    const uint32_t dm = (1u << nb) - 1;
    // P_1 patterns: the subsystem's own rank and unrank tables (local order inside each block)
    const int tl = s->dev.tab[1];
    const auto& rt = s->h.rank_tab[tl];
    const auto& ut = s->h.unrank_tab[tl];
    const auto& ss = s->h.sec_start[tl];
    const int n1max = (Q - 1) * L1;
    for (int n = 0; n <= n1max + 1; ++n) {
        P.t1start[n] = ss[n];
        P.t1len[n] = n <= n1max ? ss[n + 1] - ss[n] : 0;
        if (P.t1len[n] > 65535) return DQ_OK;
    }
    // hop directions, by where their sites lie
    struct Dir {
        int q, up, dn;  // bond, shifts of the receiving and the giving site in the whole word
    };
    std::vector<Dir> d1, d0, dx;
    for (int q = 0; q < nhop; ++q)
        for (int dir = 0; dir < 2; ++dir) {
            const int up = hop_sh[2 * q + dir], dn = hop_sh[2 * q + 1 - dir];
            if (up < B && dn < B)
                d1.push_back({q, up, dn});
            else if (up >= B && dn >= B)
                d0.push_back({q, up - B, dn - B});
            else
                dx.push_back({q, up, dn});
        }
    if ((int)dx.size() > kPQMaxCut) return DQ_OK;
    P.ncut = (int)dx.size();
    auto digit = [&](uint32_t w, int sh) { return (int)((w >> sh) & dm); };
    // per-pattern tables
    const size_t npat = ut.size();
    std::vector<long long> rdiag(npat, 0);
    std::vector<uint32_t> p1ell, cutt;
    for (int n = 0; n <= n1max; ++n) {
        const uint32_t C1 = P.t1len[n], b0 = P.t1start[n];
        std::vector<std::vector<uint32_t>> lists(C1);
        size_t mx = 0;
        for (uint32_t c = 0; c < C1; ++c) {
            const uint32_t s1 = ut[b0 + c];
            long long dg = 0;
            for (int q = 0; q < nsite; ++q)
                if (site_sh[q] < B) dg += msite[(size_t)q * Q + digit(s1, site_sh[q])];
            rdiag[b0 + c] = dg;
            for (const Dir& d : d1) {
                const int nu = digit(s1, d.up), nd = digit(s1, d.dn);
                if (nu >= Q - 1 || nd == 0) continue;
                const uint32_t j = rt[s1 + (1u << d.up) - (1u << d.dn)];
                lists[c].push_back(j | ((uint32_t)((d.q * Q + nu) * Q + nd) << 16));
            }
            mx = std::max(mx, lists[c].size());
        }
        P.p1base[n] = (uint32_t)p1ell.size();
        P.p1m[n] = (uint32_t)mx;
        for (size_t m = 0; m < mx; ++m)  // padding: the row itself with the zero amplitude nM
            for (uint32_t c = 0; c < C1; ++c)
                p1ell.push_back(m < lists[c].size() ? lists[c][m] : (c | ((uint32_t)P.nM << 16)));
        P.cutbase[n] = (uint32_t)cutt.size();
        for (const Dir& d : dx)
            for (uint32_t c = 0; c < C1; ++c) {
                const uint32_t s1 = ut[b0 + c];
                uint32_t v = 1u << 31;
                if (d.up >= B) {  // b+_a b_b: a particle leaves P_1 site b for P_0 site a
                    const int db = digit(s1, d.dn);
                    if (db > 0) v = rt[s1 - (1u << d.dn)] | ((uint32_t)db << 16);
                } else {  // b+_b b_a: a particle enters P_1 site b from P_0 site a
                    const int db = digit(s1, d.up);
                    if (db < Q - 1) v = rt[s1 + (1u << d.up)] | ((uint32_t)(db * Q) << 16);
                }
                cutt.push_back(v);
            }
    }
    P.p1base[n1max + 1] = (uint32_t)p1ell.size();
    P.cutbase[n1max + 1] = (uint32_t)cutt.size();
    // panels: every P_0 pattern that P_1 can complete, longest first
    const auto& c0 = s->h.c0_tab;
    std::vector<std::pair<std::pair<uint32_t, uint64_t>, uint32_t>> pl;  // ((~length, start), s0)
    for (uint64_t p = 0; p < c0.size(); ++p) {
        if (c0[p] == UINT64_MAX) continue;
        int n0 = 0;
        for (int k = 0; k < L0; ++k) n0 += (int)((p >> (nb * k)) & dm);
        const int n1 = N - n0;
        if (n1 < 0 || n1 > n1max) continue;
        const uint32_t C1 = P.t1len[n1];
        if (C1 == 0) continue;
        pl.push_back({{~C1, c0[p]}, (uint32_t)p});
    }
    std::sort(pl.begin(), pl.end());
    P.npanels = (uint32_t)pl.size();
    std::vector<uint32_t> ps0(pl.size());
    std::vector<uint64_t> pst(pl.size());
    std::vector<long long> pdiag(pl.size());
    std::vector<uint32_t> loff(pl.size() + 1, 0), lhdr(pl.size(), 0);
    std::vector<uint64_t> lst;
    lst.reserve(pl.size() * (d0.size() + dx.size()));
    auto digit0 = [&](uint32_t s0, int sh) { return (int)((s0 >> sh) & dm); };
    for (size_t i = 0; i < pl.size(); ++i) {
        const uint32_t s0 = pl[i].second;
        ps0[i] = s0;
        pst[i] = pl[i].first.second;
        long long dg = MC;
        for (int q = 0; q < nsite; ++q)
            if (site_sh[q] >= B) dg += msite[(size_t)q * Q + digit0(s0, site_sh[q] - B)];
        pdiag[i] = dg;
        loff[i] = (uint32_t)lst.size();
        uint32_t n0e = 0, nxe = 0;
        for (const Dir& d : d0) {
            const int nu = digit0(s0, d.up), nd = digit0(s0, d.dn);
            if (nu >= Q - 1 || nd == 0) continue;
            const uint32_t s0n = s0 + (1u << d.up) - (1u << d.dn);
            const uint64_t st = c0[s0n];
            if (st == UINT64_MAX) return DQ_OK;  // the same particle number: always completable
            lst.push_back(st | ((uint64_t)((d.q * Q + nu) * Q + nd) << 40));
            ++n0e;
        }
        for (int di = 0; di < (int)dx.size(); ++di) {
            const Dir& d = dx[di];
            uint64_t st, base;
            if (d.up >= B) {  // b+_a b_b: a particle from P_1 site b into P_0 site a
                const int pd = digit0(s0, d.up - B);
                if (pd >= Q - 1) continue;
                st = c0[s0 + (1u << (d.up - B))];
                base = (uint64_t)((d.q * Q + pd) * Q);        // + n_b
            } else {  // b+_b b_a: a particle from P_0 site a into P_1 site b
                const int pd = digit0(s0, d.dn - B);
                if (pd == 0) continue;
                st = c0[s0 - (1u << (d.dn - B))];
                base = (uint64_t)(d.q * Q * Q + pd);          // + n_b Q
            }
            if (st == UINT64_MAX) continue;  // P_1 cannot hold one more (or one fewer) particle
            lst.push_back(st | ((uint64_t)di << 40) | (base << 48));
            ++nxe;
        }
        if (n0e + nxe > (uint32_t)kPQMaxList) return DQ_OK;
        lhdr[i] = n0e | (nxe << 8);
    }
    loff[pl.size()] = (uint32_t)lst.size();
    int rc;
    void* p;
    auto up = [&](const void* src, size_t bytes, const void** dst) -> int {
        if (bytes == 0) {
            *dst = nullptr;
            return DQ_OK;
        }
        int r = dev_upload(t->dev_allocs, src, bytes, &p);
        *dst = p;
        return r;
    };
    std::vector<long long> mh(mhop);
    mh.push_back(0);  // entry nM: the zero amplitude of the padding
    if ((rc = up(ps0.data(), ps0.size() * 4, (const void**)&P.panel_s0))) return rc;
    if ((rc = up(pst.data(), pst.size() * 8, (const void**)&P.panel_start))) return rc;
    if ((rc = up(mh.data(), mh.size() * 8, (const void**)&P.Mhop))) return rc;
    if ((rc = up(rdiag.data(), rdiag.size() * 8, (const void**)&P.rdiag))) return rc;
    if ((rc = up(p1ell.data(), p1ell.size() * 4, (const void**)&P.p1ell))) return rc;
    if ((rc = up(cutt.data(), cutt.size() * 4, (const void**)&P.cutt))) return rc;
    if ((rc = up(pdiag.data(), pdiag.size() * 8, (const void**)&P.pdiag))) return rc;
    if ((rc = up(loff.data(), loff.size() * 4, (const void**)&P.list_off))) return rc;
    if ((rc = up(lhdr.data(), lhdr.size() * 4, (const void**)&P.list_hdr))) return rc;
    if ((rc = up(lst.data(), lst.size() * 8, (const void**)&P.list))) return rc;
    t->pq_ok = P.npanels > 0;
    return DQ_OK;
}

// ------------------------------------------------------------------ kernel -------------------

// x in split fixed point: X = round(x 2^F) with |X| < 2^56 (as in the other panel kernels), stored
// as one 64-bit word whose high half is X_h = X >> 28 (signed) and whose low half is
// X_l = X mod 2^28, so that X = X_h 2^28 + X_l. A coefficient M (|M| < 2^55) splits the same way
// (M_h, M_l), and a hop adds the four 32 x 32 -> 64-bit products to three int64 sums
//   hh += M_h X_h,  mid += M_h X_l + M_l X_h,  ll += M_l X_l
// (each product below 2^56, so at most 63 hops per row keep every sum below 2^63); the row is
// hh 2^56 + mid 2^28 + ll, exactly M X summed, plus the diagonal's 128-bit product.
template <typename T>
__global__ void k_split_fixed(const T* __restrict__ x, long long* __restrict__ X, uint64_t n, WsHeader* h) {
    using U = typename FBits<T>::U;
    constexpr int BIAS = FBits<T>::BIAS;
    const int emax = h->emax;
    if (emax == FBits<T>::EMASK) {  // Inf or NaN in x
        if (blockIdx.x == 0 && threadIdx.x == 0) h->bad = 1;
        return;
    }
    const int F = XHead<long long>::HEAD - (emax - BIAS + 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) h->F = F;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = t0; i < n; i += step) {
        const long long v = to_fixed<T, long long>(reinterpret_cast<const U*>(x)[i], F);
        X[i] = (long long)(((unsigned long long)(uint32_t)(int)(v >> 28) << 32) | (unsigned long long)(v & 0xfffffffll));
    }
}

struct Acc3 {
    long long hh, mid, ll;
};

// d = a b + c with the signed 32 x 32 -> 64-bit product (one mad.wide.s32; the same sum written
// with 64-bit operands in C++ took about a fifth longer on workload 3)
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void acc_hop(Acc3& a, int2 m, long long xs) {
    const int xh = (int)(xs >> 32), xl = (int)(xs & 0xffffffffll);
    a.hh = mad_wide(m.x, xh, a.hh);
    a.mid = mad_wide(m.y, xh, mad_wide(m.x, xl, a.mid));
    a.ll = mad_wide(m.y, xl, a.ll);
}

// a += v 2^sh for 0 <= sh < 64
__device__ __forceinline__ void add_shifted(I128& a, long long v, int sh) {
    const unsigned long long lo = sh ? (unsigned long long)v << sh : (unsigned long long)v;
    const long long hi = sh ? (v >> (64 - sh)) : (v >> 63);
    const unsigned long long s = a.lo + lo;
    a.hi += hi + (s < a.lo ? 1 : 0);
    a.lo = s;
}

constexpr int kPQT = 512;           // threads per CTA
constexpr int kPQW = kPQT / 32;     // warps per CTA, one panel each at a time

// Shared memory: the split amplitudes (int2 per Mhop entry, the zero entry nM last) and one
// source-list slot per warp.
struct PQSmem {
    size_t ms, lst, total;
    __host__ __device__ PQSmem(const PanelQ& P) {
        ms = 0;
        lst = ((size_t)(P.nM + 1) * 8 + 15) & ~(size_t)15;
        total = lst + (size_t)8 * kPQMaxList * kPQW;
    }
};

template <typename OUT>
__global__ void __launch_bounds__(kPQT, 2)
    k_panel_q(PanelQ P, const long long* __restrict__ X, OUT* __restrict__ y, const WsHeader* __restrict__ h,
              unsigned long long* queue, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const PQSmem L(P);
    int2* Ms = reinterpret_cast<int2*>(smem + L.ms);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* wl = reinterpret_cast<uint64_t*>(smem + L.lst) + warp * kPQMaxList;
    const uint32_t dm = (1u << P.nb) - 1;
    if (h->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint32_t pi = blockIdx.x; pi < P.npanels; pi += gridDim.x) {
            const uint64_t st = P.panel_start[pi];
            int n0 = 0;
            for (int k = 0; k < 32; k += P.nb) n0 += (int)((P.panel_s0[pi] >> k) & dm);
            const int C = (int)P.t1len[P.N - n0];
            for (int c = tid; c < C; c += kPQT) y[st + c] = (OUT)NAN;
        }
        if (blockIdx.x == 0 && tid == 0) atomicAdd(err, 1);
        return;
    }
    for (int q = tid; q <= P.nM; q += kPQT) {
        const long long m = __ldg(P.Mhop + q);
        Ms[q] = make_int2((int)(m >> 28), (int)(m & 0xfffffffll));
    }
    __syncthreads();
    const int scale = P.emin - h->F;
    for (;;) {
        uint32_t pi = 0;
        if (lane == 0) pi = (uint32_t)atomicAdd(queue, 1ull);
        pi = __shfl_sync(0xffffffffu, pi, 0);
        if (pi >= P.npanels) break;
        const uint32_t s0 = __ldg(P.panel_s0 + pi);
        const uint64_t start = __ldg(P.panel_start + pi);
        int n0 = 0;
        for (int k = 0; k < 32; k += P.nb) n0 += (int)((s0 >> k) & dm);
        const int n1 = P.N - n0;
        const int C = (int)P.t1len[n1];
        const uint32_t hd = __ldg(P.list_hdr + pi), lo = __ldg(P.list_off + pi);
        const int np0 = (int)(hd & 255u), nx = (int)((hd >> 8) & 255u);
        __syncwarp();  // the warp's rows of the previous panel are done with its list slot
        for (int q = lane; q < np0 + nx; q += 32) wl[q] = __ldg(P.list + lo + q);
        __syncwarp();
        const long long pd = __ldg(P.pdiag + pi);
        const long long* rdg = P.rdiag + P.t1start[n1];
        const uint32_t* e1 = P.p1ell + P.p1base[n1];
        const int m1 = (int)P.p1m[n1];
        const uint32_t* ct = P.cutt + P.cutbase[n1];
        const long long* Xo = X + start;
        for (int c = lane; c < C; c += 32) {
            const long long xo = __ldg(Xo + c);
            const long long dg = pd + __ldg(rdg + c);
            Acc3 a = {0, 0, 0};
            // hops inside P_1: partner rows of the same panel (padding: the row itself, amplitude 0)
#pragma unroll 4
            for (int m = 0; m < m1; ++m) {
                const uint32_t v = __ldg(e1 + (size_t)m * C + c);
                acc_hop(a, Ms[v >> 16], __ldg(Xo + (v & 0xffffu)));
            }
            // hops inside P_0: partner panels element by element
#pragma unroll 4
            for (int e = 0; e < np0; ++e) {
                const uint64_t ent = wl[e];
                acc_hop(a, Ms[ent >> 40], __ldg(X + (ent & kPQStart) + c));
            }
            // hops across the cut: the partner panel at the row's tabulated local index
#pragma unroll 2
            for (int e = np0; e < np0 + nx; ++e) {
                const uint64_t ent = wl[e];
                const uint32_t v = __ldg(ct + (size_t)((ent >> 40) & 255u) * C + c);
                const int mi = (v >> 31) ? P.nM : (int)(ent >> 48) + (int)((v >> 16) & 0x7fffu);
                acc_hop(a, Ms[mi], __ldg(X + (ent & kPQStart) + (v & 0xffffu)));
            }
            I128 r = {0, 0};
            const long long xi = (long long)(int)(xo >> 32) * (1ll << 28) + (long long)(xo & 0xffffffffll);
            mac(r, dg, xi);
            add_shifted(r, a.hh, 56);
            add_shifted(r, a.mid, 28);
            add_shifted(r, a.ll, 0);
            y[start + c] = i128_to<OUT>(r, scale);
        }
    }
}

// ------------------------------------------------------------------ launch -------------------

template <typename T>
static int run_panel_q(const dq_sector* s, const dq_terms* t, const T* x, T* y, void* ws, cudaStream_t st) {
    const PanelQ& P = t->pqp;
    WsHeader* h = reinterpret_cast<WsHeader*>(ws);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws) + 128);
    long long* X = reinterpret_cast<long long*>(reinterpret_cast<char*>(ws) + 256);
    cudaMemsetAsync(ws, 0, 256, st);  // the header and the panel counter
    const int sms = sm_count_cached();
    k_exp_max<T><<<sms * 8, 256, 0, st>>>(x, s->D, h);
    k_split_fixed<T><<<sms * 8, 256, 0, st>>>(x, X, s->D, h);
    const size_t sm = PQSmem(P).total;
    auto kern = k_panel_q<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPQT, sm)) != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    const uint32_t wslots = (uint32_t)sms * (uint32_t)per_sm * kPQW;
    const unsigned grid = (unsigned)((P.npanels < wslots ? (P.npanels + kPQW - 1) / kPQW : wslots / kPQW));
    const int tslot = timing_start(st);
    kern<<<grid, kPQT, sm, st>>>(P, X, y, h, queue, s->dev.err);
    timing_stop(tslot, st, 3);
    return (int)cudaGetLastError();
}

int launch_panel_q_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* ws,
                      void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64) return run_panel_q<double>(s, t, (const double*)x, (double*)y, ws, st);
    return run_panel_q<float>(s, t, (const float*)x, (float*)y, ws, st);
}

int launch_panel_q(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream) {
    const size_t need = panel_scratch_bytes(s, DQ_F64);  // split 64-bit x for both dtypes
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    return launch_panel_q_ws(s, t, x, y, dtype, t->scratch, stream);
}

}  // namespace dq
