// Host side of the panel product: decides whether it applies and builds its plan.
//
// With two subsystems the canonical index is c_0(s0) + index_1(s1) (Sec. 3.3, Lin's two tables),
// so all states with one P_0 pattern s0 occupy a contiguous range of D_2(L_1, N - n_0) indices,
// ordered by the local index of s1. A bond between sites i < j acts on such "panels" in one of
// three ways:
//   both sites in P_1:  a permutation inside the panel, the same for every panel of a block;
//   both sites in P_0:  panel s0 receives panel s0' (two bits swapped) element by element;
//   across the cut:     panel s0 receives panel s0 ^ bit_a (the neighbouring particle-number
//                       block) through the map s1 -> index_1(s1 ^ bit_b).
// Requirements: Q = 2, two subsystems, L_1 <= 15 (panels of at most 6435 rows), uniform
// single-site fields, at most two distinct hop amplitudes and four distinct coefficients of
// [s_i != s_j], and coefficients that are small integer multiples of one power of two.
//
// With three or more subsystems the same holds with P_0 = all subsystems but the last and P_1 =
// the last one (Eq. (index): the last subsystem has offset 0 and stride 1 inside the block of its
// particle number, so the rows sharing the prefix pattern s0 are again contiguous, in P_1's local
// order). Those panels are small (P_1 of 8 to 10 sites: at most 252 rows) and many, so the
// warp-panel kernel (dq_panel_w.cu) gives each panel one warp and ranks the partner panels on the
// device; the host builds only the panel list and the bond tables. Two subsystems whose P_1 has 8
// to 10 sites take that kernel too.
//
// Three or more subsystems whose last one is shorter than 8 (or longer than 10) sites use P_1 =
// the last TWO subsystems (the "tail") in the panel kernel instead: with the prefix pattern s0
// fixed, the canonical key (n_0, σ0, ..., n_{n-2}, σ_{n-2}, n_{n-1}, σ_{n-1}) leaves only the
// tail's two entries free, so those rows are again one contiguous range, ordered by the tail's
// own two-subsystem canonical order (Eq. (index) restricted to the tail). That order depends on
// the tail's particle number only; the host tabulates it (tail pattern -> local index) from the
// sector's own rank and checks every panel's first and last row.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "dq_internal.h"

namespace dq {

// Exponent of the lowest set bit of v's mantissa: v = m * 2^e with m odd.
static int low_exponent(double v) {
    int ex;
    double f = std::frexp(std::fabs(v), &ex);  // |v| = f 2^ex, f in [0.5, 1)
    long long m = (long long)std::ldexp(f, 53);
    int e = ex - 53;
    while ((m & 1) == 0) {
        m >>= 1;
        ++e;
    }
    return e;
}

// The rest of the plan for three or more subsystems: the panel list (every prefix pattern s0
// whose P_1 particle number N - |s0| fits, with its first index), the prefix masks
// of the cut Sz Sz bonds per class and position b, the sector view for the device rank.
static int build_panel_w(const dq_sector* s, PanelPlan& P, const std::vector<uint16_t>& t1rank,
                         const std::vector<uint16_t>& t1states,
                         const std::vector<std::pair<int, std::pair<uint32_t, uint32_t>>>& xz, dq_terms* t) {
    const int L1 = P.L1, L0 = P.L0, N = P.N, last = s->n_sub - 1;
    const int tl = s->dev.tab[last];
    // panels grouped by length (the warps in flight then run one row-count variant of the
    // kernel, which keeps its code in the instruction cache), in canonical order inside a group
    std::vector<std::pair<std::pair<uint32_t, uint64_t>, uint32_t>> pl;  // ((length, start), s0)
    int cmax = 0;
    uint64_t smax = 0;
    for (uint64_t s0 = 0; s0 < (1ull << L0); ++s0) {
        const int n1 = N - __builtin_popcountll(s0);
        if (n1 < 0 || n1 > L1) continue;
        const uint32_t first = s->h.unrank_tab[tl][s->h.sec_start[tl][n1]];  // local index 0
        const u128 w = ((u128)s0 << L1) | first;
        const uint64_t st = host_rank(s, w);
        pl.push_back({{P.t1len[n1], st}, (uint32_t)s0});
        cmax = std::max(cmax, (int)P.t1len[n1]);
        smax = std::max(smax, st);
    }
    std::sort(pl.begin(), pl.end());
    if (pl.empty() || smax >> 48) return DQ_OK;
    std::vector<uint32_t> ps0(pl.size());
    std::vector<uint64_t> pst(pl.size());
    for (size_t q = 0; q < pl.size(); ++q) {
        pst[q] = pl[q].first.second;
        ps0[q] = pl[q].second;
    }
    P.npanels = (uint32_t)pl.size();
    P.cmax = cmax;
    std::memset(P.xzA, 0, sizeof P.xzA);
    for (auto& e : xz) P.xzA[e.first][__builtin_ctz(e.second.second)] |= e.second.first;
    PWRank& R = t->pwr;
    std::memset(&R, 0, sizeof R);
    R.n_sub = s->n_sub;
    R.N = N;
    R.L1 = L1;
    R.os_total = s->dev.os_total;
    R.D = s->D;
    for (int k = 0; k < s->n_sub; ++k) {
        R.shift[k] = s->dev.shift[k];
        R.os_base[k] = s->dev.os_base[k];
        R.os_ld[k] = s->dev.os_ld[k];
        R.fmask[k] = (uint32_t)((1ull << s->Lk[k]) - 1);
        R.rank[k] = s->dev.rank_tab[s->dev.tab[k]];
    }
    R.off = s->dev.off;
    R.str = s->dev.str;
    int rc;
    void* p;
    if ((rc = dev_upload(t->dev_allocs, ps0.data(), ps0.size() * 4, &p))) return rc;
    P.panel_s0 = (const uint32_t*)p;
    if ((rc = dev_upload(t->dev_allocs, pst.data(), pst.size() * 8, &p))) return rc;
    P.panel_start = (const uint64_t*)p;
    if ((rc = dev_upload(t->dev_allocs, t1rank.data(), t1rank.size() * 2, &p))) return rc;
    P.t1rank = (const uint16_t*)p;
    if ((rc = dev_upload(t->dev_allocs, t1states.data(), t1states.size() * 2, &p))) return rc;
    P.t1states = (const uint16_t*)p;
    t->pw_ok = true;
    return DQ_OK;
}

int build_panel_plan(const dq_sector* s, double C, bool uniform_lin,
                     const std::vector<std::pair<std::pair<int, int>, std::pair<double, double>>>& pairs, dq_terms* t) {
    t->panel_ok = false;
    t->pw_ok = false;
    if (s->Q != 2 || s->n_sub < 2 || !uniform_lin || s->wide) return DQ_OK;
    // the warp-panel kernel for three or more subsystems, and for two when the panels are small
    // (P_1 of 8 to 10 sites: at most 252 rows, which leave most of a 1024-thread CTA idle)
    const int ns = s->n_sub;
    const bool warp = s->Lk[ns - 1] >= 8 && s->Lk[ns - 1] <= 10;
    const bool tail = ns >= 3 && !warp;  // P_1 = the last two subsystems
    const int L1 = tail ? s->Lk[ns - 2] + s->Lk[ns - 1] : s->Lk[ns - 1], L0 = s->L - L1, N = s->N;
    if (warp) {
        if (ns > kPWMaxSub || L0 > 24) return DQ_OK;
    } else if (L1 > 15 || L1 < 1 || L0 > (tail ? 22 : 16)) {
        return DQ_OK;
    }
    PanelPlan& P = t->pp;
    std::memset(&P, 0, sizeof P);
    P.L0 = L0;
    P.L1 = L1;
    P.N = N;
    std::vector<double> Avals, Kvals;
    auto cls_of = [](std::vector<double>& vals, double v, int maxn) -> int {
        for (size_t q = 0; q < vals.size(); ++q)
            if (vals[q] == v) return (int)q;
        if ((int)vals.size() >= maxn) return -1;
        vals.push_back(v);
        return (int)vals.size() - 1;
    };
    // collect bonds by category, keyed so that iteration order is by class
    std::map<std::pair<int, int>, uint32_t> p1z;                      // (class, d) -> low-position mask
    std::map<int, std::vector<std::pair<int, int>>> p1o;               // d -> (class, lo)
    std::vector<std::pair<int, uint32_t>> p0o, p0z;                   // (class, s0 mask)
    std::map<uint32_t, std::vector<std::pair<int, uint32_t>>> xo;     // a bit -> (class, b bit)
    std::vector<std::pair<int, std::pair<uint32_t, uint32_t>>> xz;    // (class, (a bit, b bit))
    for (auto& e : pairs) {
        int lo = e.first.first, d = e.first.second, hi = lo + d;
        double K = e.second.first, A = e.second.second;
        int ka = -1, kk = -1;
        if (A != 0.0 && (ka = cls_of(Avals, A, kPanelMaxA)) < 0) return DQ_OK;
        if (K != 0.0 && (kk = cls_of(Kvals, K, kPanelMaxK)) < 0) return DQ_OK;
        if (hi < L1) {  // both in P_1
            if (A != 0.0) p1o[d].push_back({ka, lo});
            if (K != 0.0) p1z[{kk, d}] |= 1u << lo;
        } else if (lo >= L1) {  // both in P_0
            uint32_t m = (1u << (lo - L1)) | (1u << (hi - L1));
            if (A != 0.0) p0o.push_back({ka, m});
            if (K != 0.0) p0z.push_back({kk, m});
        } else {  // across the cut: a = hi (in P_0), b = lo (in P_1)
            uint32_t abit = 1u << (hi - L1), bbit = 1u << lo;
            if (A != 0.0) xo[abit].push_back({ka, bbit});
            if (K != 0.0) xz.push_back({kk, {abit, bbit}});
        }
    }
    size_t n_p1b = 0;
    for (auto& e : p1o) n_p1b += e.second.size();
    if ((int)p1o.size() > kPanelMaxLayers || n_p1b > (size_t)kPanelMaxBonds || (int)p1z.size() > kPanelMaxLayers || (int)xo.size() > kPanelMaxGroups ||
        (int)p0o.size() > kPanelMaxBonds || (int)p0z.size() > kPanelMaxBonds || (int)xz.size() > kPanelMaxBonds)
        return DQ_OK;
    std::sort(p0o.begin(), p0o.end());
    std::sort(p0z.begin(), p0z.end());
    std::sort(xz.begin(), xz.end());
    {
        int q = 0;
        for (int k = 0; k < kPanelMaxA; ++k) {
            for (auto& e : p0o)
                if (e.first == k) P.p0_mask[q++] = e.second;
            P.p0_end[k] = q;
        }
        q = 0;
        for (auto& layer : p1o) {
            auto v = layer.second;
            std::sort(v.begin(), v.end());
            const int d = layer.first;
            P.p1l_d[P.n_p1l] = d;
            P.p1l_first[P.n_p1l] = q;
            for (auto& e : v)
                if (e.first == 0) {
                    P.p1b_lobit[q] = 1u << e.second;
                    P.p1b_pm2[q++] = ((1u << e.second) | (1u << (e.second + d))) << 1;
                }
            P.p1l_cut[P.n_p1l] = q;
            for (auto& e : v)
                if (e.first == 1) {
                    P.p1b_lobit[q] = 1u << e.second;
                    P.p1b_pm2[q++] = ((1u << e.second) | (1u << (e.second + d))) << 1;
                }
            P.p1l_end[P.n_p1l++] = q;
        }
        q = 0;
        for (int k = 0; k < kPanelMaxK; ++k) {
            for (auto& e : p0z)
                if (e.first == k) P.p0z_mask[q++] = e.second;
            P.p0z_end[k] = q;
        }
        q = 0;
        for (int k = 0; k < kPanelMaxK; ++k) {
            for (auto& e : p1z)
                if (e.first.first == k) {
                    P.p1z_d[q] = e.first.second;
                    P.p1z_mask[q++] = e.second;
                }
            P.p1z_end[k] = q;
        }
        q = 0;
        for (int k = 0; k < kPanelMaxK; ++k) {
            // at most 7 bonds of one class per (b, value of s_a): the kernel counts them in 3 bit planes
            std::map<uint32_t, int> mult;
            for (auto& e : xz)
                if (e.first == k) {
                    if (++mult[e.second.second] > 7) return DQ_OK;
                    P.xz_abit[q] = e.second.first;
                    P.xz_bbit[q++] = e.second.second;
                }
            P.xz_end[k] = q;
        }
        int nb = 0;
        size_t total = 0;
        for (auto& g : xo) total += g.second.size();
        if (total > (size_t)kPanelMaxBonds) return DQ_OK;
        for (auto& g : xo) {
            auto v = g.second;
            std::sort(v.begin(), v.end());
            P.xg_abit[P.n_xg] = g.first;
            P.xg_first[P.n_xg] = nb;
            for (auto& e : v) {
                if (e.first == 0) P.xb_bit[nb++] = e.second;
            }
            P.xg_cut[P.n_xg] = nb;
            for (auto& e : v) {
                if (e.first == 1) P.xb_bit[nb++] = e.second;
            }
            P.xg_end[P.n_xg++] = nb;
        }
    }
    P.nA = (int)Avals.size();
    P.nK = (int)Kvals.size();
    // common power of two of all coefficients
    std::vector<double> all = Avals;
    all.insert(all.end(), Kvals.begin(), Kvals.end());
    all.push_back(C);
    int emin = 1 << 20;
    for (double v : all)
        if (v != 0.0) emin = std::min(emin, low_exponent(v));
    if (emin == (1 << 20)) emin = 0;
    auto scaled = [&](double v, long long& out) -> bool {
        double m = std::ldexp(v, -emin);
        if (std::fabs(m) >= 9.0e15) return false;  // keep |M| < 2^53 so the sums below stay exact
        out = (long long)m;
        return (double)out == m;
    };
    if (!scaled(C, P.MC)) return DQ_OK;
    for (int k = 0; k < P.nK; ++k)
        if (!scaled(Kvals[k], P.MK[k])) return DQ_OK;
    for (int k = 0; k < P.nA; ++k)
        if (!scaled(Avals[k], P.MA[k])) return DQ_OK;
    P.emin = emin;
    // P_1 tables (local index within its particle-number sector, and the states per sector)
    std::vector<uint16_t> t1rank, t1states;
    if (!tail) {
        const int tl = s->dev.tab[ns - 1];
        const auto& rt = s->h.rank_tab[tl];
        const auto& ut = s->h.unrank_tab[tl];
        const auto& ss = s->h.sec_start[tl];
        t1rank.resize(rt.size());
        t1states.resize(ut.size());
        for (size_t q = 0; q < rt.size(); ++q) t1rank[q] = (uint16_t)(rt[q] == 0xffffffffu ? 0 : rt[q]);
        for (size_t q = 0; q < ut.size(); ++q) t1states[q] = (uint16_t)ut[q];
        for (int n = 0; n <= L1 + 1 && n < 18; ++n) {
            P.t1start[n] = ss[n <= L1 ? n : L1 + 1];
            P.t1len[n] = n <= L1 ? ss[n + 1] - ss[n] : 0;
        }
    } else {
        // the tail's order per particle number n: rank the tail patterns behind one prefix s0
        // with |s0| = N - n and subtract the smallest index
        t1rank.assign((size_t)1 << L1, 0);
        t1states.assign((size_t)1 << L1, 0);
        std::vector<std::vector<uint32_t>> byn(L1 + 1);
        for (uint32_t w = 0; w < (1u << L1); ++w) byn[__builtin_popcount(w)].push_back(w);
        uint32_t at = 0;
        for (int n = 0; n <= L1 + 1 && n < 18; ++n) {
            P.t1start[n] = at;
            P.t1len[n] = 0;
            if (n > L1) continue;
            const int n0 = N - n;
            if (n0 >= 0 && n0 <= L0) {
                const u128 rep = (u128)((1ull << n0) - 1) << L1;
                std::vector<uint64_t> r(byn[n].size());
                uint64_t lo = UINT64_MAX;
                for (size_t q = 0; q < byn[n].size(); ++q) lo = std::min(lo, r[q] = host_rank(s, rep | byn[n][q]));
                std::vector<char> hit(byn[n].size(), 0);
                for (size_t q = 0; q < byn[n].size(); ++q) {
                    const uint64_t c = r[q] - lo;
                    if (c >= byn[n].size() || hit[c]) return DQ_OK;  // not a contiguous range
                    hit[c] = 1;
                    t1rank[byn[n][q]] = (uint16_t)c;
                    t1states[at + c] = (uint16_t)byn[n][q];
                }
            } else {
                for (size_t q = 0; q < byn[n].size(); ++q) {
                    t1rank[byn[n][q]] = (uint16_t)q;
                    t1states[at + q] = (uint16_t)byn[n][q];
                }
            }
            P.t1len[n] = (uint32_t)byn[n].size();
            at += P.t1len[n];
        }
    }
    if (warp) return build_panel_w(s, P, t1rank, t1states, xz, t);
    // panels in canonical order: particle number of P_0, then its local order
    std::vector<uint32_t> ps0;
    std::vector<uint64_t> pst;
    int cmax = 0;
    std::vector<uint64_t> tail_start;  // first index of every prefix pattern's panel (tail form)
    if (!tail) {
        const auto& u0 = s->h.unrank_tab[s->dev.tab[0]];
        const auto& s0s = s->h.sec_start[s->dev.tab[0]];
        for (int n0 = 0; n0 <= L0; ++n0) {
            int n1 = N - n0;
            if (n1 < 0 || n1 > L1) continue;
            for (uint32_t q = s0s[n0]; q < s0s[n0 + 1]; ++q) {
                uint32_t p = u0[q];
                ps0.push_back(p);
                pst.push_back(s->h.c0_tab[p]);
            }
            cmax = std::max(cmax, (int)P.t1len[n1]);
        }
    } else {
        tail_start.assign((size_t)1 << L0, UINT64_MAX);
        std::vector<std::pair<uint64_t, uint32_t>> pl;
        for (uint32_t s0 = 0; s0 < (1u << L0); ++s0) {
            const int n1 = N - __builtin_popcount(s0);
            if (n1 < 0 || n1 > L1) continue;
            const u128 w = (u128)s0 << L1;
            const uint32_t C1 = P.t1len[n1];
            const uint64_t st = host_rank(s, w | t1states[P.t1start[n1]]);
            // the panel is the contiguous range [st, st + C1) in the tail's order
            if (host_rank(s, w | t1states[P.t1start[n1] + C1 - 1]) != st + C1 - 1) return DQ_OK;
            tail_start[s0] = st;
            pl.push_back({st, s0});
            cmax = std::max(cmax, (int)C1);
        }
        std::sort(pl.begin(), pl.end());
        for (auto& e : pl) {
            ps0.push_back(e.second);
            pst.push_back(e.first);
        }
    }
    auto start_of = [&](uint32_t p) -> uint64_t { return tail ? tail_start[p] : s->h.c0_tab[p]; };
    P.npanels = (uint32_t)ps0.size();
    P.cmax = cmax;
    // per-panel diagonal counters (see PanelDiag)
    std::vector<PanelDiag> pdiag(ps0.size());
    for (size_t q = 0; q < ps0.size(); ++q) {
        const uint32_t s0 = ps0[q];
        PanelDiag& g = pdiag[q];
        std::memset(&g, 0, sizeof g);
        for (int k = 0; k < P.nK; ++k) {
            for (int l = (k ? P.p0z_end[k - 1] : 0); l < P.p0z_end[k]; ++l)
                g.cnt0[k] += __builtin_popcount(s0 & P.p0z_mask[l]) == 1;
            int c0[32] = {0}, c1[32] = {0};  // per position b of P_1: bonds with s_a = 0 / s_a = 1
            for (int l = (k ? P.xz_end[k - 1] : 0); l < P.xz_end[k]; ++l) {
                const int b = __builtin_ctz(P.xz_bbit[l]);
                if (s0 & P.xz_abit[l])
                    ++c1[b];
                else
                    ++c0[b];
            }
            for (int b = 0; b < 32; ++b)
                for (int qq = 0; qq < 3; ++qq) {
                    g.w0[k][qq] |= (uint32_t)((c0[b] >> qq) & 1) << b;
                    g.w1[k][qq] |= (uint32_t)((c1[b] >> qq) & 1) << b;
                }
        }
    }
    // per-panel source lists
    std::vector<uint32_t> loff(ps0.size() + 1, 0), lhdr(ps0.size(), 0);
    std::vector<uint64_t> lst;
    lst.reserve(ps0.size() * 24);
    for (size_t q = 0; q < ps0.size(); ++q) {
        const uint32_t s0 = ps0[q];
        loff[q] = (uint32_t)lst.size();
        uint32_t cnt[kPanelMaxA] = {0, 0};
        for (int k = 0; k < kPanelMaxA; ++k)
            for (int l = (k ? P.p0_end[k - 1] : 0); l < P.p0_end[k]; ++l) {
                uint32_t m = P.p0_mask[l];
                if (__builtin_popcount(s0 & m) != 1) continue;
                lst.push_back(start_of(s0 ^ m));
                ++cnt[k];
            }
        uint32_t nx = 0;
        for (int g = 0; g < P.n_xg; ++g) {
            uint64_t src = start_of(s0 ^ P.xg_abit[g]);
            if (src == UINT64_MAX) continue;
            if (src >> 48) return DQ_OK;  // indices this large are left to the general kernel
            lst.push_back(src | ((uint64_t)g << 48));
            ++nx;
        }
        lhdr[q] = cnt[0] | (cnt[1] << 8) | (nx << 16);
    }
    loff[ps0.size()] = (uint32_t)lst.size();
    int rc;
    void* p;
    if ((rc = dev_upload(t->dev_allocs, ps0.data(), ps0.size() * 4, &p))) return rc;
    P.panel_s0 = (const uint32_t*)p;
    if ((rc = dev_upload(t->dev_allocs, pst.data(), pst.size() * 8, &p))) return rc;
    P.panel_start = (const uint64_t*)p;
    if ((rc = dev_upload(t->dev_allocs, t1rank.data(), t1rank.size() * 2, &p))) return rc;
    P.t1rank = (const uint16_t*)p;
    if ((rc = dev_upload(t->dev_allocs, t1states.data(), t1states.size() * 2, &p))) return rc;
    P.t1states = (const uint16_t*)p;
    if ((rc = dev_upload(t->dev_allocs, loff.data(), loff.size() * 4, &p))) return rc;
    P.list_off = (const uint32_t*)p;
    if ((rc = dev_upload(t->dev_allocs, lhdr.data(), lhdr.size() * 4, &p))) return rc;
    P.list_hdr = (const uint32_t*)p;
    if ((rc = dev_upload(t->dev_allocs, lst.data(), lst.size() * 8, &p))) return rc;
    P.list = (const uint64_t*)p;
    if ((rc = dev_upload(t->dev_allocs, pdiag.data(), pdiag.size() * sizeof(PanelDiag), &p))) return rc;
    P.diag = (const PanelDiag*)p;
    P.c0 = s->dev.c0_tab;
    t->panel_ok = true;
    return DQ_OK;
}

}  // namespace dq
