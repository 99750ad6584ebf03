// Compilation of operator terms into the device forms used by the product kernels.
//
// Q = 2 (one bit per site, spin-1/2 or hard-core bosons): with sigma_p the bit at position
// p = L-1-i of site i, every diagonal pair term reduces to a constant, single-site fields, and
// a coefficient of [sigma_i != sigma_j]:
//   ZZ:  c (s_i - 1/2)(s_j - 1/2) = c/4 - c/2 [s_i != s_j]
//   NN:  c s_i s_j               = c/2 s_i + c/2 s_j - c/2 [s_i != s_j]
// and every off-diagonal pair term flips both bits of a pair with s_i != s_j:
//   XY:  amplitude c/2;   HOP: amplitude -c   (b+_i b_j on Q = 2 is S+_i S-_j).
// Bonds are grouped into "layers" of equal bit distance, so that [s_p != s_{p+d}] over a whole
// layer is ((s ^ (s >> d)) & mask), and the per-bond work of the kernel is a popcount (uniform
// couplings) or a loop over the set bits (per-bond couplings).
//
// General Q (bosons): per-site digit functions f_i(n) from N and U, pair coefficients of
// n_i n_j from NN, and a list of hops with the amplitude table sqrt((n_a + 1) n_b).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

// Significant bits of the FP32-path coefficients: 24, fewer when a row can have so many hops
// that max_hops * 2^(bits + 30) would reach 2^62 (int64 hop sums of int32 x below 2^30).
static int fp32_mbits(int max_hops) {
    int lg = 0;
    while ((1 << lg) < std::max(max_hops, 1)) ++lg;
    return std::min(24, 32 - lg);
}

// Grids of the FP32 path: hop amplitudes (largest |c| = cmax_h) on 2^e_h with fp32_mbits(max_hops)
// bits, diagonal coefficients (largest cmax_d, at most tdiag unit terms per row) on a finer 2^e_d
// with up to 52 bits and the row's diagonal below 2^62. 0 <= e_h - e_d <= 60, so a row's hop sum
// (int64) shifted onto the diagonal grid fits in 128 bits.
static void fp32_grids(double cmax_h, double cmax_d, long long tdiag, int max_hops, int* e_h, int* e_d) {
    int lg = 0;
    while ((1ll << lg) < std::max(tdiag, 1ll)) ++lg;
    const int bd = std::min(52, 62 - lg), bh = fp32_mbits(max_hops);
    int eh = cmax_h > 0.0 ? std::ilogb(cmax_h) + 1 - bh : INT32_MIN / 2;
    int ed = cmax_d > 0.0 ? std::ilogb(cmax_d) + 1 - bd : INT32_MIN / 2;
    if (cmax_h <= 0.0 && cmax_d <= 0.0) eh = ed = 0;
    else if (cmax_h <= 0.0) eh = ed;
    else if (cmax_d <= 0.0) ed = eh;
    if (ed > eh) eh = ed;            // hops far below the diagonal: their grid coarsens
    if (eh - ed > 60) ed = eh - 60;  // diagonal far below the hops: its grid coarsens
    *e_h = eh;
    *e_d = ed;
}

static int compile_q2(const dq_sector* s, const dq_term* terms, int n, dq_terms* t) {
    const int L = s->L;
    double C = 0.0;
    double lin[64] = {0};
    std::map<std::pair<int, int>, std::pair<double, double>> pairs;  // (lo, d) -> (K, A)
    for (int q = 0; q < n; ++q) {
        const dq_term& u = terms[q];
        int pi = L - 1 - u.i;
        int pj = (u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_HOP || u.kind == DQ_NN) ? L - 1 - u.j : -1;
        int lo = pj < 0 ? -1 : (pi < pj ? pi : pj);
        int d = pj < 0 ? 0 : (pi < pj ? pj - pi : pi - pj);
        double c = u.coef;
        switch (u.kind) {
            case DQ_XY: pairs[{lo, d}].second += 0.5 * c; break;
            case DQ_HOP: pairs[{lo, d}].second += -c; break;
            case DQ_ZZ: C += 0.25 * c; pairs[{lo, d}].first += -0.5 * c; break;
            case DQ_NN:
                lin[pi] += 0.5 * c;
                lin[pj] += 0.5 * c;
                pairs[{lo, d}].first += -0.5 * c;
                break;
            case DQ_Z: lin[pi] += c; C += -0.5 * c; break;
            case DQ_N: lin[pi] += c; break;
            case DQ_U: break;  // n (n - 1) = 0 when n <= 1
        }
    }
    DevTermsQ2& v = t->q2v;
    std::memset(&v, 0, sizeof v);
    bool uniform_lin = true;
    for (int p = 1; p < L; ++p)
        if (lin[p] != lin[0]) uniform_lin = false;
    std::vector<double> pos;  // per-position tables, 64 entries each
    double Kh[kMaxLayers] = {0}, Ah[kMaxLayers] = {0};
    std::vector<double> lin_host;
    const double C_raw = C;  // before the uniform field is folded in (per-bond panel plan)
    if (uniform_lin) {
        C += lin[0] * s->N;  // sum_p lin sigma_p = lin * N on the sector
    } else {
        lin_host.assign(lin, lin + 64);
    }
    v.C = C;
    // group by distance
    std::map<int, std::vector<std::pair<int, std::pair<double, double>>>> byd;
    for (auto& kv : pairs) byd[kv.first.second].push_back({kv.first.first, kv.second});
    // A distance with at most three coefficient groups becomes one layer per group (uniform
    // coefficients); otherwise one per-position layer. If the grouped form would need more than
    // kMaxLayers layers, every distance with more than one group takes the per-position form, so
    // at most one layer per distance (at most 63) remains.
    int max_groups = 3;
    {
        int count = 0;
        for (auto& kv : byd) {
            std::map<std::pair<double, double>, int> g;
            for (auto& e : kv.second) g[e.second] = 1;
            int nz = 0;
            for (auto& e : g)
                if (e.first.first != 0.0 || e.first.second != 0.0) ++nz;
            count += g.size() <= 3 ? nz : 1;
        }
        if (count > kMaxLayers) max_groups = 1;
    }
    int nl = 0;
    int hops = 0;
    for (auto& kv : byd) {
        int d = kv.first;
        auto& lst = kv.second;
        std::map<std::pair<double, double>, uint64_t> groups;
        for (auto& e : lst) groups[e.second] |= 1ull << e.first;
        for (auto& e : lst)
            if (e.second.second != 0.0) ++hops;
        if ((int)groups.size() <= max_groups) {
            for (auto& g : groups) {
                if (g.first.first == 0.0 && g.first.second == 0.0) continue;
                if (nl >= kMaxLayers) return set_error(DQ_EINVAL, "too many bond layers");
                v.dist[nl] = d;
                v.dmask[nl] = g.first.first != 0.0 ? g.second : 0;
                v.omask[nl] = g.first.second != 0.0 ? g.second : 0;
                Kh[nl] = g.first.first;
                Ah[nl] = g.first.second;
                v.kpos[nl] = -1;
                v.apos[nl] = -1;
                ++nl;
            }
        } else {
            if (nl >= kMaxLayers) return set_error(DQ_EINVAL, "too many bond layers");
            v.dist[nl] = d;
            int kb = (int)pos.size();
            pos.resize(pos.size() + 64, 0.0);
            int ab = (int)pos.size();
            pos.resize(pos.size() + 64, 0.0);
            for (auto& e : lst) {
                if (e.second.first != 0.0) {
                    v.dmask[nl] |= 1ull << e.first;
                    pos[kb + e.first] = e.second.first;
                }
                if (e.second.second != 0.0) {
                    v.omask[nl] |= 1ull << e.first;
                    pos[ab + e.first] = e.second.second;
                }
            }
            v.kpos[nl] = kb;
            v.apos[nl] = ab;
            ++nl;
        }
    }
    v.nl = nl;
    t->max_hops = hops;
    {
        std::vector<std::pair<std::pair<int, int>, std::pair<double, double>>> plist(pairs.begin(), pairs.end());
        int rc = build_panel_plan(s, C, uniform_lin, plist, t);
        if (rc) return rc;
        if (!t->panel_ok && !t->pw_ok && (rc = build_panel_pb(s, C_raw, lin, plist, t))) return rc;
    }
    v.Cf = (float)v.C;
    // Fixed-point coefficients for FP64 vectors: one exponent emin for all of them, chosen so
    // that a row's diagonal (at most T_diag terms) stays below 2^62 in int64 and every hop
    // coefficient below 2^57 (128-bit row sums). Relative to the largest coefficient the
    // quantisation error is at most 2^-(Mbits+1).
    {
        double cmax = std::fabs(C);
        for (int l = 0; l < nl; ++l) cmax = std::max(cmax, std::max(std::fabs(Kh[l]), std::fabs(Ah[l])));
        for (double u : lin_host) cmax = std::max(cmax, std::fabs(u));
        for (double u : pos) cmax = std::max(cmax, std::fabs(u));
        int tdiag = 1 + (lin_host.empty() ? 0 : L);
        for (int l = 0; l < nl; ++l) tdiag += __builtin_popcountll(v.dmask[l]);
        int lg = 0;
        while ((1 << lg) < tdiag) ++lg;
        const int mbits = std::min(55, 62 - lg);
        v.emin = cmax > 0.0 ? std::ilogb(cmax) + 1 - mbits : 0;
        auto M = [&](double c) { return (long long)std::llrint(std::ldexp(c, -v.emin)); };
        v.MC = M(C);
        std::vector<long long> mka(2 * kMaxLayers, 0);
        for (int l = 0; l < nl; ++l) {
            mka[l] = M(Kh[l]);
            mka[kMaxLayers + l] = M(Ah[l]);
        }
        int rc0;
        void* q;
        if ((rc0 = dev_upload(t->dev_allocs, mka.data(), mka.size() * 8, &q))) return rc0;
        v.MKA = (const long long*)q;
        if (!lin_host.empty()) {
            std::vector<long long> ml(64, 0);
            for (int p = 0; p < 64; ++p) ml[p] = M(lin_host[p]);
            if ((rc0 = dev_upload(t->dev_allocs, ml.data(), ml.size() * 8, &q))) return rc0;
            v.Mlin = (const long long*)q;
        }
        if (!pos.empty()) {
            std::vector<long long> mp(pos.size());
            for (size_t k = 0; k < pos.size(); ++k) mp[k] = M(pos[k]);
            if ((rc0 = dev_upload(t->dev_allocs, mp.data(), mp.size() * 8, &q))) return rc0;
            v.Mpos = (const long long*)q;
        }
        // FP32 vectors: hop amplitudes with at most 24 bits, the diagonal on a finer grid
        {
            double cmax_h = 0.0, cmax_d = std::fabs(C);
            for (int l = 0; l < nl; ++l) {
                cmax_h = std::max(cmax_h, std::fabs(Ah[l]));
                cmax_d = std::max(cmax_d, std::fabs(Kh[l]));
            }
            for (double u : lin_host) cmax_d = std::max(cmax_d, std::fabs(u));
            for (int l = 0; l < nl; ++l) {
                if (v.kpos[l] >= 0)
                    for (int q2 = 0; q2 < 64; ++q2) cmax_d = std::max(cmax_d, std::fabs(pos[v.kpos[l] + q2]));
                if (v.apos[l] >= 0)
                    for (int q2 = 0; q2 < 64; ++q2) cmax_h = std::max(cmax_h, std::fabs(pos[v.apos[l] + q2]));
            }
            fp32_grids(cmax_h, cmax_d, tdiag, hops, &v.emin32, &v.emin32d);
        }
        auto md32 = [&](double c) { return (long long)std::llrint(std::ldexp(c, -v.emin32d)); };
        auto mh32 = [&](double c) { return (long long)std::llrint(std::ldexp(c, -v.emin32)); };
        v.MC32 = md32(C);
        std::vector<long long> mka32(2 * kMaxLayers, 0);
        for (int l = 0; l < nl; ++l) {
            mka32[l] = md32(Kh[l]);
            mka32[kMaxLayers + l] = mh32(Ah[l]);
        }
        if ((rc0 = dev_upload(t->dev_allocs, mka32.data(), mka32.size() * 8, &q))) return rc0;
        v.MKA32 = (const long long*)q;
        if (!lin_host.empty()) {
            std::vector<long long> ml(64, 0);
            for (int p = 0; p < 64; ++p) ml[p] = md32(lin_host[p]);
            if ((rc0 = dev_upload(t->dev_allocs, ml.data(), ml.size() * 8, &q))) return rc0;
            v.Mlin32 = (const long long*)q;
        }
        if (!pos.empty()) {
            std::vector<long long> mp(pos.size(), 0);
            for (int l = 0; l < nl; ++l) {
                if (v.kpos[l] >= 0)
                    for (int q2 = 0; q2 < 64; ++q2) mp[v.kpos[l] + q2] = md32(pos[v.kpos[l] + q2]);
                if (v.apos[l] >= 0)
                    for (int q2 = 0; q2 < 64; ++q2) mp[v.apos[l] + q2] = mh32(pos[v.apos[l] + q2]);
            }
            if ((rc0 = dev_upload(t->dev_allocs, mp.data(), mp.size() * 8, &q))) return rc0;
            v.Mpos32 = (const long long*)q;
        }
    }
    std::vector<float> kaf(2 * kMaxLayers, 0.f);
    std::vector<double> ka(2 * kMaxLayers, 0.0);
    for (int l = 0; l < nl; ++l) {
        ka[l] = Kh[l];
        ka[kMaxLayers + l] = Ah[l];
        kaf[l] = (float)Kh[l];
        kaf[kMaxLayers + l] = (float)Ah[l];
    }
    int rc;
    void* p;
    if ((rc = dev_upload(t->dev_allocs, ka.data(), ka.size() * 8, &p))) return rc;
    v.KA = (const double*)p;
    if ((rc = dev_upload(t->dev_allocs, kaf.data(), kaf.size() * 4, &p))) return rc;
    v.KAf = (const float*)p;
    if (!lin_host.empty()) {
        if ((rc = dev_upload(t->dev_allocs, lin_host.data(), 64 * 8, &p))) return rc;
        v.lin = (const double*)p;
        std::vector<float> lf(lin_host.begin(), lin_host.end());
        if ((rc = dev_upload(t->dev_allocs, lf.data(), lf.size() * 4, &p))) return rc;
        v.linf = (const float*)p;
    }
    if (!pos.empty()) {
        if ((rc = dev_upload(t->dev_allocs, pos.data(), pos.size() * 8, &p))) return rc;
        v.pos = (const double*)p;
        std::vector<float> pf(pos.begin(), pos.end());
        if ((rc = dev_upload(t->dev_allocs, pf.data(), pf.size() * 4, &p))) return rc;
        v.posf = (const float*)p;
    }
    return DQ_OK;
}

static int compile_qg(const dq_sector* s, const dq_term* terms, int n, dq_terms* t) {
    const int L = s->L, Q = s->Q, nb = s->nb;
    std::vector<std::vector<double>> f(L, std::vector<double>(Q, 0.0));
    std::map<std::pair<int, int>, double> nn;
    std::vector<int> hop_sh;
    std::vector<double> hop_t;
    double C = 0.0;  // constant part of the diagonal
    for (int q = 0; q < n; ++q) {
        const dq_term& u = terms[q];
        switch (u.kind) {
            // spin-1/2 kinds in this form (Q = 2, used for states of two words): Sz = n - 1/2,
            //   Z:  c Sz_i               = c n_i - c/2
            //   ZZ: c Sz_i Sz_j          = c n_i n_j - c/2 n_i - c/2 n_j + c/4
            //   XY: c/2 (S+_i S-_j + h.c.) = a hop with amplitude c/2, i.e. t = -c/2
            case DQ_Z:
                for (int d = 0; d < Q; ++d) f[u.i][d] += u.coef * d;
                C += -0.5 * u.coef;
                break;
            case DQ_ZZ:
                nn[{u.i < u.j ? u.i : u.j, u.i < u.j ? u.j : u.i}] += u.coef;
                for (int d = 0; d < Q; ++d) {
                    f[u.i][d] += -0.5 * u.coef * d;
                    f[u.j][d] += -0.5 * u.coef * d;
                }
                C += 0.25 * u.coef;
                break;
            case DQ_XY:
                hop_sh.push_back(nb * (L - 1 - u.i));
                hop_sh.push_back(nb * (L - 1 - u.j));
                hop_t.push_back(-0.5 * u.coef);
                break;
            case DQ_N:
                for (int d = 0; d < Q; ++d) f[u.i][d] += u.coef * d;
                break;
            case DQ_U:
                for (int d = 0; d < Q; ++d) f[u.i][d] += 0.5 * u.coef * d * (d - 1);
                break;
            case DQ_NN: nn[{u.i < u.j ? u.i : u.j, u.i < u.j ? u.j : u.i}] += u.coef; break;
            case DQ_HOP:
                hop_sh.push_back(nb * (L - 1 - u.i));
                hop_sh.push_back(nb * (L - 1 - u.j));
                hop_t.push_back(u.coef);
                break;
            default: return set_error(DQ_EINVAL, "unknown term kind %d", u.kind);
        }
    }
    DevTermsQG& v = t->qgv;
    std::memset(&v, 0, sizeof v);
    std::vector<int> site_sh;
    std::vector<double> site_f;
    for (int i = 0; i < L; ++i) {
        bool any = false;
        for (int d = 0; d < Q; ++d)
            if (f[i][d] != 0.0) any = true;
        if (!any) continue;
        site_sh.push_back(nb * (L - 1 - i));
        for (int d = 0; d < Q; ++d) site_f.push_back(f[i][d]);
    }
    std::vector<int> pair_sh;
    std::vector<double> pair_K;
    for (auto& kv : nn) {
        if (kv.second == 0.0) continue;
        pair_sh.push_back(nb * (L - 1 - kv.first.first));
        pair_sh.push_back(nb * (L - 1 - kv.first.second));
        pair_K.push_back(kv.second);
    }
    std::vector<double> amp((size_t)Q * Q, 0.0);
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) amp[(size_t)a * Q + b] = std::sqrt((double)((a + 1) * b));
    v.nsite = (int)site_sh.size();
    v.npair = (int)pair_K.size();
    v.nhop = (int)hop_t.size();
    t->max_hops = 2 * v.nhop;
    int rc;
    void* p;
    if ((rc = dev_upload(t->dev_allocs, site_sh.data(), site_sh.size() * 4, &p))) return rc;
    v.site_sh = (const int*)p;
    if ((rc = dev_upload(t->dev_allocs, pair_sh.data(), pair_sh.size() * 4, &p))) return rc;
    v.pair_sh = (const int*)p;
    if ((rc = dev_upload(t->dev_allocs, hop_sh.data(), hop_sh.size() * 4, &p))) return rc;
    v.hop_sh = (const int*)p;
    // Fixed-point coefficients for FP64 vectors, as for Q = 2 (compile_q2): one exponent emin,
    // a row's diagonal (at most T_diag unit terms, a pair counting (Q-1)^2) below 2^62 in int64,
    // every hop amplitude below 2^55.
    {
        std::vector<double> hop_amp((size_t)v.nhop * Q * Q, 0.0);
        for (int q = 0; q < v.nhop; ++q)
            for (int a = 0; a < Q - 1; ++a)
                for (int b = 1; b < Q; ++b) hop_amp[((size_t)q * Q + a) * Q + b] = -hop_t[q] * amp[(size_t)a * Q + b];
        double cmax = std::fabs(C);
        for (double u : site_f) cmax = std::max(cmax, std::fabs(u));
        for (double u : pair_K) cmax = std::max(cmax, std::fabs(u));
        for (double u : hop_amp) cmax = std::max(cmax, std::fabs(u));
        const long long tdiag = 1 + (long long)v.nsite + (long long)v.npair * (Q - 1) * (Q - 1);
        int lg = 0;
        while ((1ll << lg) < tdiag) ++lg;
        const int mbits = std::min(55, 62 - lg);
        v.emin = cmax > 0.0 ? std::ilogb(cmax) + 1 - mbits : 0;
        auto M = [&](double c) { return (long long)std::llrint(std::ldexp(c, -v.emin)); };
        v.MC = M(C);
        auto upm = [&](const std::vector<double>& src, const long long** dst) -> int {
            std::vector<long long> m(src.size());
            for (size_t k = 0; k < src.size(); ++k) m[k] = M(src[k]);
            void* q;
            int r = dev_upload(t->dev_allocs, m.data(), m.size() * 8, &q);
            *dst = (const long long*)q;
            return r;
        };
        if ((rc = upm(site_f, &v.Msite))) return rc;
        if ((rc = upm(pair_K, &v.Mpair))) return rc;
        if ((rc = upm(hop_amp, &v.Mhop))) return rc;
        {
            // the boson panel product takes the same integer coefficients
            std::vector<long long> msite(site_f.size()), mhop(hop_amp.size());
            for (size_t k = 0; k < site_f.size(); ++k) msite[k] = M(site_f[k]);
            for (size_t k = 0; k < hop_amp.size(); ++k) mhop[k] = M(hop_amp[k]);
            if ((rc = build_panel_q(s, site_sh, msite, hop_sh, mhop, v.MC, v.emin, v.npair, t))) return rc;
        }
        // FP32 vectors: hop amplitudes with at most 24 bits (int32), the diagonal on a finer grid
        {
            double cmax_h = 0.0, cmax_d = std::fabs(C);
            for (double u : hop_amp) cmax_h = std::max(cmax_h, std::fabs(u));
            for (double u : site_f) cmax_d = std::max(cmax_d, std::fabs(u));
            for (double u : pair_K) cmax_d = std::max(cmax_d, std::fabs(u));
            fp32_grids(cmax_h, cmax_d, tdiag, 2 * v.nhop, &v.emin32, &v.emin32d);
        }
        v.MC32 = (long long)std::llrint(std::ldexp(C, -v.emin32d));
        auto upd = [&](const std::vector<double>& src, const long long** dst) -> int {
            std::vector<long long> m(src.size());
            for (size_t k = 0; k < src.size(); ++k) m[k] = (long long)std::llrint(std::ldexp(src[k], -v.emin32d));
            void* q;
            int r = dev_upload(t->dev_allocs, m.data(), m.size() * 8, &q);
            *dst = (const long long*)q;
            return r;
        };
        std::vector<int> mh(hop_amp.size());
        for (size_t k = 0; k < hop_amp.size(); ++k) mh[k] = (int)std::llrint(std::ldexp(hop_amp[k], -v.emin32));
        if ((rc = upd(site_f, &v.Msite32))) return rc;
        if ((rc = upd(pair_K, &v.Mpair32))) return rc;
        if ((rc = dev_upload(t->dev_allocs, mh.data(), mh.size() * 4, &p))) return rc;
        v.Mhop32 = (const int*)p;
    }
    return DQ_OK;
}

int check_terms(const dq_sector* s, const dq_term* terms, int n_terms) {
    for (int q = 0; q < n_terms; ++q) {
        const dq_term& u = terms[q];
        if (u.kind < DQ_XY || u.kind > DQ_U) return set_error(DQ_EINVAL, "term %d: unknown kind %d", q, u.kind);
        if (u.i < 0 || u.i >= s->L) return set_error(DQ_EINVAL, "term %d: site i out of range", q);
        bool pair = u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_HOP || u.kind == DQ_NN;
        if (pair && (u.j < 0 || u.j >= s->L || u.j == u.i))
            return set_error(DQ_EINVAL, "term %d: pair term needs two distinct sites in range", q);
        bool spin = u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_Z;
        if (spin && s->Q != 2) return set_error(DQ_EINVAL, "term %d: spin-1/2 kinds need Q = 2", q);
        if (!std::isfinite(u.coef)) return set_error(DQ_EINVAL, "term %d: coefficient is not finite", q);
    }
    return DQ_OK;
}

}  // namespace dq

using namespace dq;

extern "C" {

int dq_make_terms(const dq_sector* s, const dq_term* terms, int n_terms, dq_terms** out) {
    clear_error();
    if (!s || !out || (n_terms > 0 && !terms) || n_terms < 0) return set_error(DQ_EINVAL, "bad argument");
    *out = nullptr;
    if (int rc = check_terms(s, terms, n_terms)) return rc;
    dq_terms* t = new (std::nothrow) dq_terms();
    if (!t) return set_error(DQ_ENOMEM, "host allocation");
    t->sector = s;
    // Q = 2 takes the bond-layer form (64-bit words only); general Q, and every sector whose
    // states take two words, the per-term form
    t->q2 = (s->Q == 2) && !s->wide;
    int rc;
    try {
        rc = t->q2 ? compile_q2(s, terms, n_terms, t) : compile_qg(s, terms, n_terms, t);
    } catch (...) {
        rc = set_error(DQ_ENOMEM, "host allocation failed while compiling terms");
    }
    if (rc) {
        for (void* p : t->dev_allocs) cudaFree(p);
        delete t;
        return rc;
    }
    *out = t;
    return DQ_OK;
}

int dq_terms_path(const dq_terms* t, int* path) {
    clear_error();
    if (!t || !path) return set_error(DQ_EINVAL, "NULL argument");
    *path = t->cluster ? 2 : (t->panel_ok ? 1 : (t->pw_ok ? 4 : (t->pb_ok ? 3 : (t->pq_ok ? 5 : 0))));
    return DQ_OK;
}

void dq_free_terms(dq_terms* t) {
    if (!t) return;
    if (t->scratch) cudaFree(t->scratch);
    for (void* p : t->dev_allocs) cudaFree(p);
    delete t;
}

}  // extern "C"
