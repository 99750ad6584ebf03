// Cluster-merged operator (App. C): all terms that lie inside one cluster of sites are merged
// into one sparse matrix over the cluster's digit patterns, so a row applies one precomputed
// column per cluster instead of every term one by one.
//
// Host (dq_make_cluster_terms): the terms are assigned to clusters of at most m sites (clusters
// may overlap; a term goes to the first cluster that holds its sites, or that can take them
// without growing past m sites, else it opens a new one). For every cluster c and every digit
// pattern p of its sites, the column S_c[., p] is built by applying the cluster's terms to the
// local state p with the conventions of the term kinds (include/dq.h); an entry is stored as the
// XOR mask between the word with pattern p and the word with pattern p' (the cluster's digits
// deposited at their bit positions), and the coefficient as an integer M on one grid 2^emin.
// The operator is real symmetric, so column p is also row p: the gather form of the product
// reads, for row word s with cluster pattern p, the entries of column p.
//
// Device (k_matvec_cl): per row (the warp walk of the general kernels), per cluster: the pattern
// p from the digits of the cluster's sites; the diagonal entries add into an int64 sum; every
// other entry ranks s ^ mask by Eq. (index) and adds M X[j] to a 128-bit row sum (exact fixed
// point, x scaled per column to int64 by the prepass, one rounding per y_i).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "dq_device.cuh"
#include "dq_fixed.cuh"
#include "dq_internal.h"

namespace dq {

// ------------------------------------------------------------------ host: clusters ----------

struct HostCluster {
    std::vector<int> sites;   // cluster site k holds pattern digit k
    std::vector<int> terms;   // indices of the terms merged here
};

static int site_pos(const HostCluster& c, int site) {
    for (size_t k = 0; k < c.sites.size(); ++k)
        if (c.sites[k] == site) return (int)k;
    return -1;
}

// Greedy assignment of terms to clusters of at most m sites, in the order of the terms sorted by
// their sites.
static std::vector<HostCluster> make_clusters(const dq_term* terms, int n, int m) {
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    auto sites_of = [&](int q) {
        const dq_term& u = terms[q];
        const bool pair = u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_HOP || u.kind == DQ_NN;
        std::vector<int> v{u.i};
        if (pair) v.push_back(u.j);
        std::sort(v.begin(), v.end());
        return v;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sites_of(a) < sites_of(b); });
    std::vector<HostCluster> cl;
    for (int q : order) {
        const std::vector<int> st = sites_of(q);
        int best = -1, best_new = 1 << 30;
        for (size_t c = 0; c < cl.size(); ++c) {
            int add = 0;
            for (int x : st) add += site_pos(cl[c], x) < 0;
            if ((int)cl[c].sites.size() + add <= m && add < best_new) {
                best = (int)c;
                best_new = add;
                if (add == 0) break;
            }
        }
        if (best < 0) {
            cl.push_back(HostCluster());
            best = (int)cl.size() - 1;
        }
        for (int x : st)
            if (site_pos(cl[best], x) < 0) cl[best].sites.push_back(x);
        cl[best].terms.push_back(q);
    }
    return cl;
}

// Column p of a cluster's matrix: the terms applied to the local state with digits d (site k
// of the cluster holds d[k]); returns pattern -> value, the diagonal under p itself.
static void apply_cluster(const HostCluster& c, const dq_term* terms, int Q, int nb, uint32_t p,
                          std::map<uint32_t, double>& col) {
    const int ns = (int)c.sites.size();
    const uint32_t dm = (1u << nb) - 1;
    std::vector<int> d(ns);
    for (int k = 0; k < ns; ++k) d[k] = (int)((p >> (nb * k)) & dm);
    auto pat = [&](const std::vector<int>& dd) {
        uint32_t r = 0;
        for (int k = 0; k < ns; ++k) r |= (uint32_t)dd[k] << (nb * k);
        return r;
    };
    for (int q : c.terms) {
        const dq_term& u = terms[q];
        const int a = site_pos(c, u.i);
        const int b = (u.kind == DQ_XY || u.kind == DQ_ZZ || u.kind == DQ_HOP || u.kind == DQ_NN) ? site_pos(c, u.j) : -1;
        switch (u.kind) {
            case DQ_ZZ: col[p] += u.coef * (d[a] - 0.5) * (d[b] - 0.5); break;
            case DQ_Z: col[p] += u.coef * (d[a] - 0.5); break;
            case DQ_NN: col[p] += u.coef * d[a] * d[b]; break;
            case DQ_N: col[p] += u.coef * d[a]; break;
            case DQ_U: col[p] += 0.5 * u.coef * d[a] * (d[a] - 1); break;
            case DQ_XY:
                if (d[a] != d[b]) {
                    std::vector<int> e = d;
                    std::swap(e[a], e[b]);
                    col[pat(e)] += 0.5 * u.coef;
                }
                break;
            case DQ_HOP:
                for (int dir = 0; dir < 2; ++dir) {  // b+_up b_dn, then its conjugate
                    const int up = dir ? b : a, dn = dir ? a : b;
                    if (d[up] < Q - 1 && d[dn] > 0) {
                        std::vector<int> e = d;
                        e[up] += 1;
                        e[dn] -= 1;
                        col[pat(e)] += -u.coef * std::sqrt((double)((d[up] + 1) * d[dn]));
                    }
                }
                break;
        }
    }
}

static int build_clusters(const dq_sector* s, const dq_term* terms, int n, int m, dq_terms* t) {
    const int Q = s->Q, nb = s->nb, L = s->L;
    std::vector<HostCluster> cl = make_clusters(terms, n, m);
    if ((int)cl.size() > kClMax) return set_error(DQ_EINVAL, "the terms need %zu clusters of %d sites; at most %d",
                                                  cl.size(), m, kClMax);
    std::vector<int> nsite(cl.size()), sh(cl.size() * kClMaxSites, 0), col_base(cl.size());
    std::vector<uint32_t> col_off;
    std::vector<uint64_t> dlo, dhi;
    std::vector<double> coef;
    long long max_row = 0;  // most entries a row can meet (sum over clusters of the longest column)
    for (size_t c = 0; c < cl.size(); ++c) {
        const int ns = (int)cl[c].sites.size();
        nsite[c] = ns;
        for (int k = 0; k < ns; ++k) sh[c * kClMaxSites + k] = nb * (L - 1 - cl[c].sites[k]);
        col_base[c] = (int)col_off.size();
        const uint32_t npat = 1u << (nb * ns);
        int longest = 0;
        for (uint32_t p = 0; p < npat; ++p) {
            col_off.push_back((uint32_t)coef.size());
            bool valid = true;
            for (int k = 0; k < ns; ++k)
                if ((int)((p >> (nb * k)) & ((1u << nb) - 1)) >= Q) valid = false;
            if (!valid) continue;
            std::map<uint32_t, double> col;
            apply_cluster(cl[c], terms, Q, nb, p, col);
            int cnt = 0;
            // diagonal first, then the other patterns in ascending order
            for (int pass = 0; pass < 2; ++pass)
                for (auto& e : col) {
                    if ((e.first == p) != (pass == 0) || e.second == 0.0) continue;
                    unsigned __int128 mask = 0;
                    const uint32_t x = e.first ^ p;
                    for (int k = 0; k < ns; ++k)
                        mask |= (unsigned __int128)((x >> (nb * k)) & ((1u << nb) - 1)) << sh[c * kClMaxSites + k];
                    dlo.push_back((uint64_t)mask);
                    dhi.push_back((uint64_t)(mask >> 64));
                    coef.push_back(e.second);
                    ++cnt;
                }
            longest = std::max(longest, cnt);
        }
        col_off.push_back((uint32_t)coef.size());
        max_row += longest;
    }
    // one grid 2^emin: |M| < 2^mbits, and a row's at most max_row products M X (|X| < 2^56) and
    // its diagonal sum stay below 2^126 in the 128-bit row sum
    double cmax = 0.0;
    for (double v : coef) cmax = std::max(cmax, std::fabs(v));
    int lg = 0;
    while ((1ll << lg) < std::max(max_row, 1ll)) ++lg;
    const int mbits = std::min(55, 126 - 56 - lg);
    DevTermsCL& v = t->clv;
    std::memset(&v, 0, sizeof v);
    v.ncl = (int)cl.size();
    v.emin = cmax > 0.0 ? std::ilogb(cmax) + 1 - mbits : 0;
    std::vector<long long> M(coef.size());
    for (size_t e = 0; e < coef.size(); ++e) M[e] = (long long)std::llrint(std::ldexp(coef[e], -v.emin));
    int rc;
    void* p;
    if ((rc = dev_upload(t->dev_allocs, nsite.data(), nsite.size() * 4, &p))) return rc;
    v.nsite = (const int*)p;
    if ((rc = dev_upload(t->dev_allocs, sh.data(), sh.size() * 4, &p))) return rc;
    v.sh = (const int*)p;
    if ((rc = dev_upload(t->dev_allocs, col_base.data(), col_base.size() * 4, &p))) return rc;
    v.col_base = (const int*)p;
    if ((rc = dev_upload(t->dev_allocs, col_off.data(), col_off.size() * 4, &p))) return rc;
    v.col_off = (const uint32_t*)p;
    if ((rc = dev_upload(t->dev_allocs, dlo.data(), dlo.size() * 8, &p))) return rc;
    v.dlo = (const uint64_t*)p;
    if ((rc = dev_upload(t->dev_allocs, dhi.data(), dhi.size() * 8, &p))) return rc;
    v.dhi = (const uint64_t*)p;
    if ((rc = dev_upload(t->dev_allocs, M.data(), M.size() * 8, &p))) return rc;
    v.M = (const long long*)p;
    t->max_hops = (int)std::min<long long>(max_row, 1 << 30);
    t->cl_sites.assign(cl.size() * kClMaxSites, -1);
    for (size_t c = 0; c < cl.size(); ++c)
        for (size_t k = 0; k < cl[c].sites.size(); ++k) t->cl_sites[c * kClMaxSites + k] = cl[c].sites[k];
    return DQ_OK;
}

// ------------------------------------------------------------------ device ------------------

template <typename W>
__device__ __forceinline__ W cl_mask(const DevTermsCL& H, uint32_t e) {
    if constexpr (sizeof(W) == 8)
        return (W)__ldg(H.dlo + e);
    else
        return ((W)__ldg(H.dhi + e) << 64) | (W)__ldg(H.dlo + e);
}

// y = H x in the cluster-merged form, x in int64 fixed point (both vector precisions), CH
// right-hand sides per pass, rows walked as in the general kernels.
template <typename W, typename OUT, int CH>
__global__ void __launch_bounds__(256)
    k_matvec_cl(DevSector S, DevTermsCL H, const long long* __restrict__ X, OUT* __restrict__ y,
                const ColScale* __restrict__ hdr, int ld, int col0, int ch, bool use_sm, int R) {
    extern __shared__ uint64_t sm[];
    const uint64_t *off_s, *str_s;
    stage_os(S, sm, use_sm, off_s, str_s);
    if (hdr->bad) {  // an Inf or NaN in x: y is NaN and the error word is raised
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S.D; i += (uint64_t)gridDim.x * blockDim.x)
            for (int c = 0; c < ch; ++c) y[i * ld + col0 + c] = (OUT)NAN;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(S.err, 1);
        return;
    }
    int sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sc[c] = c < ch ? H.emin - hdr->F[col0 + c] : 0;
    const uint32_t dm = (1u << S.nb) - 1;
    const uint64_t wid_ = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp_ = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t span_ = 32ull * (uint64_t)R;
    for (uint64_t base_ = wid_ * span_; base_ < S.D; base_ += nwarp_ * span_) {
        RowWalk<W> rw;
        uint64_t i = base_ + (threadIdx.x & 31);
        for (int r_ = 0; r_ < R && i < S.D; ++r_, i += 32) {
            if (r_ == 0)
                walk_start(S, off_s, str_s, i, rw);
            else
                walk_next(S, off_s, str_s, i, rw);
            const W s = rw.s;
            long long md = 0;
            I128 r[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) r[c] = {0, 0};
            for (int q = 0; q < H.ncl; ++q) {
                const int ns = __ldg(H.nsite + q);
                uint32_t p = 0;
                for (int k = 0; k < ns; ++k)
                    p |= ((uint32_t)(s >> __ldg(H.sh + q * kClMaxSites + k)) & dm) << (S.nb * k);
                const uint32_t* co = H.col_off + __ldg(H.col_base + q);
                const uint32_t e1 = __ldg(co + p + 1);
                for (uint32_t e = __ldg(co + p); e < e1; ++e) {
                    const W mk = cl_mask<W>(H, e);
                    const long long M = __ldg(H.M + e);
                    if (mk == 0) {
                        md += M;
                    } else {
                        const uint64_t j = d_rank(S, off_s, str_s, s ^ mk);
                        const long long* Xj = X + j * ld + col0;
#pragma unroll
                        for (int c = 0; c < CH; ++c)
                            if (c < ch) mac(r[c], M, __ldg(Xj + c));
                    }
                }
            }
            const long long* Xi = X + i * ld + col0;
            OUT* yi = y + i * ld + col0;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (c < ch) {
                    mac(r[c], md, __ldg(Xi + c));
                    yi[c] = i128_to<OUT>(r[c], sc[c]);
                }
        }
    }
}

template <typename W, typename T>
static int run_cluster(const dq_sector* s, dq_terms* t, const T* x, T* y, int nrhs, cudaStream_t st) {
    const size_t need = kColScaleBytes + (size_t)s->D * nrhs * sizeof(long long);
    if (t->scratch_bytes < need) {
        if (t->scratch) cudaFree(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&t->scratch, need);
        if (e != cudaSuccess) return (int)e;
        t->scratch_bytes = need;
    }
    ColScale* h = reinterpret_cast<ColScale*>(t->scratch);
    long long* X = reinterpret_cast<long long*>(reinterpret_cast<char*>(t->scratch) + kColScaleBytes);
    const int sms = sm_count_cached();
    launch_col_prepass<T, long long>(x, X, s->D, nrhs, h, sms, st);
    const DevSector& S = s->dev;
    const size_t osb = (size_t)S.os_total * 16;
    const bool sm = osb <= 48 * 1024;
    const size_t smb = sm ? osb : 0;
    const int tslot = timing_start(st);
    int passes = 0;
    constexpr int kCh = 8;
    for (int c0 = 0; c0 < nrhs; c0 += kCh, ++passes) {
        const int ch = nrhs - c0 < kCh ? nrhs - c0 : kCh;
        auto kern = nrhs == 1 ? k_matvec_cl<W, T, 1> : k_matvec_cl<W, T, kCh>;
        const int per_sm = occupancy_cached(reinterpret_cast<const void*>(kern), 256, smb);
        const uint64_t need_blocks = (s->D + 255) / 256, cap = (uint64_t)sms * per_sm;
        const unsigned grid = (unsigned)(need_blocks < cap ? (need_blocks ? need_blocks : 1) : cap);
        uint64_t R = s->D / ((uint64_t)grid * 256 * 4);
        R = R < 1 ? 1 : (R > 16 ? 16 : R);
        kern<<<grid, 256, smb, st>>>(S, t->clv, X, y, h, nrhs, c0, ch, sm, (int)R);
    }
    timing_stop(tslot, st, 2 + passes);
    return (int)cudaGetLastError();
}

int launch_cluster_matvec(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DQ_F64) {
        if (s->wide) return run_cluster<u128, double>(s, t, (const double*)x, (double*)y, nrhs, st);
        return run_cluster<uint64_t, double>(s, t, (const double*)x, (double*)y, nrhs, st);
    }
    if (s->wide) return run_cluster<u128, float>(s, t, (const float*)x, (float*)y, nrhs, st);
    return run_cluster<uint64_t, float>(s, t, (const float*)x, (float*)y, nrhs, st);
}

}  // namespace dq

using namespace dq;

extern "C" int dq_make_cluster_terms(const dq_sector* s, const dq_term* terms, int n_terms, int cluster_sites,
                                     dq_terms** out) {
    clear_error();
    if (!s || !out || (n_terms > 0 && !terms) || n_terms < 0) return set_error(DQ_EINVAL, "bad argument");
    *out = nullptr;
    if (cluster_sites < 2 || cluster_sites > kClMaxSites || s->nb * cluster_sites > 12)
        return set_error(DQ_EINVAL, "cluster_sites must be in [2, %d] with Nbits * cluster_sites <= 12", kClMaxSites);
    if (int rc = check_terms(s, terms, n_terms)) return rc;
    dq_terms* t = new (std::nothrow) dq_terms();
    if (!t) return set_error(DQ_ENOMEM, "host allocation");
    t->sector = s;
    t->q2 = false;
    t->cluster = true;
    int rc;
    try {
        rc = build_clusters(s, terms, n_terms, cluster_sites, t);
    } catch (...) {
        rc = set_error(DQ_ENOMEM, "host allocation failed while building clusters");
    }
    if (rc) {
        for (void* p : t->dev_allocs) cudaFree(p);
        delete t;
        return rc;
    }
    *out = t;
    return DQ_OK;
}

extern "C" int dq_cluster_info(const dq_terms* t, int* n_clusters, int* sites, int* entries) {
    clear_error();
    if (!t || !n_clusters) return set_error(DQ_EINVAL, "NULL argument");
    if (!t->cluster) return set_error(DQ_EINVAL, "the terms are not in the cluster-merged form");
    *n_clusters = t->clv.ncl;
    if (sites)
        for (size_t q = 0; q < t->cl_sites.size(); ++q) sites[q] = t->cl_sites[q];
    if (entries) *entries = t->max_hops;
    return DQ_OK;
}
