// Host sector builder and the host forms of the paper's three basis functions.
//
//  - D_Q(l, m) from Eq. (dim) (App. A): alternating binomial sum, exact in 128-bit integers.
//  - offset_k(n, lambda) and stride_k(n, lambda): Eq. (offset) and Eq. (stride) of Sec. 3.2,
//    with Gamma_k the length of the complement after P_k.
//  - local rank tables ("memory-aligned list", Sec. 4.2 container (i)), filled with the
//    on-the-fly rank of Alg. 1 (Eq. (N=L)) applied to each subsystem on its own.
//  - get_index (Alg. 2), increment (Alg. 3), get_state (Alg. 4).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

bool device_present() {
    static int present = -1;
    if (present < 0) {
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess) {
            n = 0;
            cudaGetLastError();  // clear the runtime's "no device" status
        }
        present = n > 0;
    }
    return present == 1;
}

int sm_count_cached() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    cache[dev] = sms;
    return sms;
}

int occupancy_cached(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(kernel, threads, smem, dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    cache[key] = per_sm;
    return per_sm;
}

int dev_upload(std::vector<void*>& allocs, const void* host, size_t bytes, void** dptr) {
    *dptr = nullptr;
    if (!device_present()) return DQ_OK;  // host-only object on a machine without a GPU
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return set_error(DQ_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    allocs.push_back(p);
    if (host) {
        e = cudaMemcpy(p, host, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return set_error(DQ_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    *dptr = p;
    return DQ_OK;
}

static const uint64_t kSat = UINT64_MAX;

// Binomial C(n, k) in 128-bit (exact for the sizes allowed here); 0 outside 0 <= k <= n.
static __int128 binom(long n, long k) {
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    __int128 c = 1;
    for (long i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

// Eq. (dim): D_Q(l, m) = sum_{k=0}^{floor(m/Q)} (-1)^k C(l, k) C(l - 1 + m - Qk, l - 1), with the
// conventions D_Q(0, 0) = 1 and D_Q(l, m) = 0 for m < 0 or m > (Q-1) l. For Q = 2 the sum is
// C(l, m) (Sec. 2.1), used directly to keep the partial sums small. Saturates at UINT64_MAX.
static uint64_t dq_eq_dim(int l, int Q, long m) {
    if (m < 0 || m > (long)(Q - 1) * l) return 0;
    if (l == 0) return m == 0 ? 1 : 0;
    __int128 r;
    if (Q == 2) {
        r = binom(l, m);
    } else {
        r = 0;
        for (long k = 0; k <= m / Q; ++k) {
            __int128 t = binom(l, k) * binom(l - 1 + m - (long)Q * k, l - 1);
            r += (k & 1) ? -t : t;
        }
    }
    if (r < 0) return 0;
    if (r >= (__int128)kSat) return kSat;
    return (uint64_t)r;
}

static inline uint64_t Dq(const dq_sector* s, int l, long m) {
    if (l < 0 || m < 0 || m > (long)(s->Q - 1) * l) return 0;
    return s->h.Dq[(size_t)l * s->h.dq_ld + (size_t)m];
}

// States are handled as 128-bit words on the host; a one-word state is the low word.
static inline int digit(const dq_sector* s, u128 w, int site) {
    return (int)((uint32_t)(w >> (s->nb * (s->L - 1 - site))) & ((1u << s->nb) - 1));
}

static inline uint32_t field(const dq_sector* s, u128 w, int k) {
    return (uint32_t)(w >> s->dev.shift[k]) & (uint32_t)((1ull << (s->nb * s->Lk[k])) - 1);
}

static int pattern_n(int nb, uint32_t pat, int len) {
    int n = 0;
    for (int i = 0; i < len; ++i) n += (pat >> (nb * i)) & ((1u << nb) - 1);
    return n;
}

bool host_valid_state(const dq_sector* s, u128 w) {
    int bits = s->L * s->nb;
    if (bits < 128 && (w >> bits) != 0) return false;
    int n = 0;
    for (int i = 0; i < s->L; ++i) {
        int d = digit(s, w, i);
        if (d >= s->Q) return false;
        n += d;
    }
    return n == s->N;
}

// Alg. 2 (function (i), get_index): index = sum_k offset_k(n_k, lambda_k) + stride_k * index_k.
uint64_t host_rank(const dq_sector* s, u128 w) {
    uint64_t idx = 0;
    int lam = 0;
    for (int k = 0; k < s->n_sub; ++k) {
        uint32_t f = field(s, w, k);
        int t = s->dev.tab[k];
        int n = pattern_n(s->nb, f, s->Lk[k]);
        uint64_t li = s->h.rank_tab[t][f];
        size_t o = (size_t)s->dev.os_base[k] + (size_t)lam * s->dev.os_ld[k] + n;
        idx += s->h.off[o] + s->h.str[o] * li;
        lam += n;
    }
    return idx;
}

// Alg. 4 (function (iii), get_state): per subsystem, the particle number is the n with
// offset(n) <= idx < offset(n+1); the local index is the quotient by the stride.
u128 host_unrank(const dq_sector* s, uint64_t idx) {
    u128 w = 0;
    int lam = 0;
    for (int k = 0; k < s->n_sub; ++k) {
        int t = s->dev.tab[k];
        size_t row = (size_t)s->dev.os_base[k] + (size_t)lam * s->dev.os_ld[k];
        int n = 0;
        if (k == s->n_sub - 1) {
            n = s->N - lam;
        } else {
            while (n <= s->dev.nmax[k] && !(s->h.off[row + n] <= idx && idx < s->h.off[row + n + 1])) ++n;
        }
        uint64_t rem = idx - s->h.off[row + n];
        uint64_t st = s->h.str[row + n];
        uint64_t li = (k == s->n_sub - 1) ? rem : rem / st;
        idx = rem - li * st;
        uint32_t pat = s->h.unrank_tab[t][s->h.sec_start[t][n] + li];
        w |= (u128)pat << s->dev.shift[k];
        lam += n;
    }
    return w;
}

// Minimal state of `len` sites holding n particles: particles as far right as possible
// (index 0 of the canonical order, App. B get_minimal_state). Returned right-aligned.
static u128 minimal_state(int nb, int Q, int len, int n) {
    u128 w = 0;
    for (int i = 0; i < len && n > 0; ++i) {  // i counts sites from the right end
        int d = n < Q - 1 ? n : Q - 1;
        w |= (u128)d << (nb * i);
        n -= d;
    }
    return w;
}

// Alg. 3 (function (ii), increment).
static u128 host_increment(const dq_sector* s, u128 w) {
    int lam = 0;    // particles in the suffix after P_k
    int gamma = 0;  // sites in that suffix
    for (int j = 1; j <= s->n_sub; ++j) {
        int k = s->n_sub - j;
        uint32_t f = field(s, w, k);
        int t = s->dev.tab[k];
        int n = pattern_n(s->nb, f, s->Lk[k]);
        uint64_t li = s->h.rank_tab[t][f];
        uint64_t dim_local = Dq(s, s->Lk[k], n);
        const int top = s->dev.shift[k] + s->nb * s->Lk[k];
        const u128 keep_mask = top >= 128 ? (u128)0 : (~(u128)0 << top);
        if (li + 1 < dim_local) {
            uint32_t nxt = s->h.unrank_tab[t][s->h.sec_start[t][n] + li + 1];
            return (w & keep_mask) | ((u128)nxt << s->dev.shift[k]) | minimal_state(s->nb, s->Q, gamma, lam);
        } else if (lam > 0 && n < (s->Q - 1) * s->Lk[k]) {
            u128 pk = minimal_state(s->nb, s->Q, s->Lk[k], n + 1);
            return (w & keep_mask) | (pk << s->dev.shift[k]) | minimal_state(s->nb, s->Q, gamma, lam - 1);
        }
        gamma += s->Lk[k];
        lam += n;
    }
    return minimal_state(s->nb, s->Q, s->L, s->N);
}

static void free_dev(std::vector<void*>& a) {
    for (void* p : a) cudaFree(p);
    a.clear();
}

static int build(dq_sector* s) {
    const int L = s->L, Q = s->Q, N = s->N, nb = s->nb;
    // D_Q table
    int nmax_all = (Q - 1) * L;
    s->h.dq_ld = nmax_all + 1;
    s->h.Dq.assign((size_t)(L + 1) * s->h.dq_ld, 0);
    for (int l = 0; l <= L; ++l)
        for (int m = 0; m <= nmax_all; ++m) s->h.Dq[(size_t)l * s->h.dq_ld + m] = dq_eq_dim(l, Q, m);
    uint64_t D = Dq(s, L, N);
    if (D == kSat || D >= (1ull << 63)) return set_error(DQ_ERANGE, "sector dimension >= 2^63");
    s->D = D;

    DevSector& v = s->dev;
    std::memset(&v, 0, sizeof v);
    std::memset(v.sub_of, -1, sizeof v.sub_of);
    v.L = L; v.Q = Q; v.N = N; v.nb = nb; v.n_sub = s->n_sub; v.D = D;
    // partition bookkeeping and distinct table lengths
    int ntab = 0;
    int tab_len[kMaxTables] = {0, 0};
    int pos = 0;
    for (int k = 0; k < s->n_sub; ++k) {
        s->start[k] = pos;
        pos += s->Lk[k];
        v.Lk[k] = s->Lk[k];
        v.shift[k] = nb * (L - pos);
        for (int b = v.shift[k]; b < v.shift[k] + nb * s->Lk[k] && b < 64; ++b) v.sub_of[b] = (signed char)k;
        v.nmax[k] = (Q - 1) * s->Lk[k];
        int t = -1;
        for (int q = 0; q < ntab; ++q)
            if (tab_len[q] == s->Lk[k]) t = q;
        if (t < 0) {
            if (ntab == kMaxTables) return set_error(DQ_EINVAL, "more than two distinct subsystem lengths");
            t = ntab;
            tab_len[ntab++] = s->Lk[k];
        }
        v.tab[k] = t;
        if (nb * s->Lk[k] > kMaxTabBits)
            return set_error(DQ_ERANGE, "subsystem of %d sites needs a table wider than %d bits; use more subsystems",
                             s->Lk[k], kMaxTabBits);
    }
    // Eq. (offset) and Eq. (stride); Gamma_k = sites after P_k
    int total = 0;
    for (int k = 0; k < s->n_sub; ++k) {
        v.os_base[k] = total;
        v.os_ld[k] = v.nmax[k] + 2;
        total += (N + 1) * v.os_ld[k];
    }
    v.os_total = total;
    s->h.off.assign(total, 0);
    s->h.str.assign(total, 0);
    for (int k = 0; k < s->n_sub; ++k) {
        int gamma = L - (s->start[k] + s->Lk[k]);
        for (int lam = 0; lam <= N; ++lam) {
            long rest = (long)N - lam;
            long nlow = rest - (long)(Q - 1) * gamma;
            if (nlow < 0) nlow = 0;
            unsigned __int128 acc = 0;
            for (int n = 0; n <= v.nmax[k] + 1; ++n) {
                size_t o = (size_t)v.os_base[k] + (size_t)lam * v.os_ld[k] + n;
                s->h.off[o] = (uint64_t)acc;  // sum over m in [nlow, n-1]
                if (n <= v.nmax[k]) {
                    s->h.str[o] = Dq(s, gamma, rest - n);
                    if (n >= nlow) acc += (unsigned __int128)Dq(s, s->Lk[k], n) * Dq(s, gamma, rest - n);
                }
            }
        }
    }
    // local tables per distinct length, filled by the on-the-fly rank (Alg. 1, Eq. (N=L))
    for (int t = 0; t < ntab; ++t) {
        int len = tab_len[t];
        int bits = nb * len;
        v.tab_bits[t] = bits;
        v.tab_len[t] = len;
        size_t npat = (size_t)1 << bits;
        auto& rt = s->h.rank_tab[t];
        auto& ut = s->h.unrank_tab[t];
        auto& ss = s->h.sec_start[t];
        rt.assign(npat, 0xffffffffu);
        int nmax = (Q - 1) * len;
        ss.assign(nmax + 2, 0);
        for (int n = 0; n <= nmax; ++n) ss[n + 1] = ss[n] + (uint32_t)Dq(s, len, n);
        ut.assign(ss[nmax + 1], 0);
        for (size_t p = 0; p < npat; ++p) {
            bool ok = true;
            int n = 0;
            for (int i = 0; i < len; ++i) {
                int d = (int)((p >> (nb * (len - 1 - i))) & ((1u << nb) - 1));
                if (d >= Q) ok = false;
                n += d;
            }
            if (!ok) continue;
            uint64_t li = 0;
            int lam = 0;
            for (int i = 0; i < len; ++i) {
                int d = (int)((p >> (nb * (len - 1 - i))) & ((1u << nb) - 1));
                for (int q = 0; q < d; ++q) li += Dq(s, len - 1 - i, (long)n - lam - q);
                lam += d;
            }
            rt[p] = (uint32_t)li;
            ut[ss[n] + li] = (uint32_t)p;
        }
    }
    // Lin's two-table form (Sec. 3.3): c_0 = offset_0(n_0) + stride_0(n_0) index_0 per pattern
    if (s->n_sub == 2) {
        size_t npat = (size_t)1 << (nb * s->Lk[0]);
        s->h.c0_tab.assign(npat, kSat);
        for (size_t p = 0; p < npat; ++p) {
            uint32_t li = s->h.rank_tab[v.tab[0]][p];
            if (li == 0xffffffffu) continue;
            int n = pattern_n(nb, (uint32_t)p, s->Lk[0]);
            size_t o = (size_t)v.os_base[0] + n;  // lambda_0 = 0
            if (N - n < 0 || N - n > v.nmax[1]) continue;  // P_1 cannot complete it
            s->h.c0_tab[p] = s->h.off[o] + s->h.str[o] * li;
        }
    }
    return DQ_OK;
}

// Copy the tables to the current device (done at creation when a CUDA device is present).
static int upload(dq_sector* s) {
    DevSector& v = s->dev;
    const int total = v.os_total;
    int ntab = (v.tab_len[1] != 0) ? 2 : 1;
    int rc;
    void* p;
    if ((rc = dev_upload(s->dev_allocs, s->h.off.data(), total * 8, &p))) return rc;
    v.off = (const uint64_t*)p;
    if ((rc = dev_upload(s->dev_allocs, s->h.str.data(), total * 8, &p))) return rc;
    v.str = (const uint64_t*)p;
    for (int t = 0; t < ntab; ++t) {
        if ((rc = dev_upload(s->dev_allocs, s->h.rank_tab[t].data(), s->h.rank_tab[t].size() * 4, &p))) return rc;
        v.rank_tab[t] = (const uint32_t*)p;
        if ((rc = dev_upload(s->dev_allocs, s->h.unrank_tab[t].data(), s->h.unrank_tab[t].size() * 4, &p))) return rc;
        v.unrank_tab[t] = (const uint32_t*)p;
        if ((rc = dev_upload(s->dev_allocs, s->h.sec_start[t].data(), s->h.sec_start[t].size() * 4, &p))) return rc;
        v.sec_start[t] = (const uint32_t*)p;
    }
    if (s->n_sub == 2) {
        if ((rc = dev_upload(s->dev_allocs, s->h.c0_tab.data(), s->h.c0_tab.size() * 8, &p))) return rc;
        v.c0_tab = (const uint64_t*)p;
    }
    int zero = 0;
    if ((rc = dev_upload(s->dev_allocs, &zero, sizeof zero, &p))) return rc;
    v.err = (int*)p;
    return DQ_OK;
}

}  // namespace dq

using namespace dq;

extern "C" {

const char* dq_last_error(void) { return dq::g_err.c_str(); }

int dq_make_sector(int L, int Q, int N, int n_sub, dq_sector** out) {
    clear_error();
    if (!out) return set_error(DQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (Q < 2 || Q > 16) return set_error(DQ_EINVAL, "Q must be in [2, 16]");
    int nb = 0;
    while ((1 << nb) < Q) ++nb;
    if (L < 1 || L * nb > 128) return set_error(DQ_EINVAL, "need 1 <= L and L * Nbits <= 128");
    if (N < 0 || N > (Q - 1) * L) return set_error(DQ_EINVAL, "need 0 <= N <= (Q-1) L");
    if (n_sub < 0 || n_sub > L) return set_error(DQ_EINVAL, "need 0 <= n_sub <= L");
    if (n_sub == 0) n_sub = (nb * L + 15) / 16;  // Eq. (Nopt_from_L)
    if (n_sub < 1) n_sub = 1;
    if (n_sub > kMaxSub) return set_error(DQ_EINVAL, "at most %d subsystems", kMaxSub);
    dq_sector* s = new (std::nothrow) dq_sector();
    if (!s) return set_error(DQ_ENOMEM, "host allocation");
    s->L = L; s->Q = Q; s->N = N; s->nb = nb; s->n_sub = n_sub;
    s->wide = L * nb > 64;
    int base = L / n_sub, extra = L % n_sub;  // most-equal, longer parts first (Sec. 4.3)
    for (int k = 0; k < n_sub; ++k) s->Lk[k] = base + (k < extra ? 1 : 0);
    s->device = 0;
    if (device_present()) cudaGetDevice(&s->device);
    int rc;
    try {
        rc = build(s);
    } catch (...) {
        rc = set_error(DQ_ENOMEM, "host allocation failed while building tables");
    }
    s->has_device = device_present();
    if (!rc && s->has_device) rc = upload(s);
    if (rc) {
        free_dev(s->dev_allocs);
        delete s;
        return rc;
    }
    *out = s;
    return DQ_OK;
}

void dq_free_sector(dq_sector* s) {
    if (!s) return;
    if (s->grad_ws) cudaFree(s->grad_ws);
    free_dev(s->dev_allocs);
    delete s;
}

int dq_sector_dim(const dq_sector* s, uint64_t* D) {
    clear_error();
    if (!s || !D) return set_error(DQ_EINVAL, "NULL argument");
    *D = s->D;
    return DQ_OK;
}

int dq_sector_partition(const dq_sector* s, int* n_sub, int* L_k) {
    clear_error();
    if (!s || !n_sub) return set_error(DQ_EINVAL, "NULL argument");
    *n_sub = s->n_sub;
    if (L_k)
        for (int k = 0; k < s->n_sub; ++k) L_k[k] = s->Lk[k];
    return DQ_OK;
}

static int narrow_only(const dq_sector* s, const char* fn) {
    if (s->wide)
        return set_error(DQ_EINVAL, "%s: the sector's states are %d bits wide; use the two-word form %s2", fn,
                         s->L * s->nb, fn);
    return DQ_OK;
}

int dq_state_at(const dq_sector* s, uint64_t index, uint64_t* state) {
    clear_error();
    if (!s || !state) return set_error(DQ_EINVAL, "NULL argument");
    if (int rc = narrow_only(s, "dq_state_at")) return rc;
    if (index >= s->D) return set_error(DQ_EINDEX, "index %llu >= D = %llu", (unsigned long long)index,
                                        (unsigned long long)s->D);
    *state = (uint64_t)host_unrank(s, index);
    return DQ_OK;
}

int dq_index_of(const dq_sector* s, uint64_t state, uint64_t* index) {
    clear_error();
    if (!s || !index) return set_error(DQ_EINVAL, "NULL argument");
    if (int rc = narrow_only(s, "dq_index_of")) return rc;
    if (!host_valid_state(s, state)) return set_error(DQ_ESTATE, "word 0x%llx is not a state of the sector",
                                                      (unsigned long long)state);
    *index = host_rank(s, state);
    return DQ_OK;
}

int dq_next_state(const dq_sector* s, uint64_t state, uint64_t* next) {
    clear_error();
    if (!s || !next) return set_error(DQ_EINVAL, "NULL argument");
    if (int rc = narrow_only(s, "dq_next_state")) return rc;
    if (!host_valid_state(s, state)) return set_error(DQ_ESTATE, "word 0x%llx is not a state of the sector",
                                                      (unsigned long long)state);
    *next = (uint64_t)host_increment(s, state);
    return DQ_OK;
}

static inline u128 from_words(const uint64_t* w) { return ((u128)w[1] << 64) | (u128)w[0]; }
static inline void to_words(u128 v, uint64_t* w) {
    w[0] = (uint64_t)v;
    w[1] = (uint64_t)(v >> 64);
}

int dq_state_at2(const dq_sector* s, uint64_t index, uint64_t* state) {
    clear_error();
    if (!s || !state) return set_error(DQ_EINVAL, "NULL argument");
    if (index >= s->D) return set_error(DQ_EINDEX, "index %llu >= D = %llu", (unsigned long long)index,
                                        (unsigned long long)s->D);
    to_words(host_unrank(s, index), state);
    return DQ_OK;
}

int dq_index_of2(const dq_sector* s, const uint64_t* state, uint64_t* index) {
    clear_error();
    if (!s || !state || !index) return set_error(DQ_EINVAL, "NULL argument");
    const u128 w = from_words(state);
    if (!host_valid_state(s, w))
        return set_error(DQ_ESTATE, "word 0x%016llx%016llx is not a state of the sector", (unsigned long long)state[1],
                         (unsigned long long)state[0]);
    *index = host_rank(s, w);
    return DQ_OK;
}

int dq_next_state2(const dq_sector* s, const uint64_t* state, uint64_t* next) {
    clear_error();
    if (!s || !state || !next) return set_error(DQ_EINVAL, "NULL argument");
    const u128 w = from_words(state);
    if (!host_valid_state(s, w))
        return set_error(DQ_ESTATE, "word 0x%016llx%016llx is not a state of the sector", (unsigned long long)state[1],
                         (unsigned long long)state[0]);
    to_words(host_increment(s, w), next);
    return DQ_OK;
}

int dq_state_at_batch(const dq_sector* s, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream) {
    clear_error();
    if (!s || (n && (!d_index || !d_state))) return set_error(DQ_EINVAL, "NULL argument");
    if (int rc = narrow_only(s, "dq_state_at_batch")) return rc;
    if (n == 0) return DQ_OK;
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    int e = launch_state_at_batch(s->dev, d_index, d_state, n, stream);
    if (e) return set_error(DQ_ECUDA, "state_at_batch launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}

int dq_index_of_batch(const dq_sector* s, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream) {
    clear_error();
    if (!s || (n && (!d_index || !d_state))) return set_error(DQ_EINVAL, "NULL argument");
    if (int rc = narrow_only(s, "dq_index_of_batch")) return rc;
    if (n == 0) return DQ_OK;
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    int e = launch_index_of_batch(s->dev, d_state, d_index, n, stream);
    if (e) return set_error(DQ_ECUDA, "index_of_batch launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}

int dq_state_at_batch2(const dq_sector* s, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream) {
    clear_error();
    if (!s || (n && (!d_index || !d_state))) return set_error(DQ_EINVAL, "NULL argument");
    if (n == 0) return DQ_OK;
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    int e = launch_state_at_batch_w(s->dev, d_index, d_state, n, stream);
    if (e) return set_error(DQ_ECUDA, "state_at_batch2 launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}

int dq_index_of_batch2(const dq_sector* s, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream) {
    clear_error();
    if (!s || (n && (!d_index || !d_state))) return set_error(DQ_EINVAL, "NULL argument");
    if (n == 0) return DQ_OK;
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    int e = launch_index_of_batch_w(s->dev, d_state, d_index, n, stream);
    if (e) return set_error(DQ_ECUDA, "index_of_batch2 launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}

int dq_check_device(const dq_sector* s, void* stream) {
    clear_error();
    if (!s) return set_error(DQ_EINVAL, "NULL argument");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->dev.err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "dq_check_device: %s", cudaGetErrorString(e));
    if (h) {
        int zero = 0;
        cudaMemcpy(s->dev.err, &zero, sizeof zero, cudaMemcpyHostToDevice);
        return set_error(DQ_EDEVICE, "a kernel flagged %d invalid input element(s)", h);
    }
    return DQ_OK;
}

}  // extern "C"
