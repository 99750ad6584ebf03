// Internal definitions shared by the host builder (dq_sector.cpp, dq_terms.cpp) and the CUDA
// kernels (dq_kernels.cu, dq_lanczos.cu). Not part of the public ABI (include/dq.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dq.h"

namespace dq {

constexpr int kMaxSub = 64;      // at most one subsystem per site (L * Nbits <= 64)
constexpr int kMaxTables = 2;    // most-equal partitions have at most two distinct lengths
constexpr int kMaxLayers = 64;   // bond layers of the Q = 2 operator form (>= the 63 distances of 64 sites)
constexpr int kMaxTabBits = 24;  // widest subsystem pattern that gets a rank table

// Plain-old-data view of a sector, passed by value to kernels. Device pointers only.
struct DevSector {
    int L, Q, N, nb, n_sub;
    uint64_t D;
    int Lk[kMaxSub];       // subsystem lengths
    int shift[kMaxSub];    // bit position of the least significant bit of P_k's field
    signed char sub_of[64];  // subsystem holding bit position p (-1 above L * Nbits)
    int tab[kMaxSub];      // which local table P_k uses
    int nmax[kMaxSub];     // (Q-1) * L_k
    int os_base[kMaxSub];  // start of P_k's block in off / str: [lam 0..N][n 0..nmax_k+1]
    int os_ld[kMaxSub];    // nmax_k + 2
    int os_total;          // entries in off / str
    const uint64_t* off;   // Eq. (offset), entry n = nmax_k + 1 holds the block total
    const uint64_t* str;   // Eq. (stride)
    int tab_bits[kMaxTables];     // Nbits * length of each table's subsystems
    int tab_len[kMaxTables];      // length (sites)
    const uint32_t* rank_tab[kMaxTables];    // local index of every pattern (0xffffffff: digit >= Q)
    const uint32_t* unrank_tab[kMaxTables];  // patterns grouped by particle number, local order
    const uint32_t* sec_start[kMaxTables];   // start of particle number n inside unrank_tab
    const uint64_t* c0_tab;  // n_sub == 2 only: c_0 of every P_0 pattern (Sec. 3.3, Lin's table)
    int* err;                // device error word
};

// Q = 2 operator in "bond layer" form: a layer groups the bonds (p, p + dist) between bit
// positions, so [sigma_p != sigma_{p+dist}] for all of them is one shift and one xor.
struct DevTermsQ2 {
    double C;                  // constant part of the diagonal
    const double* lin;         // per bit position: coefficient of sigma_p (NULL if folded into C)
    int nl;                    // number of layers
    int dist[kMaxLayers];
    uint64_t dmask[kMaxLayers];  // low positions p with a diagonal coefficient
    uint64_t omask[kMaxLayers];  // low positions p with an off-diagonal amplitude
    const double* KA;            // [2 * kMaxLayers] device array: uniform coefficient K of
                                 // [sigma_p != sigma_{p+dist}] at l, uniform hop amplitude A at
                                 // kMaxLayers + l
    int kpos[kMaxLayers];        // -1: uniform K; else offset of 64 per-position values in pos
    int apos[kMaxLayers];        // -1: uniform A; else offset in pos
    const double* pos;           // per-position coefficients
    // FP32 copies of the coefficients, used when the vectors are FP32 (device arrays, so that
    // the structure stays small enough to be passed by value: kernel parameters <= 4 KB)
    float Cf;
    const float* KAf;  // [2 * kMaxLayers]: K of layer l at l, A of layer l at kMaxLayers + l
    const float* linf;
    const float* posf;
    // Fixed-point copies used when the vectors are FP64: every coefficient c is M 2^emin with
    // an integer M (|M| < 2^55 or less, see compile_q2); the same layout as KA, lin and pos
    int emin;
    long long MC;
    const long long* MKA;
    const long long* Mlin;  // NULL when lin is
    const long long* Mpos;
    // Fixed-point copies used when the vectors are FP32: hop amplitudes c = m 2^emin32 with
    // |m| < 2^24 (int32); diagonal coefficients on their own finer grid c = m 2^emin32d (int64),
    // 0 <= emin32 - emin32d <= 60
    int emin32, emin32d;
    long long MC32;
    const long long* MKA32;  // K of layer l (grid emin32d) at l, A (grid emin32) at kMaxLayers + l
    const long long* Mlin32;
    const long long* Mpos32;  // per-position K (grid emin32d) and A (grid emin32) values
};
static_assert(sizeof(DevSector) + sizeof(DevTermsQ2) + 64 <= 4096, "product kernel parameters exceed 4 KB");

// General-Q operator (bosons): per-site digit functions, density-density pairs, hops.
struct DevTermsQG {
    int nsite;           // sites with a nonzero digit function f_i(d)
    const int* site_sh;  // bit shift of each such site's digit
    int npair;
    const int* pair_sh;  // [npair][2] shifts of the n_i n_j pairs
    int nhop;
    const int* hop_sh;   // [nhop][2] shifts (a, b): term -t (b+_a b_b + b+_b b_a)
    // Coefficients as integers on one grid, for FP64 vectors: c = M 2^emin
    int emin;
    long long MC;
    const long long* Msite;  // [nsite][Q]: f_i(d)
    const long long* Mpair;  // [npair]: coefficient of d_i d_j
    const long long* Mhop;   // [nhop][Q][Q]: -t sqrt((n_a + 1) n_b), zero where the hop is not allowed
    // The same for FP32 vectors: hop amplitudes m 2^emin32 with |m| < 2^24 (int32), diagonal
    // coefficients on their own finer grid 2^emin32d (int64), 0 <= emin32 - emin32d <= 60
    int emin32, emin32d;
    long long MC32;
    const long long* Msite32;
    const long long* Mpair32;
    const int* Mhop32;
};

// Plan of the panel product (Q = 2, two subsystems, Sec. 3.3): with index = c_0(s0) + index_1(s1),
// the states sharing one P_0 pattern s0 form a contiguous "panel" of D_2(L_1, N - n_0) rows.
// Hops inside P_1 stay inside a panel, hops inside P_0 map a panel onto another panel of the same
// length element by element, and hops across the cut map a panel onto a panel of the
// neighbouring particle-number block. All coefficients are integer multiples of 2^emin.
constexpr int kPanelMaxBonds = 64;
constexpr int kPanelMaxLayers = 16;
constexpr int kPanelMaxGroups = 16;
constexpr int kPanelMaxA = 2;  // distinct hop amplitudes
constexpr int kPanelMaxK = 4;  // distinct [s_i != s_j] coefficients
constexpr int kPanelMaxList = kPanelMaxBonds + kPanelMaxGroups;
// Per-panel values shared by all rows of the panel: counts of [s_i != s_j] over the Sz Sz bonds
// inside P_0 per coefficient class, and the bit-plane counters (3 bits per position b of P_1) of
// the Sz Sz bonds across the cut, for s_a = 0 (w0: counts b occupied) and s_a = 1 (w1: b empty).
struct PanelDiag {
    int cnt0[kPanelMaxK];
    uint32_t w0[kPanelMaxK][3], w1[kPanelMaxK][3];
};

struct PanelPlan {
    int L0, L1, N;
    uint32_t npanels;
    const uint32_t* panel_s0;     // P_0 pattern of every panel, canonical order
    const uint64_t* panel_start;  // first global index of every panel
    const uint64_t* c0;           // c_0 of every P_0 pattern (UINT64_MAX: no panel)
    const uint16_t* t1rank;       // local index of every P_1 pattern
    const uint16_t* t1states;     // P_1 patterns grouped by particle number
    uint32_t t1start[18], t1len[18];
    // off-diagonal, each list sorted by amplitude class; *_end[k] = end of class k
    int p0_end[kPanelMaxA];       // P_0-internal pairs (two-bit mask in s0)
    uint32_t p0_mask[kPanelMaxBonds];
    int n_p1l;                    // P_1-internal pairs grouped in layers of equal distance d
    int p1l_d[kPanelMaxLayers], p1l_first[kPanelMaxLayers], p1l_cut[kPanelMaxLayers], p1l_end[kPanelMaxLayers];
    uint32_t p1b_lobit[kPanelMaxBonds];  // bit of the pair's lower position
    uint32_t p1b_pm2[kPanelMaxBonds];    // pair mask shifted left by one (byte offset into the rank table)
    int n_xg;                     // crossing groups: one per site a of P_0
    uint32_t xg_abit[kPanelMaxGroups];
    int xg_first[kPanelMaxGroups], xg_cut[kPanelMaxGroups], xg_end[kPanelMaxGroups];  // class 0 in [first, cut)
    uint32_t xb_bit[kPanelMaxBonds];  // bit of site b in s1
    // diagonal counts of [s_i != s_j], each list sorted by K class
    int p0z_end[kPanelMaxK];
    uint32_t p0z_mask[kPanelMaxBonds];
    int p1z_end[kPanelMaxK];
    int p1z_d[kPanelMaxLayers];
    uint32_t p1z_mask[kPanelMaxLayers];
    int xz_end[kPanelMaxK];
    uint32_t xz_abit[kPanelMaxBonds], xz_bbit[kPanelMaxBonds];
    int nA, nK;
    long long MC, MK[kPanelMaxK], MA[kPanelMaxA];  // coefficients / 2^emin
    int emin;
    int cmax;  // longest panel
    // per-panel source lists (built on the host): panel p owns entries [list_off[p], list_off[p+1])
    // = its active P_0 partners (first list_cnt0[p] of class 0, then class 1) and then its valid
    // crossing partners. Entry: global start index | (crossing group << 48).
    const uint32_t* list_off;
    const uint32_t* list_hdr;   // bits 0-7: class-0 P_0 partners, 8-15: class-1, 16-23: crossing
    const uint64_t* list;
    const PanelDiag* diag;      // per panel, built on the host (two subsystems)
    // three or more subsystems (the warp-panel kernel): prefix bits of the Sz Sz bonds across the
    // cut, per class and per position b of P_1 (the per-panel counters are built on the device)
    uint32_t xzA[kPanelMaxK][32];
};

// What the warp-panel kernel needs of the sector to rank a prefix pattern on the device: Eq.
// (index) over the subsystems above the last one (at most kPWMaxSub subsystems in all).
constexpr int kPWMaxSub = 8;
struct PWRank {
    int n_sub, N, L1, os_total;
    int shift[kPWMaxSub], os_base[kPWMaxSub], os_ld[kPWMaxSub];
    uint32_t fmask[kPWMaxSub];           // mask of P_k's field after the shift
    const uint32_t* rank[kPWMaxSub];     // local index of every pattern of P_k
    const uint64_t* off;                 // Eq. (offset) and Eq. (stride), os_total entries each
    const uint64_t* str;
    uint64_t D;
};

// Cluster-merged operator (App. C): every term lies in one cluster of at most kClMaxSites sites,
// and the terms of a cluster are merged into one sparse matrix S_c over the cluster's digit
// patterns (pattern p = sum_k digit(site_k) << (Nbits k)), stored by columns: column p lists the
// entries (XOR mask that turns a word with cluster pattern p into one with pattern p', and the
// coefficient S_c[p', p] as an integer M with S = M 2^emin). The diagonal entry has mask 0.
constexpr int kClMaxSites = 12;  // and Nbits * sites <= 12 (at most 4096 patterns per cluster)
constexpr int kClMax = 64;
struct DevTermsCL {
    int ncl;
    int emin;
    const int* nsite;        // [ncl]
    const int* sh;           // [ncl][kClMaxSites]: bit shift of the digit of cluster site k
    const int* col_base;     // [ncl]: start of cluster c's column offsets in col_off
    const uint32_t* col_off; // per cluster 2^(Nbits nsite) + 1 offsets into the entry arrays
    const uint64_t* dlo;     // entry mask, bits 0..63
    const uint64_t* dhi;     // entry mask, bits 64..127 (two-word states)
    const long long* M;      // entry coefficient / 2^emin
};

// Plan of the per-bond panel product (Q = 2, two subsystems, P_1 of at most 13 sites): the
// structural rank of the panel product (rows sharing a P_0 pattern form one panel) with a
// coefficient per bond and per site, rounded to one integer grid 2^emin. Bit positions: P_1 holds
// bits 0 .. L1-1 of the word, P_0 the bits above (s0 = word >> L1).
constexpr int kPBMaxL1 = 13;
constexpr int kPBMaxBonds = 64;
constexpr int kPBMaxGroups = 16;
struct PanelPB {
    int L0, L1, N, emin, cmax;
    uint32_t npanels;
    const uint32_t* panel_s0;     // P_0 pattern of every panel, canonical order
    const uint64_t* panel_start;  // first index of every panel
    const uint16_t* t1rank;       // local index of every P_1 pattern
    const uint16_t* t1states;     // P_1 patterns grouped by particle number
    uint32_t t1start[kPBMaxL1 + 2], t1len[kPBMaxL1 + 2];
    // bonds inside P_1: pair mask (bits lo, hi), hop amplitude and Sz Sz coefficient (device)
    int n1b;
    uint32_t p1_lo[kPBMaxBonds], p1_hi[kPBMaxBonds];
    const long long* p1_A;        // [n1b]
    const long long* p1_K;        // [n1b]
    // bonds across the cut, grouped by the P_0 bit a (partner panel s0 ^ a): P_1 bit b and
    // coefficients; groups with a hop amplitude only (the Sz Sz parts are in xz_*)
    int nxg;
    uint32_t xg_abit[kPBMaxGroups];
    int xg_first[kPBMaxGroups], xg_end[kPBMaxGroups];
    uint32_t xb_bit[kPBMaxBonds];
    const long long* xb_A;        // [bonds]
    int nxz;                       // Sz Sz bonds across the cut: [s_a != s_b] with coefficient K
    uint32_t xz_abit[kPBMaxBonds], xz_bbit[kPBMaxBonds];
    const long long* xz_K;
    const long long* f1;          // [L1]: field of P_1 bit b (coefficient of s_b)
    const long long* pdiag;       // per panel: constant + P_0 fields + P_0 Sz Sz bonds
    const long long* p0_A;        // hop amplitude of each P_0 bond (index in the partner entry)
    // per-panel sources: P_0 partners (start | bond << 48) then cross partners (start | group << 48)
    const uint32_t* list_off;
    const uint32_t* list_hdr;     // bits 0-7: P_0 partners, 8-15: cross partners
    const uint64_t* list;
};

// Plan of the boson panel product (Q > 2, two subsystems; dq_panel_q.cu): the panels of the
// canonical order (rows sharing one P_0 pattern s0, contiguous by Lin's two tables, Sec. 3.3).
// Everything that depends only on the row's P_1 pattern is tabulated once per pattern and read
// by every panel of its particle-number block: the P_1 site functions, the hops inside P_1 (the
// partner's local index and the amplitude entry, padded to one length per block with a zero
// amplitude), and the local index of the partner row for every hop direction across the cut.
constexpr int kPQMaxBits = 14;  // nb * L_1: at most 16384 P_1 patterns
constexpr int kPQMaxN = 32;     // particle numbers of P_1 (plus one)
constexpr int kPQMaxCut = 255;  // hop directions across the cut
constexpr int kPQMaxList = 64;  // P_0 and cut entries of one panel
struct PanelQ {
    int Q, nb, L1, N, emin, nM, ncut;
    uint32_t npanels;
    const uint32_t* panel_s0;     // P_0 pattern of every panel, longest panels first
    const uint64_t* panel_start;  // first index of every panel
    uint32_t t1start[kPQMaxN + 1], t1len[kPQMaxN + 1];  // P_1 patterns per particle number
    const long long* Mhop;        // [bonds][Q][Q]: -t sqrt((n_up + 1) n_dn) on the grid 2^emin; entry nM is 0
    // per P_1 pattern (index t1start[n1] + local index c):
    const long long* rdiag;       // the P_1 site functions
    const uint32_t* p1ell;        // from p1base[n1], p1m[n1] slots of C entries: partner | Mhop entry << 16
    uint32_t p1base[kPQMaxN + 1], p1m[kPQMaxN + 1];
    const uint32_t* cutt;         // from cutbase[n1], ncut slots of C entries: partner local index |
                                  // row part of the Mhop entry << 16 | (the hop is not allowed) << 31
    uint32_t cutbase[kPQMaxN + 1];
    const long long* pdiag;       // per panel: the constant plus the P_0 site functions
    // per-panel sources: P_0 partners (start | Mhop entry << 40), then cut partners
    // (start | cut direction << 40 | panel part of the Mhop entry << 48)
    const uint32_t* list_off;
    const uint32_t* list_hdr;     // bits 0-7: P_0 entries, 8-15: cut entries
    const uint64_t* list;
};

// Host-side tables kept by a sector.
struct HostTables {
    std::vector<uint64_t> Dq;  // (L+1) x (nmax_total+1), saturated at UINT64_MAX
    int dq_ld = 0;
    std::vector<uint64_t> off, str;
    std::vector<uint32_t> rank_tab[kMaxTables], unrank_tab[kMaxTables], sec_start[kMaxTables];
    std::vector<uint64_t> c0_tab;
};

}  // namespace dq

struct dq_sector {
    int L, Q, N, nb, n_sub;
    bool wide;  // L * Nbits > 64: states take two words (the 128-bit forms of every function)
    uint64_t D;
    int Lk[dq::kMaxSub], start[dq::kMaxSub];
    dq::HostTables h;
    dq::DevSector dev;  // device view (pointers into device allocations below)
    std::vector<void*> dev_allocs;
    int device;
    bool has_device;  // tables were uploaded (a CUDA device was present at creation)
    void* grad_ws = nullptr;  // workspace of dq_term_grads, grown on demand, freed with the sector
    size_t grad_ws_bytes = 0;
};

struct dq_terms {
    const dq_sector* sector;
    bool q2;
    dq::DevTermsQ2 q2v;
    dq::DevTermsQG qgv;
    std::vector<void*> dev_allocs;
    int max_hops;  // upper bound on off-diagonal elements per row
    bool panel_ok = false;     // the panel product applies (see PanelPlan)
    bool pb_ok = false;        // the per-bond panel product applies (PanelPB)
    bool pw_ok = false;        // the warp-panel product applies (three or more subsystems, PanelPlan)
    bool pq_ok = false;        // the boson panel product applies (Q > 2, PanelQ)
    dq::PanelQ pqp;
    dq::PanelPB pbp;
    bool cluster = false;      // cluster-merged form (App. C), dq_make_cluster_terms
    dq::DevTermsCL clv;
    std::vector<int> cl_sites; // host copy: the sites of each cluster, -1 after the last
    dq::PanelPlan pp;
    dq::PWRank pwr;            // the warp-panel product's view of the sector
    void* scratch = nullptr;   // fixed-point copy of x and the exponent word, grown on demand
    size_t scratch_bytes = 0;
};

namespace dq {

// error reporting (thread-local message)
int set_error(int code, const char* fmt, ...);
void clear_error();

// host-side rank / unrank used by the ABI functions, on 128-bit words (a one-word state is the
// low word)
using u128 = unsigned __int128;
bool host_valid_state(const dq_sector* s, u128 w);
uint64_t host_rank(const dq_sector* s, u128 w);
u128 host_unrank(const dq_sector* s, uint64_t idx);

// kernel launchers (dq_kernels.cu); return a cudaError_t as int
int launch_state_at_batch(const DevSector& S, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream);
int launch_index_of_batch(const DevSector& S, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream);
int launch_matvec(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream);
// the same batches for states stored as two uint64 words (low word first)
int launch_state_at_batch_w(const DevSector& S, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream);
int launch_index_of_batch_w(const DevSector& S, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream);

// per-bond panel product (dq_panel_pb.cu): plan from the Q = 2 pair list (bit lo, distance) ->
// (K of [s_lo != s_hi], hop amplitude A), per-position fields and the constant
int build_panel_pb(const dq_sector* s, double C, const double* lin,
                   const std::vector<std::pair<std::pair<int, int>, std::pair<double, double>>>& pairs, dq_terms* t);
int launch_panel_pb(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream);

// validation shared by the term compilers (dq_terms.cpp): DQ_OK or the error status
int check_terms(const dq_sector* s, const dq_term* terms, int n_terms);
// cluster-merged product (dq_cluster.cu)
int launch_cluster_matvec(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream);

// panel product (dq_panel.cpp / dq_panel.cu)
int build_panel_plan(const dq_sector* s, double C, bool uniform_lin,
                     const std::vector<std::pair<std::pair<int, int>, std::pair<double, double>>>& pairs, dq_terms* t);
int launch_panel_matvec(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream);
int launch_panel_w(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream);
// boson panel product (dq_panel_q.cu): the plan from the compiled per-term coefficients (site
// shifts and their [site][Q] functions, hop shifts and the [hop][Q][Q] amplitudes, all on the grid
// 2^emin), and the launch
int build_panel_q(const dq_sector* s, const std::vector<int>& site_sh, const std::vector<long long>& msite,
                  const std::vector<int>& hop_sh, const std::vector<long long>& mhop, long long MC, int emin,
                  int npair, dq_terms* t);
int launch_panel_q(const dq_sector* s, dq_terms* t, const void* x, void* y, int dtype, void* stream);
// the same with caller-provided scratch of panel_scratch_bytes(s, DQ_F64) bytes (both dtypes)
int launch_panel_q_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* ws,
                      void* stream);
int launch_panel_w_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* ws,
                      void* stream);
size_t panel_scratch_bytes(const dq_sector* s, int dtype);
int launch_panel_matvec_ws(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* scratch,
                           void* stream);

// kernel timing (dq_timing.cpp): timing_start records the start event of a main kernel on `st`
// and returns its slot (-1: timing off or stream capturing); timing_stop records the stop event
// and counts the call's `kernels` launches
int timing_start(cudaStream_t st);
void timing_stop(int slot, cudaStream_t st, int kernels);

// device memory helpers; without a CUDA device dev_upload returns DQ_OK and a NULL pointer
bool device_present();
// SM count of the current device, cached per device index (thread-safe)
int sm_count_cached();
// resident blocks per SM of `kernel` with `threads` threads and `smem` bytes of dynamic shared
// memory on the current device, from the occupancy calculator, cached per (kernel, threads,
// smem, device); at least 1
int occupancy_cached(const void* kernel, int threads, size_t smem);
int dev_upload(std::vector<void*>& allocs, const void* host, size_t bytes, void** dptr);

}  // namespace dq
