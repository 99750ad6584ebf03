// Internal definitions shared by the host builder (dq_sector.cpp, dq_terms.cpp) and the CUDA
// kernels (dq_kernels.cu, dq_lanczos.cu). Not part of the public ABI (include/dq.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dq.h"

namespace dq {

constexpr int kMaxSub = 64;      // at most one subsystem per site (L * Nbits <= 64)
constexpr int kMaxTables = 2;    // most-equal partitions have at most two distinct lengths
constexpr int kMaxLayers = 48;   // bond layers of the Q = 2 operator form
constexpr int kMaxTabBits = 24;  // widest subsystem pattern that gets a rank table

// Plain-old-data view of a sector, passed by value to kernels. Device pointers only.
struct DevSector {
    int L, Q, N, nb, n_sub;
    uint64_t D;
    int Lk[kMaxSub];       // subsystem lengths
    int shift[kMaxSub];    // bit position of the least significant bit of P_k's field
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
    double K[kMaxLayers];        // uniform coefficient of [sigma_p != sigma_{p+dist}]
    double A[kMaxLayers];        // uniform hop amplitude
    int kpos[kMaxLayers];        // -1: uniform K; else offset of 64 per-position values in pos
    int apos[kMaxLayers];        // -1: uniform A; else offset in pos
    const double* pos;           // per-position coefficients
};

// General-Q operator (bosons): per-site digit functions, density-density pairs, hops.
struct DevTermsQG {
    double C;
    int nsite;           // sites with a nonzero digit function
    const int* site_sh;  // bit shift of each such site's digit
    const double* site_f;  // [nsite][Q] values f_i(d)
    int npair;
    const int* pair_sh;    // [npair][2] shifts
    const double* pair_K;  // coefficient of d_i d_j
    int nhop;
    const int* hop_sh;     // [nhop][2] shifts (a, b): term -t (b+_a b_b + b+_b b_a)
    const double* hop_t;
    const double* amp;     // [Q][Q]: sqrt((n_a + 1) n_b)
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
    uint64_t D;
    int Lk[dq::kMaxSub], start[dq::kMaxSub];
    dq::HostTables h;
    dq::DevSector dev;  // device view (pointers into device allocations below)
    std::vector<void*> dev_allocs;
    int device;
    bool has_device;  // tables were uploaded (a CUDA device was present at creation)
};

struct dq_terms {
    const dq_sector* sector;
    bool q2;
    dq::DevTermsQ2 q2v;
    dq::DevTermsQG qgv;
    std::vector<void*> dev_allocs;
    int max_hops;  // upper bound on off-diagonal elements per row
};

namespace dq {

// error reporting (thread-local message)
int set_error(int code, const char* fmt, ...);
void clear_error();

// host-side rank / unrank used by the ABI functions
bool host_valid_state(const dq_sector* s, uint64_t w);
uint64_t host_rank(const dq_sector* s, uint64_t w);
uint64_t host_unrank(const dq_sector* s, uint64_t idx);

// kernel launchers (dq_kernels.cu); return a cudaError_t as int
int launch_state_at_batch(const DevSector& S, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream);
int launch_index_of_batch(const DevSector& S, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream);
int launch_matvec(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream);

// device memory helpers; without a CUDA device dev_upload returns DQ_OK and a NULL pointer
bool device_present();
int dev_upload(std::vector<void*>& allocs, const void* host, size_t bytes, void** dptr);

}  // namespace dq
