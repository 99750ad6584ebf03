/*
 * dq.h -- C-ABI of the GB300 library for one particle-number (U(1)) sector of a lattice
 * Hamiltonian: divide-and-conquer basis ranking and the matrix-free product y = H x.
 *
 * Source of the method: Schaefer and Luitz, "DanceQ: High-performance library for
 * number-conserving bases", arXiv:2407.14591.
 *   - the problem and the three basis functions (i) get_index, (ii) increment, (iii) get_state:
 *     Sec. 2.1 and Sec. 2.2;
 *   - the canonical order, Eq. (index), Eq. (ck), Eq. (lambda), Eq. (offset), Eq. (stride):
 *     Sec. 3.1 and Sec. 3.2; the two limits (Lin's two tables, on-the-fly): Sec. 3.3;
 *   - the sector dimension D_Q(L, n), Eq. (dim) and App. A;
 *   - the matrix-free product and Lanczos: Sec. 2.1, Sec. 4.4 and App. D.
 *
 * Conventions shared by every call:
 *   - L sites, local dimension Q (2 <= Q <= 16), Nbits = ceil(log2 Q) bits per site, N particles
 *     (the paper's n). A basis state is an integer word in which site i occupies bits
 *     [Nbits*(L-1-i), Nbits*(L-i)), i.e. site 0 is the most significant digit (Sec. 4.2).
 *     L * Nbits <= 128. With L * Nbits <= 64 a state is one uint64 and every function applies;
 *     wider states (Sec. 4.1: the state class holds as many words as the sites need) take two
 *     uint64 words, low word first (bits 0..63, then 64..127), and are read and written only by
 *     the two-word forms (dq_state_at2, dq_index_of2, dq_next_state2, dq_state_at_batch2,
 *     dq_index_of_batch2), which serve every sector.
 *   - The lattice is split into n_sub consecutive subsystems of most-equal length, the first
 *     (L mod n_sub) being one site longer (Sec. 4.3). n_sub = 0 selects the paper's default
 *     ceil(Nbits * L / 16) (Eq. (Nopt_from_L)).
 *   - The canonical order is that of Sec. 3.2: the last subsystem varies fastest; inside a
 *     subsystem, states are ordered by their own particle number and then lexicographically
 *     with the subsystem's first site most significant (Table 1).
 *   - Every call returns DQ_OK (0) or a negative status; dq_last_error() then describes the
 *     failure (thread-local). No C++ exception crosses this boundary.
 *   - Pointers named d_* and the x / y / v0 vectors are DEVICE pointers owned by the caller, on
 *     the device that was current when the sector was made. Host pointers are named plainly.
 *   - A `stream` argument is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that take a stream are asynchronous with respect to the host unless stated.
 */
#ifndef DQ_H
#define DQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define DQ_OK 0
#define DQ_EINVAL (-1)   /* an argument is out of its documented range                    */
#define DQ_ERANGE (-2)   /* the sector is too large (D >= 2^63, or a table would not fit)  */
#define DQ_EINDEX (-3)   /* an index >= D                                                  */
#define DQ_ESTATE (-4)   /* a word that is not a state of the sector                       */
#define DQ_ENOMEM (-5)   /* a host or device allocation failed                             */
#define DQ_ECUDA (-6)    /* a CUDA runtime call failed                                     */
#define DQ_EDEVICE (-7)  /* a kernel flagged bad input through the sector's error word     */

/* ---- vector element types ------------------------------------------------------------- */
#define DQ_F64 0 /* vectors stored as double                                         */
#define DQ_F32 1 /* vectors stored as float; accumulation is exact (fixed point)      */

/* Flag OR'ed into dq_lanczos' reorth argument: double-single arithmetic for the passes over the
 * Lanczos basis (see dq_lanczos). */
#define DQ_LZ_DOUBLE_SINGLE 16

/* ---- operator term kinds (all Hermitian, real) -------------------------------------------- */
/* Spin-1/2 (Q = 2 only; a particle is an up spin, Sz = sigma - 1/2; App. D's Hamiltonian):  */
#define DQ_XY 0  /* coef * 1/2 (S+_i S-_j + S-_i S+_j)                                        */
#define DQ_ZZ 1  /* coef * Sz_i Sz_j                                                         */
#define DQ_Z 2   /* coef * Sz_i                     (j ignored)                              */
/* Bosons, any Q (occupation n = digit, truncated at Q-1):                                   */
#define DQ_HOP 3 /* -coef * (b+_i b_j + b+_j b_i)                                            */
#define DQ_NN 4  /* coef * n_i n_j                                                           */
#define DQ_N 5   /* coef * n_i                      (j ignored)                              */
#define DQ_U 6   /* coef / 2 * n_i (n_i - 1)        (j ignored)                              */

typedef struct dq_sector dq_sector; /* opaque: partition, tables on host and device          */
typedef struct dq_terms dq_terms;   /* opaque: compiled operator for one sector               */

typedef struct dq_term {
    int kind;    /* DQ_XY .. DQ_U                                     */
    int i, j;    /* sites; j ignored by single-site kinds; i != j     */
    double coef; /* real coefficient                                  */
} dq_term;

/* Description of the last failure on the calling thread ("" if none). Never NULL. */
const char* dq_last_error(void);

/* ---- sector ------------------------------------------------------------------------------ */

/* Build the sector (L, Q, N) split into n_sub subsystems: the D_Q table (Eq. (dim)), the
 * offset and stride tables (Eq. (offset), Eq. (stride)), one local rank table and one local
 * unrank list per distinct subsystem length (Sec. 4.2, container (i); filled with the
 * on-the-fly rank of Alg. 1), and their device copies on the current device.
 * Arguments: 1 <= L, L*Nbits <= 128, 2 <= Q <= 16, 0 <= N <= (Q-1)L, 0 <= n_sub <= L and
 * n_sub <= 64.
 * Errors: DQ_EINVAL for out-of-range arguments; DQ_ERANGE if D >= 2^63 or a subsystem is wider
 * than 24 bits; DQ_ENOMEM / DQ_ECUDA on allocation failure. *out is set only on success and is
 * owned by the caller (dq_free_sector). Synchronous. */
int dq_make_sector(int L, int Q, int N, int n_sub, dq_sector** out);

/* Release a sector and its device tables. NULL is allowed. Terms made for it must be freed
 * first. */
void dq_free_sector(dq_sector* s);

/* Sector dimension D = D_Q(L, N) (Eq. (dim)). */
int dq_sector_dim(const dq_sector* s, uint64_t* D);

/* Partition: *n_sub and L_k[0 .. n_sub-1] (caller provides room for 64 ints). */
int dq_sector_partition(const dq_sector* s, int* n_sub, int* L_k);

/* Function (iii), get_state (Sec. 2.2, Alg. 4), on the host: the state with canonical index
 * `index`. DQ_EINDEX if index >= D; DQ_EINVAL if the sector's states are wider than 64 bits
 * (use dq_state_at2). */
int dq_state_at(const dq_sector* s, uint64_t index, uint64_t* state);

/* Function (i), get_index (Sec. 2.2, Alg. 2, Eq. (index)), on the host. DQ_ESTATE if `state`
 * has bits above L*Nbits, a digit >= Q, or a particle number other than N. DQ_EINVAL if the
 * sector's states are wider than 64 bits (use dq_index_of2). */
int dq_index_of(const dq_sector* s, uint64_t state, uint64_t* index);

/* Function (ii), increment (Sec. 2.2, Alg. 3), on the host: the next state in canonical order;
 * the last state wraps to the first (minimal) one. DQ_ESTATE for an invalid `state`, DQ_EINVAL
 * for a sector of states wider than 64 bits (use dq_next_state2). */
int dq_next_state(const dq_sector* s, uint64_t state, uint64_t* next);

/* Two-word forms of functions (iii), (i) and (ii) (same algorithms), for every sector: a state is
 * the host array state[2] = {bits 0..63, bits 64..127}. Errors as the one-word forms. */
int dq_state_at2(const dq_sector* s, uint64_t index, uint64_t* state);
int dq_index_of2(const dq_sector* s, const uint64_t* state, uint64_t* index);
int dq_next_state2(const dq_sector* s, const uint64_t* state, uint64_t* next);

/* Batched function (iii) on the device: d_state[t] = get_state(d_index[t]) for t < n.
 * An index >= D writes UINT64_MAX and sets the sector's error word (see dq_check_device).
 * DQ_EINVAL for a sector of states wider than 64 bits (use dq_state_at_batch2).
 * Asynchronous on `stream`. */
int dq_state_at_batch(const dq_sector* s, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream);

/* Batched function (i) on the device: d_index[t] = get_index(d_state[t]) for t < n.
 * An invalid state writes UINT64_MAX and sets the error word. DQ_EINVAL for a sector of states
 * wider than 64 bits (use dq_index_of_batch2). Asynchronous on `stream`. */
int dq_index_of_batch(const dq_sector* s, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream);

/* Two-word forms of the batches, for every sector: d_state holds 2 n uint64, state t at
 * [2t, 2t+1] (low word first). An index >= D writes two UINT64_MAX words, an invalid state the
 * index UINT64_MAX, and both raise the error word. Asynchronous on `stream`. */
int dq_state_at_batch2(const dq_sector* s, const uint64_t* d_index, uint64_t* d_state, uint64_t n, void* stream);
int dq_index_of_batch2(const dq_sector* s, const uint64_t* d_state, uint64_t* d_index, uint64_t n, void* stream);

/* Synchronise `stream`, read and clear the sector's device error word. Returns DQ_EDEVICE if a
 * kernel flagged bad input since the last check, DQ_OK otherwise. */
int dq_check_device(const dq_sector* s, void* stream);

/* ---- operator ---------------------------------------------------------------------------- */

/* Compile `n_terms` terms for sector `s` and upload them. Errors: DQ_EINVAL for an unknown kind,
 * a site out of range, i == j in a pair term, or a spin-1/2 kind with Q != 2. The same
 * (i, j) pair may appear in several terms; their contributions add. Q = 2 sectors of one-word
 * states take the bond-layer form (pairs grouped by bit distance); other Q, and every sector of
 * two-word states, take the per-term form (site functions, n_i n_j pairs, hops; the spin-1/2
 * kinds rewritten as Sz = n - 1/2 and S+_i S-_j = b+_i b_j). *out is owned by the caller
 * (dq_free_terms). Synchronous. */
int dq_make_terms(const dq_sector* s, const dq_term* terms, int n_terms, dq_terms** out);

/* Which product kernel dq_matvec uses for these terms with one right-hand side: *path = 1 for the
 * panel kernel (Q = 2, uniform single-site fields, at most two distinct hop amplitudes and four
 * distinct Sz Sz coefficients, dyadic coefficients; either two subsystems with P_1 of at most 15
 * sites and P_0 of at most 16, or three or more subsystems whose last one has fewer than 8 or more
 * than 10 sites, with P_1 = the last two subsystems, at most 15 sites, and the others at most 22
 * sites in all), 0 for the general kernels (any Q, partition and nrhs). Both sum exactly in fixed
 * point (see dq_matvec) and compute the same y up to the rounding of the coefficients to their
 * integer grid, which is exact on the panel path. *path = 3 for the per-bond panel kernel, taken
 * when the panel kernel's conditions on the coefficients fail but the structure fits (Q = 2, two
 * subsystems, P_1 of at most 13 sites and P_0 of at most 16, at most 64 bonds inside P_1, 64 across
 * the cut and 200 inside P_0, any coefficient per bond and per site). Terms made by
 * dq_make_cluster_terms report 2 (the cluster-merged kernel). *path = 4 for the warp-panel kernel:
 * the panel kernel's conditions on the coefficients with two to eight subsystems, the last one of
 * 8 to 10 sites and the others of at most 24 sites in all (panels of at most 252 rows, one warp
 * each; with two subsystems this replaces the panel kernel for such small panels). *path = 5 for
 * the boson panel kernel: Q > 2, two subsystems, one-word states, P_1 of at most 14 bits
 * (Nbits * L_1 <= 14) and P_0 of at most 24, no n_i n_j pair terms, D < 2^40, at most 31 hop
 * bonds and 4096 hop amplitude entries (bonds x Q x Q), 64 P_0 and cut hops per panel; any
 * coefficient per hop bond and any site function (the per-term form's integer coefficients, so
 * it gives the general kernel's y). */
int dq_terms_path(const dq_terms* t, int* path);

/* Compile terms in the cluster-merged form of App. C instead: the terms are grouped into clusters
 * of at most `cluster_sites` sites (clusters may overlap; each term goes to the first cluster that
 * holds its sites or can take them, in the order of the terms sorted by their sites), and all the
 * terms of one cluster are merged into one sparse matrix over the cluster's digit patterns
 * (Nbits * cluster_sites <= 12 bits, i.e. at most 4096 patterns), stored column by column: each
 * entry holds the XOR mask that moves a word between the two patterns and the merged coefficient
 * (one integer grid for all, as in dq_matvec). dq_matvec then applies one column per cluster and
 * row (any Q, one- or two-word states, 1..64 right-hand sides, both dtypes in exact fixed point
 * with 57-bit x), and dq_terms_path reports 2. Results equal those of dq_make_terms up to the
 * rounding of the merged coefficients to the grid. Errors: as dq_make_terms; DQ_EINVAL for
 * cluster_sites out of [2, 12] or Nbits * cluster_sites > 12, or more than 64 clusters.
 * Synchronous; *out is owned by the caller (dq_free_terms). */
int dq_make_cluster_terms(const dq_sector* s, const dq_term* terms, int n_terms, int cluster_sites, dq_terms** out);

/* Clusters of terms made by dq_make_cluster_terms: their number, the sites of each (host array
 * of 12 ints per cluster, -1 after the last site; may be NULL) and the largest number of matrix
 * entries one row can meet (may be NULL). DQ_EINVAL for terms in another form. */
int dq_cluster_info(const dq_terms* t, int* n_clusters, int* sites, int* entries);

/* Release compiled terms. NULL is allowed. */
void dq_free_terms(dq_terms* t);

/* y = H x for `nrhs` right-hand sides (Sec. 2.1, Sec. 4.4): x and y are device arrays of
 * D * nrhs elements of `dtype` (DQ_F64 or DQ_F32), row-major with the nrhs values of basis
 * state i contiguous at [i*nrhs, (i+1)*nrhs). y is overwritten; x and y must not overlap.
 * 1 <= nrhs <= 64. Every y[i] is written exactly once by one thread (gather form), so there
 * are no atomics and the result is deterministic. Asynchronous on `stream`.
 * FP64 vectors are summed exactly in fixed point: each column of x is scaled by a power of two
 * and rounded to a 57-bit integer, the coefficients share one power-of-two grid (at least 55
 * significant bits relative to the largest, fewer by log2 of a row's diagonal term count when
 * that exceeds 128), and each y[i] is a 128-bit integer sum rounded once. FP32 vectors take the
 * same route with 31-bit integers for x, hop amplitudes with 24 significant bits (int64 hop
 * sums) and the diagonal on a finer grid. An Inf or NaN in x makes y NaN and raises the sector's
 * error word (DQ_EDEVICE from dq_check_device). The call keeps a scratch area of
 * D * nrhs * 8 bytes (FP64) or 4 bytes (FP32) with the terms, allocated on first use (so make one
 * call before capturing calls into a CUDA graph); calls with the same terms that overlap on the
 * GPU (two streams at once) race on it, so order them on one stream or use separate terms.
 * Errors: DQ_EINVAL (NULL pointers, bad dtype or nrhs, terms of another sector). */
int dq_matvec(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, int nrhs, void* stream);

/* y = H x like dq_matvec with one right-hand side, but without allocating any device memory.
 * The paper has no counterpart; this entry point exists for callers that cannot call cudaMalloc
 * while they run: for example a solver that has handed all device memory to its own pool up
 * front, or a time-critical loop in which an allocation (which can synchronise the device) is
 * not allowed. dq_matvec, by contrast, allocates its scratch on first use and keeps it with the
 * terms.
 * The scratch (a fixed-point copy of x and a small header) lives in a static device array of
 * 64 MiB that every GPU loading this library reserves until the process exits. Hence the limit:
 * D <= 8,388,568 for DQ_F64 and D <= 16,777,144 for DQ_F32 (8,388,568 for both on the boson panel
 * path, which keeps x as 64-bit words); larger sectors return DQ_ERANGE with the limit in
 * dq_last_error(). Only terms on the panel paths (dq_terms_path 1, 4 or 5) are served; others
 * return DQ_EINVAL. The first call on a device does a one-time set-up: it looks up the
 * array's device address (cudaGetSymbolAddress) and caches it. With CUDA's default lazy module
 * loading, that lookup is also when the runtime loads the code module holding the array, so the
 * 64 MiB are taken from the device at that first call, not when the library is loaded: make the
 * first call on each device before handing the device's memory to a pool of your own, and
 * before any stream capture. Later calls allocate nothing. Every
 * call reuses the same array, and each call clears the header part it needs to start at zero;
 * calls that overlap on the GPU (for example on two streams at once) race on the array and give
 * wrong results, so order them on one stream or synchronise between them. x and y: device
 * arrays of D elements of `dtype`, must not overlap. Asynchronous on `stream`; non-finite x is
 * reported by dq_check_device as DQ_EDEVICE. */
int dq_matvec_noalloc(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype, void* stream);

/* ---- differentiation ---------------------------------------------------------------------- */

/* Coefficient gradients of the product (the adjoint of y = H x with H = sum_q coef_q T_q): for
 * the given list of terms (only kind, i, j are used; coef is ignored) and a cotangent dy,
 *   d_grads[q] = sum_i sum_r dy[i, r] (T_q x)[i, r],
 * T_q being term q with coefficient 1 (the operators of DQ_XY .. DQ_U). With a complex vector
 * stored as nrhs = 2 real columns this is Re <dy, T_q x>. The gradient with respect to x is
 * H dy (every term is real and Hermitian), i.e. another dq_matvec. x, dy: device arrays laid out
 * as in dq_matvec; d_grads: device array of n_terms doubles. For Q = 2 the products dy * x are
 * exact fixed-point values (x and dy scaled per column to int64, each product rounded once to a
 * common grid with 48 bits below the largest possible product) summed in int64; other Q multiply
 * in FP64. Each block's sums are reduced in FP64 in a fixed order (deterministic). An Inf or NaN
 * in x or dy (Q = 2) gives NaN gradients and raises the sector's error word. The workspace
 * (2 * D * nrhs * 8 bytes for Q = 2, plus a few KB) is kept with the sector, grown on demand and
 * freed by dq_free_sector; calls on one sector from several host threads at once race on it.
 * Synchronous. Errors as dq_make_terms, plus DQ_EINVAL for bad dtype or nrhs or a sector of
 * two-word states, DQ_ENOMEM. The paper's operator class (Sec. 4.1) has no derivatives; this
 * serves training-style use of the product. */
int dq_term_grads(const dq_sector* s, const dq_term* terms, int n_terms, const void* x, const void* dy, int dtype,
                  int nrhs, double* d_grads, void* stream);

/* ---- batched product ------------------------------------------------------------------- */

typedef struct dq_batch dq_batch; /* opaque: up to 64 (sector, terms) pairs for one launch      */

/* Plan one launch over n (1..64) Q = 2 sectors of uneven dimension (different L, N, disorder),
 * each with nrhs (1..8) right-hand sides stored as in dq_matvec, of `dtype`. The sectors and
 * terms must outlive the batch. Uploads the n descriptors (synchronous). FP64 vectors accumulate
 * in FP64 (the batched product is bound by its gathers of x, so the fixed-point prepass of
 * dq_matvec would only add traffic); FP32 vectors form products in FP32 and sum them with
 * compensated (Neumaier) summation. Errors: DQ_EINVAL (n, nrhs, dtype out of range; terms of
 * another sector; Q != 2 or two-word states), DQ_ENOMEM, DQ_ECUDA. *out is owned by the caller
 * (dq_batch_free). */
int dq_batch_make(int n, const dq_sector* const* sectors, const dq_terms* const* terms, int nrhs, int dtype,
                  dq_batch** out);

/* y_k = H_k x_k for every k in one persistent kernel launch (Sec. 2.2's workers over consecutive
 * rows, here over row tiles of all sectors). x and y: host arrays of n device pointers, each to
 * D_k * nrhs elements; x_k and y_k must not overlap. Asynchronous on `stream`; the launch
 * contains no allocation or host synchronisation, so it can be recorded in a CUDA graph. */
int dq_batch_matvec(dq_batch* b, const void* const* x, void* const* y, void* stream);

/* Autotuner: time every candidate (row mapping, threads per CTA, CTAs per SM, rows per tile) on
 * the given vectors (one warm-up and three timed launches each, CUDA events on `stream`), keep
 * the fastest for later dq_batch_matvec calls and return its number in *choice (may be NULL).
 * The mappings: the CTA's threads take a tile's rows with a block stride and unrank each with
 * Alg. 4, or each warp takes 32 R consecutive rows and each lane steps from row to row through
 * the last subsystem's unrank list. Tiles are pulled from an atomic queue in both. Overwrites y.
 * Synchronous. */
int dq_batch_tune(dq_batch* b, const void* const* x, void* const* y, void* stream, int* choice);

/* Select candidate `shape` (0 .. *n_shapes - 1) for later dq_batch_matvec calls instead of the
 * tuned one; a negative shape only reports the number of candidates in *n_shapes (may be NULL).
 * Errors: DQ_EINVAL. */
int dq_batch_shape(dq_batch* b, int shape, int* n_shapes);

/* Release a batch plan. NULL is allowed. */
void dq_batch_free(dq_batch* b);

/* Ground-state energy by Lanczos (Sec. 4.4, App. D): starting from v0 (device, D elements of
 * `dtype`, normalised inside the call, not modified), run up to `steps` steps of
 *   w = H v_k; alpha_k = <v_k, w>; w -= alpha_k v_k + beta_{k-1} v_{k-1};
 *   reorth == 1: full re-orthogonalisation by classical Gram-Schmidt against v_0 .. v_k,
 *                w -= V (V^T w), repeated once more when that pass shrank ||w|| below 1/sqrt(2)
 *                of its value before the pass (the Daniel-Gragg-Kaufman-Stewart criterion);
 *   reorth == 2: the same with the second pass always;
 *   reorth == 0: neither (the plain three-term recurrence);
 *   beta_k = ||w||; v_{k+1} = w / beta_k.
 * With reorth != 0 the three-term step is done on the fly inside the first Gram-Schmidt pass,
 * whose coefficient for v_k is added to alpha_k. Dot products, norms, the recurrence and the
 * vector updates are computed in FP64 whatever `dtype` is; the basis is stored in `dtype`.
 * reorth | DQ_LZ_DOUBLE_SINGLE selects double-single arithmetic for every pass over the basis
 * instead (pairs of floats with error-free products and sums, about 48 significant bits; block
 * partials combined in FP64; the basis of DQ_F64 vectors stored as float pairs): several times
 * faster on a GPU whose FP64 rate is a small fraction of its FP32 rate, at an accuracy close to
 * FP64 (the recurrence coefficients and the tridiagonal solve stay FP64); pair elements below
 * 2^-74 in magnitude keep 24 significant bits and below 2^-126 become zero, so the form suits
 * operators whose coefficients are well above that scale. E0 is the smallest
 * eigenvalue of the tridiagonal matrix T, found on the host by bisection on its Sturm sequence. The call stops early, without error,
 * when beta_k < 1e-12 * ||T||; *steps_done then holds the number of steps taken m. alpha and
 * beta (host, room for `steps` doubles each, may be NULL) receive the recurrence coefficients.
 * psi (device, D elements of `dtype`, may be NULL) receives the Ritz vector of E0,
 * sum_k y_k v_k with y the unit eigenvector of T for E0 (inverse iteration on T, sign chosen so
 * that its largest component is positive); ||H psi - E0 psi|| is the residual of E0.
 * The workspace ((steps+1) basis vectors of 8 (DQ_F64) or 4 (DQ_F32) bytes per element, three
 * more vectors, scratch, 16 bytes of pinned host memory per step) is allocated and freed by the
 * call, and the product's own scratch is kept with the terms (see dq_matvec). The steps run on `stream` without waiting for the host: the call reads each
 * step's coefficients two steps later, so after a breakdown up to two more steps may have run;
 * their results are dropped. Synchronous: returns when E0 (and psi) are known. Errors: DQ_EINVAL
 * (NULL or out-of-range arguments, steps outside [1, 4096], reorth outside [0, 2] (apart from
 * the flag), a zero or
 * non-finite v0), DQ_ENOMEM, DQ_ECUDA (also for a non-finite coefficient). */
int dq_lanczos(const dq_sector* s, const dq_terms* t, const void* v0, int steps, int dtype, int reorth,
               double* E0, double* alpha, double* beta, int* steps_done, void* psi, void* stream);

/* ---- kernel timing ------------------------------------------------------------------------ */

/* Measurement hooks; the paper has no counterpart. While timing is on, every dq_matvec,
 * dq_matvec_noalloc, dq_batch_matvec and dq_term_grads call records a pair of CUDA events on its
 * own stream around its main kernel (the panel kernel, the general product kernel, the batched
 * kernel or the term-gradient kernels) and counts the kernels the call launched (the panel path
 * launches three: two prepass kernels and the panel kernel). Calls made while the stream is being captured into a CUDA graph are neither
 * timed nor counted. dq_timing_enable(1) turns timing on and clears the record;
 * dq_timing_enable(0) turns it off and keeps the record. dq_timing_read waits for the recorded
 * events and returns (each pointer may be NULL) the summed main-kernel time in milliseconds, the
 * number of product calls counted and the number of kernels they launched. At most 65536 calls
 * are timed after a reset; later ones are counted but not timed, and dq_timing_read then returns
 * DQ_ERANGE along with the partial sums. Thread-safe. Errors: DQ_ECUDA. */
int dq_timing_enable(int on);
int dq_timing_read(double* ms, long long* launches, long long* kernels);

#ifdef __cplusplus
}
#endif

#endif /* DQ_H */
