/*
 * libasci: GB300 (sm_103a) ASCI determinant search, C ABI.
 *
 * The library implements the search step of the Adaptive Sampling
 * Configuration Interaction method (arXiv:2303.05688, Sec. 2.2, Algorithm 2,
 * Eq. 1): from the core determinants of a wavefunction it enumerates every
 * single and double excitation, evaluates H_ij by the Slater-Condon rules,
 * accumulates the numerator sum_j H_ij c_j per unique target
 * (sort-and-accumulate), scores each target outside psi as
 * num / (E0 - H_ii) and keeps the N targets of largest |score|.  Around it,
 * the variational step (Sec. 2.3: the sparse Hamiltonian of a determinant
 * list, its product with vectors, the Davidson eigensolver) closes the ASCI
 * loop of Algorithm 1.
 *
 * Conventions shared by every entry point:
 *  - A determinant is a pair of occupation words; bit p of `alpha` (`beta`) is
 *    spatial orbital p of that spin.  The GPU path packs a determinant into one
 *    64-bit key, so it accepts norb <= 32.
 *  - The Hamiltonian is H = ecore + sum h_pq a+_ps a_qs
 *    + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs with real integrals, h1 symmetric
 *    (row-major norb x norb) and eri in chemists' order, 8-fold symmetric,
 *    eri[((p*norb+q)*norb+r)*norb+s] = (pq|rs).
 *  - |D> = prod_{p in alpha asc} a+_{p,alpha} prod_{q in beta asc} a+_{q,beta}|0>;
 *    a single p->q on one spin carries (-1)^(occupied orbitals of that spin
 *    strictly between p and q); a same-spin double i<j -> a<b is i->a then j->b.
 *  - 128-bit key order: beta word high, alpha word low.
 *  - Pointers may be host or device memory (detected per pointer) unless an
 *    entry point says "device".  The caller owns every buffer; the library
 *    allocates its scratch on `cuda_stream` (stream-ordered) and frees it
 *    before returning.  `cuda_stream` may be NULL (the legacy default stream).
 *  - Every entry point returns ASCI_OK or a negative error code; no exception
 *    crosses the boundary.  On error the outputs are unspecified and any
 *    `*out_n` is set to 0.  Calls are synchronous with respect to the host:
 *    they return after their results are in the output buffers.
 */
#ifndef ASCI_H
#define ASCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASCI_OK 0
#define ASCI_EINVAL (-1)   /* invalid argument or input data */
#define ASCI_ENOMEM (-2)   /* device memory exhausted or a batch cannot fit */
#define ASCI_ECUDA (-3)    /* a CUDA runtime call failed */
#define ASCI_ETIMEOUT (-4) /* a bounded wait or an iteration limit ran out (Davidson) */

/* One determinant: occupation words of the alpha and beta spin strings. */
typedef struct {
  uint64_t alpha;
  uint64_t beta;
} asci_det;

/* One- and two-electron integrals (see conventions above). */
typedef struct {
  int32_t norb;      /* 1..32 */
  double ecore;      /* constant added to every diagonal element */
  const double *h1;  /* norb*norb */
  const double *eri; /* norb^4 */
} asci_ints;

/* Arithmetic of the per-pair values H_ij c_j (not in the paper; a variant of
 * its method).  The numerator sums, the diagonal, E0 and the denominator
 * E0 - H_ii are the same in every mode (exact fixed-point or order-independent
 * rules, FP64 results). */
enum {
  ASCI_FP64 = 0,              /* FP64 integrals and products */
  ASCI_FP32_INT_FP64_ACC = 1, /* two-electron elements from FP32 tables, FP64 products */
  ASCI_FP32_INT_COMP_ACC = 2  /* two-electron elements from FP32 tables, FP32 products */
};

typedef struct {
  /* Alg. 2 screen: keep the pair (target, core) only if |H_ij c_j / (E0 - H_ii)|
   * > eps_search.  0 keeps every generated pair (the default; the paper's runs
   * use 1e-10, Sec. 3). */
  double eps_search;
  /* Deepest constraint level (number of fixed highest occupied alpha orbitals,
   * Sec. 2.2) the batch planner may refine to; 0 means no limit (n_alpha). */
  int32_t max_constraint_level;
  int32_t precision;         /* ASCI_FP64 | ASCI_FP32_INT_FP64_ACC | ASCI_FP32_INT_COMP_ACC */
  uint64_t max_batch_pairs;  /* pairs per constraint batch; 0 = sized from free memory */
  int32_t sort_output;       /* 1: outputs sorted by key ascending; 0: unspecified order */
  /* Constraint sharding across processes (Sec. 2.2, Alg. 3): with
   * shard_count > 1 the search covers only the target alpha classes of shard
   * shard_index (0-based) and returns that shard's top N; the classes partition
   * the targets, so the top N of the union of every shard's output is the
   * unsharded result.  Classes heavier than 1/(64 shard_count) of the pairs are
   * placed by asci_shard_assign (Alg. 3's greedy), the others by a hash of their
   * alpha string.  0 or 1: no sharding. */
  int32_t shard_index;
  int32_t shard_count;
  /* CTAs per SM of the persistent generation and on-chip accumulation
   * kernels (a launch shape, not in the paper): 0 = as many as fit.  Fewer
   * leave room on the GPU for other searches running at the same time (many
   * small independent searches, asci_search_many); results do not depend on
   * it. */
  int32_t ctas_per_sm;
} asci_opts;

/* Counters and per-stage device times (milliseconds) of one search. */
typedef struct {
  uint64_t generated;  /* C * n_exc pairs enumerated */
  uint64_t surviving;  /* pairs kept by the eps screen */
  uint64_t unique;     /* unique targets after sort-and-accumulate */
  uint64_t excluded;   /* unique targets dropped because they are in psi */
  uint64_t selected;   /* *out_n */
  uint64_t batches;    /* constraint batches run */
  uint64_t max_batch;  /* pairs in the largest batch */
  uint64_t ncore;      /* core determinants used (min(C, ndets)) */
  uint64_t max_level;  /* deepest constraint level the planner used */
  uint64_t tile_launches;      /* launches of the on-chip tile kernel */
  uint64_t tile_records;       /* staged pairs reduced on chip (16 bytes read each) */
  uint64_t oversized_records;  /* staged pairs of hash buckets overfilled by hot
                                  targets: reduced by the larger tile kernels
                                  (up to 2048 or 4096 records a bucket) or, in
                                  a bigger bucket, by a global sort */
  /* The diagonal H_ii is summed exactly in 64-bit fixed point on the grid
   * 2^-diag_grid_bits: E0, ecore and each integral term of H_ii (h_pp, J - K of
   * a same-spin pair, J of an opposite-spin pair) is rounded once to the grid,
   * so E0 - H_ii carries at most (terms + 2) * 2^-(diag_grid_bits + 1) of
   * rounding before its one conversion to FP64. */
  uint64_t diag_grid_bits;
  uint64_t big_tile_records;  /* of oversized_records, those reduced on chip */
  /* device milliseconds: prepare, plan, generate (emission into the staging
     buffer), tiles (the on-chip tile kernel alone), oversized (overfilled
     buckets alone: the large tile kernel and the global-sort path), score (tiles + oversized + exact scores + pruning), select,
     total */
  double t_stage[8];
} asci_stats;

/* Fill `opts` with the defaults (eps 0, no level cap, FP64, auto batch, unsorted). */
void asci_default_opts(asci_opts *opts);

/* Library version string and the compute capability it was built for. */
const char *asci_version(void);

/* Human-readable text of an error code. */
const char *asci_strerror(int code);

/* Detail of the last error raised on the calling thread ("" if none). */
const char *asci_last_error(void);

/* Number of kernels this library has launched in the process so far. */
unsigned long long asci_launch_count(void);

/* Scratch memory is cached per device between calls (a stream-ordered pool);
 * this returns the cached memory of the current device to the system. */
void asci_trim_cache(void);

/* Fault injection for tests of the error path (no counterpart in the paper):
 * after `after` more successful scratch allocations (in any thread), the next
 * one fails as if the device had no memory left, once; the call that makes it
 * returns ASCI_ENOMEM ("injected allocation failure" in asci_last_error())
 * after releasing its scratch, and later calls run normally.  A negative
 * value cancels a pending injection.  The allocation-free entry point
 * allocates nothing and is unaffected. */
void asci_debug_fail_allocation(int64_t after);

/*
 * The ASCI search (Algorithm 2 with Eq. 1; constraint batching of Sec. 2.2).
 *
 *  dets[ndets], coeffs[ndets]  the wavefunction psi (distinct determinants, all
 *                              with the same alpha and beta electron counts).
 *  E0                          the energy in the score's denominator E0 - H_ii.
 *  ints                        integrals (the struct itself is host memory; its
 *                              arrays may be host or device memory).
 *  C                           core size: the C determinants of largest |c|
 *                              (ties by key ascending); C > ndets is clamped.
 *  N                           number of targets to return.
 *  opts                        NULL for defaults.
 *  out_dets[N], out_scores[N]  the selected targets and their signed scores
 *                              S = num / (E0 - H_ii); *out_n = min(N, U) where
 *                              U is the number of unique targets outside psi.
 *                              Among equal |S| at the cutoff, smaller keys win.
 *  stats                       may be NULL.
 *
 * Errors: ASCI_EINVAL for norb outside 1..32, ndets == 0, C == 0, NULL
 * pointers, a determinant with bits at or above norb, mixed electron counts,
 * duplicate determinants, or non-finite E0 / coefficients / integrals;
 * ASCI_ENOMEM when scratch cannot be allocated; ASCI_ECUDA on CUDA failure.
 */
int asci_search(const asci_det *dets, const double *coeffs, size_t ndets, double E0,
                const asci_ints *ints, size_t C, size_t N, const asci_opts *opts,
                asci_det *out_dets, double *out_scores, size_t *out_n, asci_stats *stats,
                void *cuda_stream);

/*
 * ASCI-PT2 (the last step of Algorithm 1): the second-order energy of the
 * determinants outside psi,
 *     E_PT2 = sum_{i not in psi} (sum_{j in core} H_ij c_j)^2 / (E0 - H_ii),
 * with the core the C determinants of largest |c| (C >= ndets: the whole
 * wavefunction, the usual PT2).  It runs the search's generation, constraint
 * batching and on-chip accumulation (a2-a5) with no threshold, and sums the
 * terms of every unique target in an exact fixed-point accumulator (grid
 * 2^-216, terms truncated to it), so the value does not depend on batching or
 * scheduling.  eps_search in opts screens pairs as in the search (0: none).
 *
 * Errors: those of asci_search; ASCI_EINVAL also when a term is not finite or
 * exceeds 2^40 in magnitude (E0 equal or too close to a target's H_ii).
 */
int asci_pt2(const asci_det *dets, const double *coeffs, size_t ndets, double E0,
             const asci_ints *ints, size_t C, const asci_opts *opts, double *e_pt2,
             asci_stats *stats, void *cuda_stream);

/*
 * Generation stage of Algorithm 2 (the inner loops: "single and double
 * connections from D_j" and the partial quantity H_ij C_j), for testing the
 * excitation kernel in isolation.  For each core determinant, in input order,
 * writes its n_exc targets and values v = H_ij * c_j in the library's fixed
 * per-determinant order: alpha singles, beta singles, alpha-alpha doubles,
 * beta-beta doubles, alpha-beta doubles (holes and particles ascending).
 * All pointers are device memory; out_* hold capacity elements and
 * *out_n = ncore * n_exc (ASCI_EINVAL if that exceeds capacity).
 */
int asci_excitations(const asci_ints *ints, const asci_det *core, const double *coeffs,
                     size_t ncore, asci_det *out_targets, double *out_values, size_t capacity,
                     size_t *out_n, void *cuda_stream);

/*
 * Diagonal elements H_ii = <D_i|H|D_i> (the denominator of Eq. 1).  Device
 * pointers; dets[n] in, out_haa[n] out.
 */
int asci_diagonal(const asci_ints *ints, const asci_det *dets, size_t n, double *out_haa,
                  void *cuda_stream);

/*
 * Sort-and-accumulate (Sec. 2.2): sorts the (key, value) pairs on the key and
 * sums the values of each unique key.  Device pointers; out_keys / out_sums
 * hold n elements; *out_n receives the number of unique keys, written in key
 * order.  Equal keys are summed in input order.  Keys are packed into 64
 * bits, so each word must be below 2^32 (at most 32 orbitals); a key with a
 * higher bit returns ASCI_EINVAL.
 */
int asci_sort_accumulate(const asci_det *keys, const double *values, size_t n,
                         asci_det *out_keys, double *out_sums, size_t *out_n,
                         void *cuda_stream);

/*
 * Sort-and-accumulate that allocates nothing.  The paper has no counterpart;
 * this serves callers that cannot allocate device memory during the call: a
 * process whose device memory is already reserved by another allocator or
 * capped, or an embedder (a latency-bound or certified code path) whose policy
 * forbids allocation behind its back.
 *
 * Same results as asci_sort_accumulate (bit for bit) for
 * n <= ASCI_NOALLOC_MAX_PAIRS (ASCI_EINVAL above that, with a message in
 * asci_last_error(); also for a key word with bits at or above 32).  Every
 * scratch buffer is carved from one fixed device array inside the library
 * (about 104 bytes per pair of the maximum plus 2 MiB, ~7 MB).  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 *
 * The array belongs to the library's device code module: each context that
 * loads the module holds one copy until the process exits (or the context is
 * destroyed).  CUDA loads modules lazily by default, so the first call on a
 * device is the one that loads the module and commits the array: make one
 * call as a warm-up before the section that must not allocate, and before any
 * stream capture.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the calling thread's current device.
 *
 * All calls share the one array and it keeps the last call's contents, so
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Every return, an error included, comes
 * after the call's GPU work has finished (the stream is synchronised), so a
 * call that has returned no longer touches the array.  Inputs and outputs may
 * be host or device memory.
 */
#define ASCI_NOALLOC_MAX_PAIRS 65536
int asci_sort_accumulate_noalloc(const asci_det *keys, const double *values, size_t n,
                                 asci_det *out_keys, double *out_sums, size_t *out_n,
                                 void *cuda_stream);

/*
 * Building blocks of a top-N selection across ranks (the role of Alg. 4: the
 * global N largest |score| of candidates spread over processes, found without
 * gathering them).  The rank word of an entry is the 128-bit unsigned
 * R = (~bits(|score|), key), words {hi, lo}: ascending R is |score|
 * descending, then key ascending (keys distinct), so the global top N are the
 * entries with R <= R_N.  A caller finds R_N byte by byte from the most
 * significant end, summing the ranks' histograms (an all-reduce of 256
 * counters per byte), then keeps its entries at or below R_N.
 *
 * asci_select_histogram: hist[256] (host memory, out) counts the entries whose
 * R agrees with prefix on the bits set in mask, by the value of byte `digit`
 * of R (15: the most significant byte of hi ... 0: the least significant byte
 * of lo).  n may be 0 (a zero histogram).
 * asci_select_below: the entries with R <= threshold (out_* hold n entries;
 * order unspecified); *out_n receives their count.
 * Pointers may be host or device memory; prefix, mask and threshold are host
 * memory.  Errors: ASCI_EINVAL for NULL arrays with n > 0, NULL prefix, mask,
 * threshold, hist or out_n, digit outside 0..15, or n >= 2^32.
 */
int asci_select_histogram(const asci_det *keys, const double *scores, size_t n, int32_t digit,
                          const uint64_t prefix[2], const uint64_t mask[2], uint64_t hist[256],
                          void *cuda_stream);

/* The digit choice of that selection (host only; no GPU).  The state holds
 * the fixed bits of R_N (prefix, with mask marking them), the rank of R_N
 * among the entries that match them (remaining) and the next byte to fix
 * (digit, 15 down to 0).
 *
 * asci_select_begin: total = the number of entries over all ranks, N the
 * number to select.  With total <= N every entry is selected: done = 1 and
 * threshold = all ones.  Otherwise prefix = mask = 0, remaining = N, digit =
 * 15, done = 0.
 * asci_select_step: hist[256] = the sum over the ranks of
 * asci_select_histogram(.., digit, prefix, mask, ..).  Fixes byte `digit` of
 * R_N to the value whose bucket holds the remaining-th matching entry
 * (counting from the smallest byte value), lowers remaining by the entries of
 * the smaller values and sets threshold = prefix; when that bucket is taken
 * whole, threshold = prefix with every unfixed bit set and done = 1; after
 * byte 0, done = 1.  Callers keep, on every rank, the entries with
 * R <= threshold (asci_select_below): N in all.
 * Errors: ASCI_EINVAL for NULL arguments, a finished state, or a histogram
 * holding fewer than `remaining` entries (the message names it). */
typedef struct {
  uint64_t prefix[2];     /* fixed bits of R_N: {hi, lo} */
  uint64_t mask[2];       /* which bits of prefix are fixed */
  uint64_t threshold[2];  /* the bound to keep entries at or below, once done */
  uint64_t remaining;     /* rank of R_N among the entries matching prefix on mask */
  int32_t digit;          /* next byte to fix; -1 when done */
  int32_t done;
} asci_select_state;
int asci_select_begin(uint64_t total, uint64_t N, asci_select_state *st);
int asci_select_step(asci_select_state *st, const uint64_t hist[256]);
int asci_select_below(const asci_det *keys, const double *scores, size_t n,
                      const uint64_t threshold[2], asci_det *out_keys, double *out_scores,
                      size_t *out_n, void *cuda_stream);

/* One independent search of a batch (asci_search_many): the arguments of
 * asci_search, and its result code. */
typedef struct {
  const asci_det *dets;
  const double *coeffs;
  size_t ndets;
  double E0;
  const asci_ints *ints;
  size_t C, N;
  asci_det *out_dets;   /* capacity N */
  double *out_scores;   /* capacity N */
  size_t *out_n;
  asci_stats *stats;    /* nullable */
  int32_t status;       /* written: ASCI_OK or the search's error code */
} asci_problem;

/* Many independent searches (the paper's method applied to uneven small
 * systems, e.g. embedding fragments; not a step of Alg. 2): up to `streams`
 * of them run at a time, each on its own CUDA stream driven by its own host
 * thread, so that small searches overlap on the GPU.  Each problem is
 * exactly asci_search(problem..., opts) (bit-identical results); pointers
 * follow asci_search's rules.  Returns ASCI_OK when every problem succeeded,
 * else the first failing problem's code (asci_last_error() holds its message);
 * every problem's status is written.  streams < 1: ASCI_EINVAL. */
int asci_search_many(asci_problem *problems, size_t count, const asci_opts *opts,
                     int32_t streams);

/*
 * The constraint classes of one level and their work (Sec. 2.2: a class is
 * the set of targets whose alpha string has the same `level` highest occupied
 * orbitals; its work is the number of (target, core) pairs it receives, the
 * quantity Alg. 3 balances and Fig. 3 plots).  The core is the C
 * determinants of largest |c| as in asci_search; level is clamped to n_alpha.
 * out_pairs[i] (host or device, capacity entries) receives the pair count of
 * the i-th non-empty class in ascending order of its target alpha strings;
 * *out_n the number of non-empty classes (always written).  With capacity <
 * *out_n nothing else is written and the call returns ASCI_OK (a size query).
 * The counts add up to C n_exc.  Errors: those of asci_search's input checks,
 * and ASCI_EINVAL for level < 1.
 */
int asci_constraint_classes(const asci_det *dets, const double *coeffs, size_t ndets,
                            const asci_ints *ints, size_t C, int32_t level, uint64_t *out_pairs,
                            size_t capacity, size_t *out_n, void *cuda_stream);

/* Alg. 3's greedy placement (longest processing time first): the n classes
 * of weights[n] (pairs) are visited in descending weight (ties: lower index
 * first) and each goes to the shard with the smallest load so far (ties: lower
 * shard), loads starting from initial_loads[shards] (nullable: zeros).  Writes
 * shard_out[n] (values in [0, shards)).  Host memory only; runs on the host.
 * Returns ASCI_EINVAL for shards < 1 or null arrays with n > 0. */
int asci_shard_assign(const uint64_t *weights, size_t n, int32_t shards,
                      const uint64_t *initial_loads, int32_t *shard_out);

/*
 * Top-N selection by |score| (Sec. 2.2, the duplicate-aware selection that
 * replaces a full sort): returns the min(N, n) entries of largest |score|,
 * breaking ties at the cutoff by key ascending.  Keys must be distinct.
 * Device pointers; output order unspecified.
 */
int asci_select_topn(const asci_det *keys, const double *scores, size_t n, size_t N,
                     asci_det *out_keys, double *out_scores, size_t *out_n,
                     void *cuda_stream);


/* ---------------------------------------------------------------------------
 * The variational step of the ASCI loop (Algorithm 1: "diagonalize the
 * Hamiltonian in the selected determinant space"; Sec. 2.3).
 * ------------------------------------------------------------------------- */

/*
 * The Hamiltonian restricted to a determinant list, as a sparse matrix in
 * compressed sparse row form (Sec. 2.3: the double loop approach over pairs of
 * determinants, here pruned by beta-string groups; CSR storage).  Row and
 * column i belong to dets[i].  Row i holds its diagonal element H_ii and every
 * H_ij != 0 with dets[j] singly or doubly excited from dets[i] (by the
 * Slater-Condon rules of the conventions above), columns ascending; the matrix
 * is symmetric.
 *
 *  dets[n]       distinct determinants with equal electron counts (n < 2^31).
 *  row_ptr[n+1]  out (int64): row i is entries row_ptr[i] .. row_ptr[i+1]-1.
 *  col, val      out: column indices (int32) and elements (FP64), capacity
 *                entries each.  Both may be NULL with capacity 0.
 *  *nnz          out: the number of stored elements (always written).
 * When capacity < *nnz only row_ptr and *nnz are written (a size query) and
 * the call still returns ASCI_OK; call again with capacity >= *nnz.  Every
 * call runs the counting pass; a call with room also runs the filling pass.
 *
 * Errors: ASCI_EINVAL for norb outside 1..32, n == 0 or n >= 2^31, NULL
 * pointers, determinants with bits at or above norb, mixed electron counts,
 * duplicates, or non-finite integrals; ASCI_ENOMEM; ASCI_ECUDA.
 */
int asci_hamiltonian(const asci_det *dets, size_t n, const asci_ints *ints, int64_t *row_ptr,
                     int32_t *col, double *val, size_t capacity, size_t *nnz,
                     void *cuda_stream);

/*
 * y = H x for a matrix from asci_hamiltonian (the local sparse product of
 * Sec. 2.3, Algorithm 6 on one device).  x[n] in, y[n] out (distinct
 * buffers).  Each y_i is summed in a fixed order: repeated calls give the same
 * bits.
 */
int asci_spmv(const int64_t *row_ptr, const int32_t *col, const double *val, size_t n,
              const double *x, double *y, void *cuda_stream);

/* Davidson controls (Algorithm 5). */
typedef struct {
  int32_t max_subspace; /* Krylov dimension k before a restart, 2..32 (default 16) */
  int32_t max_iter;     /* products with H at most (default 300) */
  double tol;           /* stop when ||H v - E v|| <= tol, v normalised (default 1e-8) */
} asci_davidson_opts;

void asci_default_davidson_opts(asci_davidson_opts *opts);

/*
 * Lowest eigenpair of a matrix from asci_hamiltonian by the Davidson method
 * (Sec. 2.3, Algorithm 5, on one device): the subspace grows by the
 * preconditioned residual R / (E - H_ii) (the shifted Jacobi preconditioner),
 * orthogonalised against the basis by two passes of Gram-Schmidt; the
 * subspace eigenproblem is solved on the device (Jacobi rotations in FP32,
 * refined in FP64); at max_subspace vectors the basis restarts from the four
 * lowest Ritz vectors (fewer when max_subspace <= 4).  The first expansion
 * vector is the unpreconditioned H v0 - (v0.H v0) v0, as in Algorithm 5.
 *
 *  guess[n]    start vector (nullable: the unit vector of the smallest H_ii).
 *  *energy     out: the Ritz value.
 *  vec[n]      out: the Ritz vector, unit norm, largest |component| positive
 *              (lowest index among equal magnitudes).
 *  *iterations out (nullable): products with H performed.
 *  *residual   out (nullable): the final ||H v - E v||.
 * Returns ASCI_OK when converged to tol, ASCI_ETIMEOUT when max_iter products
 * ran first (the outputs then hold the last Ritz pair).
 */
int asci_davidson(const int64_t *row_ptr, const int32_t *col, const double *val, size_t n,
                  const double *guess, const asci_davidson_opts *opts, double *energy,
                  double *vec, int32_t *iterations, double *residual, void *cuda_stream);

/* Controls of the ASCI loop. */
#define ASCI_LOOP_MAX_STEPS 64
typedef struct {
  uint64_t ncdets;    /* core size N_cdets of each search (Alg. 2) */
  uint64_t ntdets;    /* wavefunction size N_tdets kept by each step */
  int32_t max_steps;  /* 1..ASCI_LOOP_MAX_STEPS */
  double etol;        /* stop once a step changes the energy by at most etol */
  asci_opts search;   /* options of every search */
  asci_davidson_opts davidson;
} asci_loop_opts;

/* Per-step record of the ASCI loop (device milliseconds). */
typedef struct {
  int32_t steps;        /* steps run */
  double start_energy;  /* <psi0|H|psi0> / <psi0|psi0> of the start */
  double energy[ASCI_LOOP_MAX_STEPS];
  uint64_t ndets[ASCI_LOOP_MAX_STEPS];       /* |psi| after the step */
  uint64_t new_dets[ASCI_LOOP_MAX_STEPS];    /* determinants that entered */
  uint64_t nnz[ASCI_LOOP_MAX_STEPS];         /* stored elements of H on the step's space */
  int32_t davidson_iters[ASCI_LOOP_MAX_STEPS];
  double t_search[ASCI_LOOP_MAX_STEPS];
  double t_hamiltonian[ASCI_LOOP_MAX_STEPS];
  double t_davidson[ASCI_LOOP_MAX_STEPS];
} asci_loop_stats;

/* Defaults: ncdets 1e4, ntdets 1e5, 8 steps, etol 1e-6 Hartree, default search
 * and Davidson options. */
void asci_default_loop_opts(asci_loop_opts *opts);

/*
 * The ASCI loop (Algorithm 1) from a start wavefunction (for instance the
 * Hartree-Fock determinant with coefficient 1).  E_0 is the start's energy
 * <psi|H|psi>/<psi|psi>.  Each step:
 *   1. searches (asci_search, Algorithm 2) from (psi_k, c_k, E_k) with the
 *      min(ncdets, |psi_k|) core and N = ntdets;
 *   2. keeps the ntdets determinants of largest magnitude among psi_k (valued
 *      by c_k) and the candidates (valued by their score S, Eq. 1), ties by
 *      key ascending, ordered by key;
 *   3. builds H on that space (asci_hamiltonian) and takes its lowest
 *      eigenpair (asci_davidson, guess: the values of step 2) as
 *      (c_{k+1}, E_{k+1}).
 * A candidate whose H_ii equals E_k has no finite score: the call then
 * returns ASCI_EINVAL (start from a wavefunction whose energy lies below the
 * diagonal of every determinant it connects to, e.g. a small CI).
 * The loop stops after max_steps, once |E_{k+1} - E_k| <= etol, or once a
 * step leaves the determinant set unchanged.  The final ASCI-PT2 step of
 * Algorithm 1 is asci_pt2 on the result.
 *
 *  dets[ndets], coeffs[ndets]  the start (distinct determinants, equal counts).
 *  out_dets, out_coeffs        capacity entries each, capacity >= ntdets: the
 *                              final space in key order and its ground vector
 *                              (unit norm, largest |c| positive).
 *  *out_n, *energy             its size and energy.
 *  stats                       nullable.
 * Errors: those of asci_search, asci_hamiltonian and asci_davidson (a
 * Davidson that reaches max_iter unconverged returns ASCI_ETIMEOUT), and
 * ASCI_EINVAL for ncdets or ntdets == 0, capacity < ntdets or max_steps
 * outside 1..ASCI_LOOP_MAX_STEPS.
 */
int asci_loop(const asci_det *dets, const double *coeffs, size_t ndets, const asci_ints *ints,
              const asci_loop_opts *opts, asci_det *out_dets, double *out_coeffs,
              size_t capacity, size_t *out_n, double *energy, asci_loop_stats *stats,
              void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ASCI_H */
