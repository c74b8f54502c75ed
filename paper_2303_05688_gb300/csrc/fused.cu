// Constraint-tile search: the batched hot loop of Algorithm 2 with on-chip
// sort-and-accumulate (Sec. 2.2) and the score of Eq. 1.
//
// Work is partitioned by target alpha string A' (the finest constraint class:
// all occupied alpha orbitals fixed).  Items sorted by A' (see excite.cu) make
// each class a contiguous range; a batch of classes is generated into a
// staging buffer as records (beta', v = H_ij c_j, H_ii) and then reduced tile
// by tile on chip:
//   small classes (<= kCap/2 pairs)   packed, several per tile, in item order
//   medium classes (<= kCap pairs)    one tile each, in item order
//   big classes                       split into hash buckets of beta' (each a
//                                     tile); all contributions to one target
//                                     land in the same bucket
// A tile groups its records by target in a shared-memory hash table (the
// records of each target linked into a list), sums each target's values
// exactly (192-bit fixed point, so the sum does not depend on the order of the
// contributions and equals the sort-and-accumulate result bit for bit), drops
// targets in psi, and scores in FP64 and appends the targets whose |score| can
// reach the running top-N threshold.
//
// The diagonal H_ii is carried exactly in 64-bit fixed point: the integral
// terms are rounded once to multiples of 2^-s, and each pair's H_ii is the
// parent's H_jj plus the excitation's change, computed from the parent's
// Fock-like diagonals F_s(p) = h_pp + sum_{q in s} (J-K)_pq + sum_{q in s'} J_pq.
// Integer sums are exact, so every path to a target gives the same H_ii.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "asci_internal.cuh"
#include "fixed192.cuh"
#include "fused.cuh"

namespace asci {

// ----------------------------------------------------------- fixed point ---


namespace {

__global__ void k_fx_bound(const double *h1, const double *eri, int n, double *out3) {
  // out3[0] = max |h_pp|, out3[1] = max_{p!=q} |J-K|, out3[2] = max_{p,q} |J|
  double a = 0, b = 0, c = 0;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int p = t / n, q = t % n;
    double J = eri[(((size_t)p * n + p) * n + q) * n + q];
    double K = eri[(((size_t)p * n + q) * n + q) * n + p];
    if (p == q) a = fmax(a, fabs(h1[p * n + p]));
    if (p != q) b = fmax(b, fabs(J - K));
    c = fmax(c, fabs(J));
  }
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int i = 0; i < blockDim.x; ++i) {
      s0 = fmax(s0, sh[0][i]);
      s1 = fmax(s1, sh[1][i]);
      s2 = fmax(s2, sh[2][i]);
    }
    out3[0] = s0;
    out3[1] = s1;
    out3[2] = s2;
  }
}

__global__ void k_fx_tables(const double *h1, const double *eri, int n, int s, int64_t *hh,
                            int64_t *jk, int64_t *jj) {
  const double sc = ldexp(1.0, s);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    int p = t / n, q = t % n;
    double J = eri[(((size_t)p * n + p) * n + q) * n + q];
    double K = eri[(((size_t)p * n + q) * n + q) * n + p];
    jk[t] = (p == q) ? 0 : __double2ll_rn((J - K) * sc);
    jj[t] = __double2ll_rn(J * sc);
    if (p == q) hh[p] = __double2ll_rn(h1[p * n + p] * sc);
  }
}

// Largest single-excitation magnitude bound over (i, a):
// |h_ia| + sum_k |(ia|kk) - (ik|ka)| + sum_k |(ia|kk)|.
__global__ void k_fx_single_bound(const double *h1, const double *eri, int n, double *out) {
  double m = 0;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, a = t % n;
    double b = fabs(h1[t]);
    for (int k = 0; k < n; ++k) {
      const double iakk = eri[(((size_t)i * n + a) * n + k) * n + k];
      const double ikka = eri[(((size_t)i * n + k) * n + k) * n + a];
      b += fabs(iakk - ikka) + fabs(iakk);
    }
    m = fmax(m, b);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int i = 0; i < blockDim.x; ++i) r = fmax(r, sh[i]);
    *out = r;
  }
}

__global__ void k_fx_single_tables(const double *h1, const double *eri, int n, int s1,
                                   int64_t *h1x, int64_t *ssx, int64_t *sox) {
  const double sc = ldexp(1.0, s1);
  const size_t n3 = (size_t)n * n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % n), ia = (int)(t / n), i = ia / n, a = ia % n;
    const double iakk = eri[(((size_t)i * n + a) * n + k) * n + k];
    const double ikka = eri[(((size_t)i * n + k) * n + k) * n + a];
    ssx[t] = __double2ll_rn((iakk - ikka) * sc);
    sox[t] = __double2ll_rn(iakk * sc);
    if (k == 0) h1x[ia] = __double2ll_rn(h1[ia] * sc);
  }
}

}  // namespace

// x * 2^-s rounded to the nearest double (ties to even), by integer
// operations only; x * 2^-s must lie in the normal range.
__device__ __forceinline__ double fx64_to_double(int64_t x, int s) {
  if (x == 0) return 0.0;
  const uint64_t sign = x < 0 ? (1ull << 63) : 0ull;
  const uint64_t u = x < 0 ? 0ull - (uint64_t)x : (uint64_t)x;
  int P = 63 - __clzll((long long)u);  // leading bit
  uint64_t mant;
  if (P <= 52) {
    mant = u << (52 - P);
  } else {
    const int sh = P - 52;
    mant = u >> sh;
    const uint64_t rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++P;
      }
    }
  }
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(P - s + 1023) << 52) | (mant & ((1ull << 52) - 1ull))));
}

__device__ __forceinline__ int64_t fx_diag(const FxInts &X, uint32_t A, uint32_t B) {
  const int n = X.n;
  int64_t s = X.ecore_x;
  for (uint32_t m = A; m; m &= m - 1) {
    const int p = __ffs(m) - 1;
    s += X.hh[p];
    for (uint32_t r = m & (m - 1); r; r &= r - 1) s += X.jk[p * n + __ffs(r) - 1];
    for (uint32_t r = B; r; r &= r - 1) s += X.jj[p * n + __ffs(r) - 1];
  }
  for (uint32_t m = B; m; m &= m - 1) {
    const int p = __ffs(m) - 1;
    s += X.hh[p];
    for (uint32_t r = m & (m - 1); r; r &= r - 1) s += X.jk[p * n + __ffs(r) - 1];
  }
  return s;
}

namespace {

// Parent data of each core det (alpha-sorted order): H_jj and both Fock-like
// diagonals.  Fb is determinant-major (Fb[j n + p]: a warp's lanes read one
// determinant's row); Fa is orbital-major (Fa[p m + j]: the lanes of an
// alpha-double step read one orbital of consecutive determinants).
__global__ void k_core_fock(FxInts X, const uint32_t *core_alpha, const uint32_t *core_beta,
                            size_t m, int64_t *Dx, int64_t *Fa, int64_t *Fb) {
  const int n = X.n;
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (size_t)gridDim.x * blockDim.x) {
    const uint32_t A = core_alpha[j], B = core_beta[j];
    Dx[j] = fx_diag(X, A, B);
    for (int p = 0; p < n; ++p) {
      int64_t fa = X.hh[p], fb = X.hh[p];
      for (uint32_t r = A; r; r &= r - 1) {
        int q = __ffs(r) - 1;
        fa += X.jk[p * n + q];
        fb += X.jj[p * n + q];
      }
      for (uint32_t r = B; r; r &= r - 1) {
        int q = __ffs(r) - 1;
        fb += X.jk[p * n + q];
        fa += X.jj[p * n + q];
      }
      Fa[(size_t)p * m + j] = fa;
      Fb[j * n + p] = fb;
    }
  }
}


// ------------------------------------------------------ groups of items ---

// gid holds the exclusive scan of the head flags; it becomes each item's group
// (heads up to and including it, less one), and each head fills its group's
// row.  Row G (one past the last group) gets the totals: T items, P pairs.
__global__ void k_group_tab(const uint64_t *items, uint32_t *gid, const uint64_t *Wexcl, uint64_t T,
                            uint32_t *g_alpha, uint64_t *g_P0, uint64_t *g_item0) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t hi = (uint32_t)(items[t] >> 32);
    const bool head = t == 0 || hi != (uint32_t)(items[t - 1] >> 32);
    const uint32_t g = gid[t] + (head ? 1u : 0u) - 1u;
    gid[t] = g;
    if (head) {
      g_alpha[g] = hi;
      g_P0[g] = Wexcl[t];
      g_item0[g] = t;
    }
    if (t == T - 1) {
      g_alpha[g + 1] = 0;
      g_P0[g + 1] = Wexcl[T];
      g_item0[g + 1] = T;
    }
  }
}

// ------------------------------------------------------- tile planning ---

enum : uint32_t { kTilePacked = 0, kTileMedium = 1, kTileBucket = 2 };

// bits of the device error word of the constraint-tile kernels
constexpr unsigned kErrProbe = 1u;      // exclusion probe ran past the table
constexpr unsigned kErrTile = 2u;       // a tile descriptor outside its limits
constexpr unsigned kErrStage = 4u;      // a record position outside the staging buffer
constexpr unsigned kErrCore = 8u;       // a core index outside the core
constexpr unsigned kErrAccum = 16u;     // a value outside the exact accumulator's range

struct TileDesc {  // 32 bytes; npairs at byte offset 4 (read by the host)
  uint32_t start;   // first record in the batch staging buffer
  uint32_t npairs;  // records in the tile
  uint32_t g0;      // first group (global id)
  uint32_t ng;      // groups (packed tiles)
  uint32_t kind;
  uint32_t alpha;   // target alpha string (medium / bucket tiles)
  uint32_t psi_lo;  // psi determinants that fall in the tile: [psi_lo, psi_hi) of
  uint32_t psi_hi;  // the batch's tile-ordered psi list
};

static_assert(sizeof(TileDesc) == 32, "tile descriptor layout");

// A screened-out record (Alg. 2's eps test) keeps its slot with a NaN value.
// (Tested on the bits: NaN compares cost FP64 instructions, which are scarce.)
__device__ __forceinline__ bool is_dropped(double v) {
  return ((uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ double drop_marker() {
  return __longlong_as_double(0x7ff8000000000000ll);
}
// Sum of four values that depends only on their multiset: they are ordered by
// magnitude (then sign) with a sorting network on the bits and added from the
// smallest.  Pad with +0.0 for fewer values.
__device__ __forceinline__ uint64_t mag_order(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b << 1) | (b >> 63);
}
__device__ __forceinline__ void order2(double &x, double &y) {
  if (mag_order(y) < mag_order(x)) {
    const double t = x;
    x = y;
    y = t;
  }
}
__device__ __forceinline__ double sum4_ordered(double a, double b, double c, double d) {
  order2(a, b);
  order2(c, d);
  order2(a, c);
  order2(b, d);
  order2(b, c);
  return ((a + b) + c) + d;
}

// x with its sign flipped when flip is 1 (an integer operation on the bits).
__device__ __forceinline__ double flip_sign(double x, uint32_t flip) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(flip & 1u) << 63));
}

}  // namespace

constexpr int kCellThreads = 256;
constexpr int kCap = 1024;                          // records per tile
constexpr uint32_t kSmallMax = kCap / 2;            // packable class size
constexpr uint32_t kBucketTarget = kCap * 13 / 16;  // expected records per hash bucket

namespace {

// Tile kind of each class and its staging slots: its pairs in place, or kCap
// slots for each hash bucket of a big class.
__global__ void k_group_class(const uint64_t *g_P0, uint32_t gb0, uint32_t gb1, uint64_t Pend,
                              uint32_t *kind, uint32_t *nb, uint64_t *small_pairs,
                              uint64_t *slots) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < gb1 - gb0;
       i += gridDim.x * blockDim.x) {
    const uint32_t g = gb0 + i;
    const uint64_t P = ((g + 1 < gb1) ? g_P0[g + 1] : Pend) - g_P0[g];
    uint32_t k = P <= kSmallMax ? kTilePacked : (P <= kCap ? kTileMedium : kTileBucket);
    kind[i] = k;
    nb[i] = k == kTileBucket ? (uint32_t)((P + kBucketTarget - 1) / kBucketTarget) : 0u;
    small_pairs[i] = k == kTilePacked ? P : 0;
    slots[i] = k == kTileBucket ? (uint64_t)nb[i] * kCap : P;
  }
}

__device__ __forceinline__ bool packed_start(uint32_t i, const uint32_t *kind,
                                             const uint64_t *Ws) {
  if (kind[i] != kTilePacked) return false;
  if (i == 0 || kind[i - 1] != kTilePacked) return true;
  return (Ws[i] / kSmallMax) != (Ws[i - 1] / kSmallMax);
}

__global__ void k_tile_count(uint32_t ng, const uint32_t *kind, const uint32_t *nb,
                             const uint64_t *Ws, uint32_t *ntile) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x)
    ntile[i] = kind[i] == kTilePacked ? (packed_start(i, kind, Ws) ? 1u : 0u)
                                      : (kind[i] == kTileMedium ? 1u : nb[i]);
}

__global__ void k_tile_write(uint32_t gb0, uint32_t ng, const uint64_t *soff, uint64_t Pend,
                             const uint64_t *g_P0, const uint32_t *g_alpha,
                             const uint32_t *kind, const uint32_t *nb, const uint64_t *Ws,
                             const uint32_t *tile_base, TileDesc *tiles) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
    const uint32_t g = gb0 + i;
    const uint64_t P = ((i + 1 < ng) ? g_P0[g + 1] : Pend) - g_P0[g];
    const uint32_t start = (uint32_t)soff[i];
    const uint32_t k = kind[i];
    if (k == kTilePacked) {
      const bool st = packed_start(i, kind, Ws);
      const uint32_t t = st ? tile_base[i] : tile_base[i] - 1;
      if (st) {
        tiles[t].start = start;
        tiles[t].g0 = g;
        tiles[t].kind = kTilePacked;
        tiles[t].alpha = g_alpha[g];
      }
      atomicAdd(&tiles[t].npairs, (uint32_t)P);
      atomicAdd(&tiles[t].ng, 1u);
    } else if (k == kTileMedium) {
      TileDesc d;
      d.start = start;
      d.npairs = (uint32_t)P;
      d.g0 = g;
      d.ng = 1;
      d.kind = kTileMedium;
      d.alpha = g_alpha[g];
      d.psi_lo = d.psi_hi = 0;
      tiles[tile_base[i]] = d;
    }
  }
}

// Bucket tiles of big classes, one thread per cell: the class holding cell c
// is the last one whose first cell is at or before c.  Bucket b of a class
// owns kCap staging slots; its record count is known after emission.
__global__ void k_cell_write(uint32_t gb0, uint32_t ng, uint32_t ncells, const uint64_t *soff,
                             const uint32_t *g_alpha, const uint32_t *tile_base,
                             const uint32_t *cellbase, TileDesc *tiles, uint32_t *cell_pos0,
                             uint32_t *cell_tile) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = ng - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (cellbase[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const uint32_t g = gb0 + lo, b = c - cellbase[lo];
    TileDesc d;
    d.start = (uint32_t)(soff[lo] + (uint64_t)b * kCap);
    d.npairs = 0;
    d.g0 = g;
    d.ng = 1;
    d.kind = kTileBucket;
    d.alpha = g_alpha[g];
    d.psi_lo = d.psi_hi = 0;
    tiles[tile_base[lo] + b] = d;
    cell_pos0[c] = d.start;
    cell_tile[c] = tile_base[lo] + b;
  }
}

// Sort keys of the spilled records: tile << 32 | spill index.
__global__ void k_spill_keys(const uint32_t *spill_cell, const uint32_t *cell_tile, uint32_t n,
                             uint64_t *keys) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    keys[j] = ((uint64_t)cell_tile[spill_cell[j]] << 32) | j;
}

// Record counts of the bucket tiles after emission; a bucket that received
// more than kCap records (its surplus is in the spill list) is reduced by the
// global path.
__global__ void k_cell_finish(uint32_t ncells, const uint32_t *fill, const uint32_t *cell_tile,
                              TileDesc *tiles, unsigned *n_over, uint32_t *over_list,
                              uint32_t over_cap) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
       c += gridDim.x * blockDim.x) {
    const uint32_t f = fill[c], t = cell_tile[c];
    tiles[t].npairs = f;
    if (f > (uint32_t)kCap) {
      const unsigned slot = atomicAdd(n_over, 1u);
      if (slot < over_cap) over_list[slot] = t;
    }
  }
}

// ------------------------------------------------------------ emission ---

__device__ __forceinline__ uint32_t bucket_of(uint32_t beta, uint32_t nb) {
  return (uint32_t)(((uint64_t)(beta * 0x9E3779B1u) * nb) >> 32);
}

// ----------------------------------------------------------- emission ---
// The pairs of a batch are emitted in two kinds of work units.
//  * Determinant runs: an item (core alpha group k, alpha operation o) whose
//    o is the identity or an alpha single, applied to one core determinant of
//    the group.  For o = 0 the run holds the determinant's beta singles and
//    beta doubles (sb + dbb pairs); for an alpha single, that single alone
//    and combined with each beta single (1 + sb pairs).  One warp walks a
//    run: lane L holds the L-th occupied and the L-th virtual beta orbital of
//    the determinant and the diagonal terms that depend on them, and each
//    pair fetches its orbitals and terms with shuffles.
//  * Alpha doubles: one pair per core determinant of the group.  These items
//    are laid out flat and each lane takes one pair; the operation, its
//    matrix element and the determinant-independent part of the diagonal
//    change are computed once per item.
// A pair keeps the position p = Wexcl[t] + m * npd + e of the item order
// (t: item, m: determinant in the group, e: pair in the run), so classes that
// fit a tile are staged in place and big classes go through bucket counters.

constexpr int kRunThreads = 256;
constexpr int kRunClaim = 4;   // runs a warp claims at a time
// A determinant's o = 0 run (its beta singles and doubles, 10,314 pairs at
// (24e,30o)) is emitted in pieces of at most this many pairs, so that the
// last runs of a launch are short and its warps finish together.
constexpr uint32_t kPiecePairs = 1024;
constexpr int kPairTab = 496;  // C(32, 2): unranked index pairs
constexpr int kAdThreads = 256;
constexpr int kAdTile = 512;   // alpha-double pairs per CTA step

struct EmitArgs {
  DevInts I;
  FxInts X;
  ExcCounts E;
  FastDiv dv_va, dv_vb, dv_pa_p, dv_pb_p;
  uint32_t npd0, npd1;        // pairs per determinant for o = 0 and for an alpha single
  uint32_t npieces;           // pieces of kPiecePairs pairs a determinant's o = 0 run is cut into
  const uint64_t *items, *Wexcl;
  const uint32_t *item_group;
  uint64_t t0, P0;
  int opbits;
  const uint32_t *grp_alpha, *grp_start, *grp_count, *core_beta;
  const double *core_c;
  const int64_t *Dx, *Fa, *Fb;
  uint32_t gb0;
  const uint32_t *kind, *nb, *cellbase;
  const uint64_t *soff;       // first staging slot of each class of the batch
  const uint64_t *g_P0;       // first pair of each class
  const uint32_t *cell_pos0;  // first staging slot of each bucket cell
  uint32_t *fill;             // records placed in each bucket cell
  StageRec *spill_rec;        // records beyond a cell's kCap slots
  uint32_t *spill_cell;
  unsigned *n_spill;
  uint32_t spill_cap;
  const uint64_t *runs;       // (item - t0) << 32 | determinant in the group
  uint64_t nruns;
  unsigned long long *run_next;  // next unclaimed run (zeroed before each launch)
  const uint32_t *adl;        // alpha-double items (item - t0)
  const uint32_t *ad_off;     // first flat pair of each (exclusive prefix)
  uint32_t nad, ad_total;
  const uint32_t *opinfo;     // per batch item: alpha single i | a << 5 | parity << 10
  const uint32_t *ad_tile_item;  // first alpha-double item of each CTA step
  uint32_t ad_tiles;
  Stage st;
  double eps;                 // Alg. 2 screen; 0 keeps every pair
  float eps_f;                // eps as a float (the screen's float pre-test)
  int64_t E0_x;
  double inv_scale;
  unsigned long long *survivors;
  uint32_t ncore;
  unsigned *err;
};

__device__ __forceinline__ void dec_single(uint32_t s, uint32_t virt, uint32_t idx,
                                           const FastDiv &dv, int *i, int *a) {
  uint32_t q = dv.div(idx);
  *i = nth_set_bit(s, (int)q);
  *a = nth_set_bit(virt, (int)(idx - q * dv.d));
}

__device__ __forceinline__ void dec_double(uint32_t s, uint32_t virt, uint32_t idx,
                                           const FastDiv &dv, int *i, int *j, int *a, int *b) {
  uint32_t q = dv.div(idx);
  int h1, h2, p1, p2;
  unrank_pair(q, &h1, &h2);
  unrank_pair(idx - q * dv.d, &p1, &p2);
  *i = nth_set_bit(s, h1);
  *j = nth_set_bit(s, h2);
  *a = nth_set_bit(virt, p1);
  *b = nth_set_bit(virt, p2);
}

__device__ __forceinline__ int par_double(uint32_t s, int i, int j, int a, int b) {
  int p1 = single_parity(s, i, a);
  uint32_t s1 = s ^ (1u << i) ^ (1u << a);
  return p1 ^ single_parity(s1, j, b);
}

// Single excitation i -> a of the string s (the other spin's string o) in
// fixed point (multiples of 2^-s1): h_ia plus, over the occupied orbitals k,
// (ia|kk) - (ik|ka) for k of the same spin and (ia|kk) for k of the other.
__device__ __forceinline__ int64_t fx_single(const FxInts &X, uint32_t s, uint32_t o, int i,
                                             int a) {
  const int n = X.n;
  const int64_t *ss = X.ssx + ((size_t)i * n + a) * n;
  const int64_t *so = X.sox + ((size_t)i * n + a) * n;
  int64_t v = X.h1x[i * n + a];
  for (uint32_t m = s; m; m &= m - 1) v += ss[__ffs(m) - 1];
  for (uint32_t m = o; m; m &= m - 1) v += so[__ffs(m) - 1];
  return v;
}

__device__ __forceinline__ int64_t shfl64(int64_t x, int src) {
  return (int64_t)__shfl_sync(0xffffffffu, (long long)x, src);
}

// A float widened to a double exactly, by operations on the bits (a widening
// conversion would take the FP64 pipe, which is scarce).
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  if (e == 0xffu)  // inf or nan
    return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((uint64_t)m << 29)));
  if (e == 0) {    // zero or subnormal: normalise the mantissa
    if (!m) return __longlong_as_double((long long)sign);
    const int lz = __clz(m) - 8;  // leading zeros within the 23-bit field, plus one
    const uint64_t mm = ((uint64_t)m << lz) & 0x7fffffu;
    return __longlong_as_double(
        (long long)(sign | ((uint64_t)(1023 - 126 - lz) << 52) | (mm << 29)));
  }
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(e + 1023 - 127) << 52) | ((uint64_t)m << 29)));
}

// Precision of the pair values (the a8 variant): 0 = FP64 integrals and
// product; 1 = two-electron elements gathered from FP32 tables, FP64 product;
// 2 = FP32 tables and an FP32 product H_ij c_j.  Sums and diagonals are the
// same in all three.
template <int PREC>
__device__ __forceinline__ double pair_value(double h, double c, float cf) {
  if (PREC == 2) return widen((float)h * cf);
  return h * c;
}

// z * 2^-s as a float built from the bits (truncated, relative error below
// 2^-23); 0 when z is zero or the value lies outside the normal float range.
__device__ __forceinline__ float scaled_as_float(int64_t z, int s) {
  if (!z) return 0.0f;
  const uint64_t u = z < 0 ? 0ull - (uint64_t)z : (uint64_t)z;
  const int lz = __clzll((long long)u);
  const int e = 63 - lz - s + 127;
  if (e < 1 || e > 254) return 0.0f;
  const uint32_t mant = (uint32_t)((u << lz) >> 40) & 0x7fffffu;
  return __uint_as_float((z < 0 ? 0x80000000u : 0u) | ((uint32_t)e << 23) | mant);
}

// |x| as a float built from the bits, truncated (relative error below 2^-23);
// *ok is false when |x| lies outside the normal float range.
__device__ __forceinline__ float abs_as_float(double x, bool *ok) {
  const uint64_t b = (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
  int e = (int)(b >> 52) - 1023 + 127;
  *ok = e >= 1 && e <= 254;
  e = e < 1 ? 1 : (e > 254 ? 254 : e);
  return __uint_as_float(((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
}

template <bool EPS>
__device__ __forceinline__ void write_record(const EmitArgs &A, uint32_t pos, bool spill,
                                             uint32_t cell, uint32_t talpha, uint32_t tb,
                                             bool packed, double v, int64_t haa, bool *kept) {
  const float df = scaled_as_float(A.E0_x - haa, A.X.s);
  if (EPS) {
    // Alg. 2's screen |v / (E0 - H_ii)| > eps, without a division.  A float
    // test settles every pair that is not within 4e-6 relative of the
    // threshold (|v| and |E0 - H_ii| truncated to floats lie within 2^-23
    // below their values, eps_f within 2^-24 of eps, the product within
    // 2^-24); the rest take the FP64 test, so every decision is the FP64
    // test's.  (FP64 instructions are scarce on this GPU.)
    bool okv;
    const float vf = abs_as_float(v, &okv);
    const float t = A.eps_f * fabsf(df);
    bool keep;
    if (okv && t > 1e-37f && t < 1e37f && vf > t * 1.000004f) {
      keep = true;
    } else if (okv && t > 1e-37f && t < 1e37f && vf < t * 0.999996f) {
      keep = false;
    } else {
      const double den = __ll2double_rn(A.E0_x - haa) * A.inv_scale;
      keep = fabs(v) > A.eps * fabs(den);
    }
    if (!keep) v = drop_marker();
    *kept = keep;
  }
  const uint64_t vb = (uint64_t)__double_as_longlong(v);
  const uint4 r = make_uint4((uint32_t)vb, (uint32_t)(vb >> 32), tb, __float_as_uint(df));
  if (spill) {
    if (pos < A.spill_cap) {  // beyond: counted only, the host reports it
      reinterpret_cast<uint4 *>(A.spill_rec)[pos] = r;
      A.spill_cell[pos] = cell;
    }
  } else if (pos < A.st.cap) {
    reinterpret_cast<uint4 *>(A.st.rec)[pos] = r;
    if (packed) A.st.alpha[pos] = talpha;
  } else {
    atomicOr(A.err, kErrStage);
  }
}

// The pairs an emission thread kept under the eps screen, added to the
// search's counter once per warp when the kernel ends (one counter for the
// whole grid: an atomic per chunk would serialise on it).
__device__ __forceinline__ void add_survivors(const EmitArgs &A, unsigned long long kept) {
  for (int d = 16; d; d >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, d);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(A.survivors, kept);
}

// EPS compiles Alg. 2's screen in (eps > 0); PREC selects the pair-value
// precision (pair_value).
template <bool EPS, int PREC>
__global__ void __launch_bounds__(kRunThreads, 4) k_emit_runs(EmitArgs A) {
  extern __shared__ int64_t s_fx[];  // emit mode: jk[n*n], jj[n*n]
  __shared__ uint16_t s_pair[kPairTab];
  const int n = A.I.n;
  int64_t *s_jk = s_fx, *s_jj = s_fx + n * n;
  for (int t = threadIdx.x; t < n * n; t += kRunThreads) {
    s_jk[t] = A.X.jk[t];
    s_jj[t] = A.X.jj[t];
  }
  for (int r = threadIdx.x; r < kPairTab; r += kRunThreads) {
    int x, y;
    unrank_pair((uint32_t)r, &x, &y);
    s_pair[r] = (uint16_t)(x | (y << 8));
  }
  __syncthreads();
  const uint32_t full = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  const uint32_t omask = (1u << A.opbits) - 1u;
  const int lane = threadIdx.x & 31;
  const uint32_t sb = A.E.sb, vb = A.E.vb;
  unsigned long long my_kept = 0;  // pairs kept by the eps screen (EPS)
  // runs are claimed kRunClaim at a time from a shared counter (their lengths
  // differ by a factor of about fifty); the next claim is issued before the
  // claimed runs are emitted
  unsigned long long claim = 0;
  if (lane == 0) claim = atomicAdd(A.run_next, (unsigned long long)kRunClaim);
  uint64_t r0 = (uint64_t)__shfl_sync(0xffffffffu, claim, 0);
#pragma unroll 1
  for (; r0 < A.nruns; r0 = (uint64_t)__shfl_sync(0xffffffffu, claim, 0)) {
    if (lane == 0) claim = atomicAdd(A.run_next, (unsigned long long)kRunClaim);
    const uint64_t r1 = r0 + kRunClaim < A.nruns ? r0 + kRunClaim : A.nruns;
#pragma unroll 1
  for (uint64_t r = r0; r < r1; ++r) {
    const uint64_t run = A.runs[r];
    const uint64_t t = A.t0 + (run >> 32);
    const uint64_t it = A.items[t];
    const uint32_t k = (uint32_t)it >> A.opbits, o = (uint32_t)it & omask;
    // determinant m of the group; for o = 0, piece number m % npieces of its run
    const uint32_t mr = (uint32_t)run;
    const uint32_t m = o == 0 ? mr / A.npieces : mr;
    const uint32_t ebeg = o == 0 ? (mr - m * A.npieces) * kPiecePairs : 0u;
    const uint32_t gi = A.item_group[t] - A.gb0;
    const uint32_t kd = A.kind[gi];
    const bool big = kd == kTileBucket, packed = kd == kTilePacked;
    const uint32_t jdx = A.grp_start[k] + m;
    if (jdx >= A.ncore) {
      if (lane == 0) atomicOr(A.err, kErrCore);
      continue;
    }
    const uint32_t talpha = (uint32_t)(it >> 32);
    const uint32_t Ak = A.grp_alpha[k], B = A.core_beta[jdx];
    const uint32_t npd = o == 0 ? A.npd0 : A.npd1;
    const uint32_t eend = npd < ebeg + kPiecePairs ? npd : ebeg + kPiecePairs;
    const uint64_t p0 = A.Wexcl[t] + (uint64_t)m * npd;
    // in-place staging slot of the run's first pair (classes that fit a tile)
    const uint32_t off0 = (uint32_t)(A.soff[gi] + (p0 - A.g_P0[A.gb0 + gi]));
    const uint32_t cell0 = big ? A.cellbase[gi] : 0u, nbk = big ? A.nb[gi] : 1u;
    const uint32_t cls0 = (uint32_t)A.soff[gi];  // bucket b's slots start at cls0 + b kCap
    // lane L: the L-th occupied and the L-th virtual beta orbital of B
    const int occL = lane < (int)A.E.nb ? nth_set_bit(B, lane) : 0;
    const int virL = lane < (int)vb ? nth_set_bit(~B & full, lane) : 0;
    // emit mode: coefficient, alpha part of the diagonal change, and per lane
    // the diagonal terms of removing occL / adding virL (Fock-like diagonal of
    // B, plus the alpha-beta Coulomb change when o is an alpha single)
    double c = 0.0;
    int64_t base_x = 0, Vo = 0, Vv = 0;
    int ia = 0, aa = 0;
    uint32_t pa = 0;
    double h0 = 0.0;  // the alpha single alone
    const double *erow = A.I.eri;
    const float *erow32 = A.I.eri32;
    float cf = 0.0f;
    {
      c = A.core_c[jdx];
      cf = (float)c;
      base_x = A.Dx[jdx];
      const int64_t *Fb = A.Fb + (size_t)jdx * n;
      Vo = Fb[occL];
      Vv = Fb[virL];
      if (o != 0) {
        const uint32_t oi = A.opinfo[t - A.t0];
        ia = (int)(oi & 31u);
        aa = (int)((oi >> 5) & 31u);
        pa = (oi >> 10) & 1u;
        // its matrix element, summed across the warp: lane L adds the terms of
        // the L-th occupied alpha and beta orbitals
        const int occA = lane < (int)A.E.na ? nth_set_bit(Ak, lane) : 0;
        const size_t row = ((size_t)ia * n + aa) * n;
        int64_t part = (lane < (int)A.E.na ? A.X.ssx[row + occA] : 0) +
                       (lane < (int)A.E.nb ? A.X.sox[row + occL] : 0);
#pragma unroll
        for (int d = 16; d; d >>= 1) part += (int64_t)__shfl_xor_sync(0xffffffffu, (long long)part, d);
        h0 = flip_sign(fx64_to_double(part + A.X.h1x[ia * n + aa], A.X.s1), pa);
        base_x += A.Fa[(size_t)aa * A.ncore + jdx] - A.Fa[(size_t)ia * A.ncore + jdx] -
                  s_jk[aa * n + ia];
        Vo += s_jj[aa * n + occL] - s_jj[ia * n + occL];
        Vv += s_jj[aa * n + virL] - s_jj[ia * n + virL];
        erow = A.I.eri + ((size_t)ia * n + aa) * n * n;
        if (PREC != 0) erow32 = A.I.eri32 + ((size_t)ia * n + aa) * n * n;
      }
    }
    // one chunk of 32 pairs: the beta operation as positions in the occupied /
    // virtual lists (op 0: none, the alpha single alone; 1: beta single;
    // 2: beta double), its orbitals and the target beta string
    struct Chunk {
      uint32_t h1, h2, p1, p2;
      int op, bi, bj, ba, bb;
      uint32_t tb, pos, cell;
      bool valid, wr, spill;
      double g;  // the gathered integral (beta double; alpha x beta single), issued ahead
    };
    auto decode = [&](uint32_t e0, Chunk &q) {
      const uint32_t e = e0 + lane;
      q.valid = e < eend;
      q.op = 0;
      q.h1 = q.h2 = q.p1 = q.p2 = 0;
      if (q.valid) {
        if (o == 0 && e >= sb) {
          q.op = 2;
          const uint32_t f = e - sb, qq = A.dv_pb_p.div(f);
          const uint32_t hp = s_pair[qq], pp = s_pair[f - qq * A.dv_pb_p.d];
          q.h1 = hp & 0xffu;
          q.h2 = hp >> 8;
          q.p1 = pp & 0xffu;
          q.p2 = pp >> 8;
        } else if (o == 0 || e > 0) {
          q.op = 1;
          const uint32_t f = o == 0 ? e : e - 1, qq = A.dv_vb.div(f);
          q.h1 = qq;
          q.p1 = f - qq * vb;
        }
      }
      q.bi = __shfl_sync(0xffffffffu, occL, (int)q.h1);
      q.bj = __shfl_sync(0xffffffffu, occL, (int)q.h2);
      q.ba = __shfl_sync(0xffffffffu, virL, (int)q.p1);
      q.bb = __shfl_sync(0xffffffffu, virL, (int)q.p2);
      q.tb = B;
      if (q.op == 1) q.tb ^= (1u << q.bi) | (1u << q.ba);
      if (q.op == 2) q.tb ^= (1u << q.bi) | (1u << q.bj) | (1u << q.ba) | (1u << q.bb);
      const uint32_t bkt = big ? bucket_of(q.tb, nbk) : 0u;
      q.cell = cell0 + bkt;
      q.pos = 0;
      q.spill = false;
      q.wr = q.valid;
      if (big) {  // warp-uniform: the next free slot of the lane's bucket cell
        const uint32_t peers = __match_any_sync(0xffffffffu, q.valid ? q.cell : 0xffffffffu);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (q.valid && lane == leader) base = atomicAdd(&A.fill[q.cell], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        const uint32_t slot = base + __popc(peers & ((1u << lane) - 1u));
        if (slot < (uint32_t)kCap) {
          q.pos = cls0 + bkt * (uint32_t)kCap + slot;
        } else if (q.valid) {  // the cell is full: the spill list
          q.spill = true;
          q.pos = atomicAdd(A.n_spill, 1u);
        }
      } else {
        q.pos = off0 + e;
      }
      // the chunk's integral gather, issued now and used one chunk later
      q.g = 0.0;
      if (q.op == 2) {
        const size_t ix = (((size_t)q.bj * n + q.bb) * n + q.bi) * n + q.ba;
        q.g = PREC != 0 ? widen(A.I.asymT32[ix]) : A.I.asymT[ix];
      } else if (q.op == 1 && o != 0) {
        q.g = PREC != 0 ? widen(erow32[q.bi * n + q.ba]) : erow[q.bi * n + q.ba];
      }
    };
    // software-pipelined: the next chunk's staging slots (an atomic for big
    // classes) and integrals are requested before this chunk's matrix
    // elements are formed
    Chunk cur, nxt;
    decode(ebeg, cur);
#pragma unroll 1
    for (uint32_t e0 = ebeg; e0 < eend; e0 += 32) {
      if (e0 + 32 < eend) decode(e0 + 32, nxt);  // warp-uniform
      double h = 0.0;
      int64_t dh = 0;
      {
        const int64_t vo1 = shfl64(Vo, (int)cur.h1), vv1 = shfl64(Vv, (int)cur.p1);
        int64_t vo2 = 0, vv2 = 0;
        if (o == 0) {  // warp-uniform
          vo2 = shfl64(Vo, (int)cur.h2);
          vv2 = shfl64(Vv, (int)cur.p2);
        }
        const int bi = cur.bi, bj = cur.bj, ba = cur.ba, bb = cur.bb;
        if (cur.op == 0) {
          h = h0;
        } else if (cur.op == 1) {
          if (o == 0)
            h = flip_sign(fx64_to_double(fx_single(A.X, B, Ak, bi, ba), A.X.s1),
                          (uint32_t)single_parity(B, bi, ba));
          else
            h = flip_sign(cur.g, pa ^ (uint32_t)single_parity(B, bi, ba));
          dh = vv1 - vo1 - s_jk[ba * n + bi];
        } else {
          h = flip_sign(cur.g, (uint32_t)par_double(B, bi, bj, ba, bb));
          dh = vv1 + vv2 - vo1 - vo2 + s_jk[bi * n + bj] + s_jk[ba * n + bb] - s_jk[ba * n + bi] -
               s_jk[ba * n + bj] - s_jk[bb * n + bi] - s_jk[bb * n + bj];
        }
      }
      bool kept = false;
      if (cur.wr)
        write_record<EPS>(A, cur.pos, cur.spill, cur.cell, talpha, cur.tb, packed,
                          pair_value<PREC>(h, c, cf), base_x + dh, &kept);
      if (EPS) my_kept += kept ? 1u : 0u;
      cur = nxt;
    }
  }
  }
  if (EPS) add_survivors(A, my_kept);
}

// Alpha-double pairs, flat: CTA step s covers flat pairs [s * kAdTile, ...).
template <bool EPS, int PREC>
__global__ void __launch_bounds__(kAdThreads) k_emit_ad(EmitArgs A) {
  __shared__ uint32_t sF[kAdTile + 1];    // first flat pair of each item in the step
  __shared__ uint32_t sPos[kAdTile + 1];  // in-place staging slot of the item's first pair
  __shared__ uint32_t sG[kAdTile + 1];    // first core determinant of the item's group
  __shared__ uint32_t sOrb[kAdTile + 1];  // i | a << 5 | j << 10 | b << 15
  __shared__ uint32_t sTA[kAdTile + 1];   // target alpha string
  __shared__ uint32_t sCls[kAdTile + 1];  // class (relative to the batch)
  __shared__ uint32_t sBase[kAdTile + 1]; // first staging slot of the class
  __shared__ double sH[kAdTile + 1];      // signed matrix element
  __shared__ int64_t sD[kAdTile + 1];     // determinant-independent diagonal change
  __shared__ uint16_t sItem[kAdTile];     // item of each pair of the step
  const int n = A.I.n;
  const uint32_t full = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  const uint32_t omask = (1u << A.opbits) - 1u;
  const int lane = threadIdx.x & 31;
  unsigned long long my_kept = 0;  // pairs kept by the eps screen (EPS)
#pragma unroll 1
  for (uint32_t step = blockIdx.x; step < A.ad_tiles; step += gridDim.x) {
    const uint32_t fb = step * kAdTile;
    const uint32_t fe = fb + kAdTile < A.ad_total ? fb + kAdTile : A.ad_total;
    const uint32_t ja = A.ad_tile_item[step];
    uint32_t jl = A.ad_tile_item[step + 1];
    if (jl >= A.nad) jl = A.nad - 1;
    const int nspan = (int)(jl - ja + 1);  // <= kAdTile + 1: every item has >= 1 pair
    for (int i = threadIdx.x; i < nspan; i += kAdThreads) {
      const uint64_t t = A.t0 + A.adl[ja + i];
      const uint64_t it = A.items[t];
      const uint32_t k = (uint32_t)it >> A.opbits, o = (uint32_t)it & omask;
      const uint32_t gi = A.item_group[t] - A.gb0;
      sF[i] = A.ad_off[ja + i];
      sPos[i] = (uint32_t)(A.soff[gi] + (A.Wexcl[t] - A.g_P0[A.gb0 + gi]));
      sBase[i] = (uint32_t)A.soff[gi];
      sG[i] = A.grp_start[k];
      sTA[i] = (uint32_t)(it >> 32);
      sCls[i] = gi;
      {
        const uint32_t Ak = A.grp_alpha[k];
        int ia, ja2, aa, ba;
        dec_double(Ak, ~Ak & full, o - 1 - A.E.sa, A.dv_pa_p, &ia, &ja2, &aa, &ba);
        sOrb[i] = (uint32_t)ia | ((uint32_t)aa << 5) | ((uint32_t)ja2 << 10) | ((uint32_t)ba << 15);
        const size_t ix = (((size_t)ia * n + aa) * n + ja2) * n + ba;
        sH[i] = flip_sign(PREC != 0 ? widen(A.I.asym32[ix]) : A.I.asym[ix],
                          (uint32_t)par_double(Ak, ia, ja2, aa, ba));
        const int64_t *jk = A.X.jk;
        sD[i] = jk[ia * n + ja2] + jk[aa * n + ba] - jk[aa * n + ia] - jk[aa * n + ja2] -
                jk[ba * n + ia] - jk[ba * n + ja2];
      }
    }
    __syncthreads();
    // pair -> item map of the step: each item marks its pairs
    for (int i = threadIdx.x; i < nspan; i += kAdThreads) {
      const uint32_t a0 = sF[i] > fb ? sF[i] : fb;
      const uint32_t e1 = i + 1 < nspan ? sF[i + 1] : fe;
      const uint32_t a1 = e1 < fe ? e1 : fe;
      for (uint32_t f = a0; f < a1; ++f) sItem[f - fb] = (uint16_t)i;
    }
    __syncthreads();
#pragma unroll 1
    for (uint32_t f0 = fb + (threadIdx.x & ~31u); f0 < fe; f0 += kAdThreads) {
      const uint32_t f = f0 + lane;
      const bool valid = f < fe;
      const int lo = valid ? (int)sItem[f - fb] : 0;
      const uint32_t q = valid ? f - sF[lo] : 0u;
      uint32_t jdx = sG[lo] + q;
      const uint32_t gi = sCls[lo];
      const bool bigl = valid && A.kind[gi] == kTileBucket;
      const bool big = __any_sync(0xffffffffu, bigl);
      if (valid && jdx >= A.ncore) {
        atomicOr(A.err, kErrCore);
        jdx = 0;
      }
      const uint32_t B = valid ? A.core_beta[jdx] : 0u;
      // lanes of one warp may straddle classes of both kinds: position per lane
      uint32_t pos = sPos[lo] + q, cell = 0;
      bool spill = false;
      uint32_t bkt = 0;
      if (big) {
        bkt = bigl ? bucket_of(B, A.nb[gi]) : 0u;
        cell = bigl ? A.cellbase[gi] + bkt : 0u;
        const uint32_t peers = __match_any_sync(0xffffffffu, bigl ? cell : 0xffffffffu);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (bigl && lane == leader) base = atomicAdd(&A.fill[cell], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (bigl) {
          const uint32_t slot = base + __popc(peers & ((1u << lane) - 1u));
          if (slot < (uint32_t)kCap) {
            pos = sBase[lo] + bkt * (uint32_t)kCap + slot;
          } else {
            spill = true;
            pos = atomicAdd(A.n_spill, 1u);
          }
        }
      }
      bool kept = false;
      if (valid) {
        const uint32_t ob = sOrb[lo];
        const int64_t *Fa = A.Fa + jdx;  // orbital p at Fa[p * ncore]
        const size_t m = A.ncore;
        const int64_t dh = sD[lo] + Fa[((ob >> 5) & 31u) * m] + Fa[((ob >> 15) & 31u) * m] -
                           Fa[(ob & 31u) * m] - Fa[((ob >> 10) & 31u) * m];
        write_record<EPS>(A, pos, spill, cell, sTA[lo], B, A.kind[gi] == kTilePacked,
                          pair_value<PREC>(sH[lo], A.core_c[jdx], (float)A.core_c[jdx]),
                          A.Dx[jdx] + dh, &kept);
      }
      if (EPS) my_kept += kept ? 1u : 0u;
    }
    __syncthreads();  // the next step overwrites the item arrays
  }
  if (EPS) add_survivors(A, my_kept);
}

// Per item of the batch: determinant runs (o = 0 or an alpha single) and the
// alpha-double flag.
__global__ void k_batch_counts(const uint64_t *items, uint64_t t0, uint64_t nt, int opbits,
                               uint32_t sa, uint32_t npieces, const uint32_t *grp_count,
                               uint32_t *rcnt, uint32_t *adf) {
  const uint32_t omask = (1u << opbits) - 1u;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lo = (uint32_t)items[t0 + i];
    const uint32_t k = lo >> opbits, o = lo & omask;
    rcnt[i] = o == 0 ? grp_count[k] * npieces : (o <= sa ? grp_count[k] : 0u);
    adf[i] = o > sa ? 1u : 0u;
  }
}

__global__ void k_batch_lists(const uint64_t *items, uint64_t t0, uint64_t nt, int opbits,
                              uint32_t sa, const uint32_t *grp_count, const uint32_t *rcnt,
                              const uint32_t *roff, const uint32_t *adpos, uint64_t *runs,
                              uint32_t *adl, uint32_t *adw, const uint32_t *grp_alpha, int n,
                              FastDiv dv_va, uint32_t *opinfo) {
  const uint32_t omask = (1u << opbits) - 1u;
  const uint32_t full = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  const int lane = (int)(threadIdx.x & 31u);
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // warps take 32 items at a time (warp-uniform loop); the runs of the 32
  // items are then written by the whole warp, item by item, so that an item
  // with many runs (a big group's o = 0 item, in pieces) is not one thread's
  for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < nt;
       base += nwarps * 32) {
    const uint64_t i = base + (uint64_t)lane;
    uint32_t cnt = 0, start = 0;
    if (i < nt) {
      const uint32_t lo = (uint32_t)items[t0 + i];
      const uint32_t k = lo >> opbits, o = lo & omask;
      if (o <= sa) {
        cnt = rcnt[i];
        start = roff[i];
        uint32_t oi = 0;
        if (o != 0) {
          const uint32_t Ak = grp_alpha[k];
          int ia, aa;
          dec_single(Ak, ~Ak & full, o - 1, dv_va, &ia, &aa);
          oi = (uint32_t)ia | ((uint32_t)aa << 5) | ((uint32_t)single_parity(Ak, ia, aa) << 10);
        }
        opinfo[i] = oi;
      } else {
        adl[adpos[i]] = (uint32_t)i;
        adw[adpos[i]] = grp_count[k];
      }
    }
    for (uint32_t have = __ballot_sync(0xffffffffu, cnt != 0); have; have &= have - 1) {
      const int j = __ffs(have) - 1;
      const uint32_t c = __shfl_sync(0xffffffffu, cnt, j);
      const uint32_t st = __shfl_sync(0xffffffffu, start, j);
      const uint64_t ii = base + (uint64_t)j;
      for (uint32_t m = (uint32_t)lane; m < c; m += 32) runs[(uint64_t)st + m] = (ii << 32) | m;
    }
  }
}

// Tile of each psi determinant whose alpha string is a class of the batch
// (classes are in ascending alpha order): key (tile << 32 | psi index), else
// all ones.
__global__ void k_psi_route(const uint64_t *psi_keys, size_t npsi, const uint32_t *g_alpha,
                            uint32_t gb0, uint32_t ng, const uint32_t *kind, const uint32_t *nb,
                            const uint64_t *Ws, const uint32_t *tile_base,
                            uint64_t *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npsi;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t key = psi_keys[i];
    const uint32_t a = key_alpha(key), b = (uint32_t)(key >> 32);
    uint32_t lo = 0, hi = ng;  // first class with alpha >= a
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (g_alpha[gb0 + mid] < a) lo = mid + 1; else hi = mid;
    }
    uint64_t r = ~0ull;
    if (lo < ng && g_alpha[gb0 + lo] == a) {
      const uint32_t k = kind[lo];
      uint32_t t;
      if (k == kTilePacked) t = packed_start(lo, kind, Ws) ? tile_base[lo] : tile_base[lo] - 1;
      else if (k == kTileMedium) t = tile_base[lo];
      else t = tile_base[lo] + bucket_of(b, nb[lo]);
      r = ((uint64_t)t << 32) | (uint64_t)i;
    }
    out[i] = r;
  }
}

// Tile-ordered psi keys and each tile's range of them.
__global__ void k_psi_ranges(const uint64_t *sorted, size_t npsi, const uint64_t *psi_keys,
                             uint64_t *psi_list, TileDesc *tiles) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < npsi;
       j += (size_t)gridDim.x * blockDim.x) {
    const uint64_t k = sorted[j];
    if (k == ~0ull) continue;
    const uint32_t t = (uint32_t)(k >> 32);
    psi_list[j] = psi_keys[(uint32_t)k];
    if (j == 0 || (uint32_t)(sorted[j - 1] >> 32) != t) tiles[t].psi_lo = (uint32_t)j;
    if (j + 1 == npsi || (uint32_t)(sorted[j + 1] >> 32) != t) tiles[t].psi_hi = (uint32_t)j + 1;
  }
}

// First alpha-double item of each CTA step: the last item starting at or
// before the step's first flat pair.
__global__ void k_ad_tile_items(const uint32_t *ad_off, uint32_t nad, uint32_t total,
                                uint32_t nsteps, uint32_t *tile_item) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= nsteps;
       s += gridDim.x * blockDim.x) {
    uint32_t f = s * (uint32_t)kAdTile;
    if (f >= total) f = total - 1;
    uint32_t lo = 0, hi = nad - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (ad_off[mid] <= f) lo = mid; else hi = mid - 1;
    }
    tile_item[s] = lo;
  }
}

// ---------------------------------------------------------- tile kernel ---

struct CellArgs {
  const TileDesc *tiles;
  uint32_t ntiles;     // tiles [tile0, ntiles) are visited
  uint32_t tile0;
  Stage st;
  FxInts X;          // exact diagonal of the targets that pass the screen
  int64_t E0_x;
  double inv_scale;  // 2^-s
  double tau;
  float tau_f;
  const uint64_t *psi_ht;
  uint64_t psi_mask;
  const uint64_t *psi_list;  // psi keys of the batch in tile order
  uint64_t *cand_key;
  double *cand_score;
  unsigned long long *cand_count;
  unsigned long long cand_cap;
  unsigned long long *n_unique, *n_excluded;
  unsigned *err;
  int screened;  // records may carry the eps screen's drop marker
  // exact sums left to k_long_sums (null: formed in the tile kernel): the
  // values of each list, and per list (candidate slot, offset << 16 | length)
  double *lv;
  unsigned long long *lv_count;
  unsigned long long lv_cap;
  ulonglong2 *fix;
  unsigned long long *nfix;
  unsigned long long fix_cap;
};

__device__ __forceinline__ uint64_t mix_key(uint64_t z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

// Hash of a target key within a tile: the 32-bit finalizer of MurmurHash3
// (Appleby) over the alpha word times an odd constant xor the beta word.
// Bucket tiles hold one alpha string and the betas of one bucket, so the
// finalizer's avalanche is what spreads them; cheaper than mix_key's two
// 64-bit products.  Its low bits pick the slot of the tile's hash table
// (2048 slots), its high 13 bits the bit of the tile's singleton filter.
__device__ __forceinline__ uint32_t tile_mix(uint64_t key) {
  uint32_t h = (uint32_t)key * 0x9E3779B1u ^ (uint32_t)(key >> 32);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Open addressing with linear probing; the table is at most 1/4 full, and the
// probe count is bounded by the table size (exceeding it sets *err).
__device__ __forceinline__ bool psi_contains(const uint64_t *ht, uint64_t mask, uint64_t key,
                                             unsigned *err) {
  uint64_t h = mix_key(key) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    uint64_t s = ht[h];
    if (s == key) return true;
    if (s == ~0ull) return false;
    h = (h + 1) & mask;
  }
  atomicOr(err, kErrProbe);
  return false;
}

// A tile first sorts out its singletons: every key of the tile (records and
// the psi determinants routed to it) sets its bit of a filter of kFilterBits
// bits, and a key that finds its bit set marks it in a second filter.  A
// record whose bit is not marked shares its hash with no other key of the
// tile, so it is the only contribution to its target, which is not in psi:
// it is scored and appended at once.  (About three records in four are the
// only contribution to their target; most of those are recognised so.)
// The other records are grouped by target in a shared-memory hash table: a slot
// holds the newest record of its target and each record the index of the
// previous one, so that every target ends up with the list of its records.
// The psi determinants that fall in the tile are entered first as markers, so
// a target in psi is recognised without a global lookup.  The numerator is
// then summed over each list by a rule that depends only on the multiset of
// its values, so grouping by hashing gives the result of sorting the records
// and summing the runs.  The records of the next tile are copied in
// asynchronously meanwhile.
constexpr uint32_t kEmptySlot = 0xffffffffu;
constexpr uint32_t kPsiBit = 0x80000000u;  // slot holds psi marker (index in low bits)
constexpr uint16_t kEndList = 0xffffu;
constexpr int kPsiCap = 64;                // psi markers per tile; more: global lookups

// The tile kernel comes in two sizes: tiles of kCap records (every packed,
// medium and bucket tile) and tiles of kBigCap records for the hash buckets
// that hot targets overfilled (bucket tiles only, one CTA per SM).  Per
// record: two hash slots and eight filter bits.
constexpr int kBigCap = 4096;
constexpr int kBigThreads = 1024;
// buckets of at most kMidCap records (most overfilled ones) take a middle
// size: two CTAs of kMidThreads per SM
constexpr int kMidCap = 2048;
constexpr int kMidThreads = 512;

template <int CAP>
constexpr int log2_of() {
  int b = 0;
  while ((1 << b) < CAP) ++b;
  return b;
}

template <int CAP, bool PACKED>
struct CellSmem {
  static constexpr int kTab = 2 * CAP;           // hash slots (load <= 1/2)
  static constexpr int kFilterWords = CAP / 4;   // 8 CAP filter bits
  static constexpr int kFilterShift = 32 - (log2_of<CAP>() + 3);  // top bits pick a filter bit
  StageRec rec[2][CAP];      // records (double-buffered by tile)
  uint32_t seen[kFilterWords];  // filter bits of the tile's keys (records and psi entries)
  uint32_t dup[kFilterWords];   // filter bits met twice or more
  uint32_t alpha[2][PACKED ? CAP : 1];  // record target alpha strings (packed tiles)
  uint64_t psik[2][kPsiCap]; // psi keys of the tile
  uint32_t slot[kTab];       // newest record of the slot's target, a psi marker, or empty
  uint32_t psibit[2][kTab / 32];  // slots whose key is in psi
  uint16_t next[CAP];        // previous record of the same target, or kEndList
  uint16_t targets[CAP];     // slots claimed by records, in order of claiming
  uint16_t psi_slot[kPsiCap];  // slot claimed by each psi marker, or kEndList
  uint32_t ntargets[2];      // by tile parity
  static_assert(CAP < 0xffff && kTab <= 0xffff, "indices must fit 16 bits");
  static_assert((1 << log2_of<CAP>()) == CAP, "capacity must be a power of two");
};
using TileSmem = CellSmem<kCap, true>;
using BigTileSmem = CellSmem<kBigCap, false>;
using MidTileSmem = CellSmem<kMidCap, false>;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// A tile that the kernel reduces on chip; oversized hash buckets go to the
// global path, anything else outside the limits is a planning bug.
template <int CAP>
__device__ __forceinline__ bool tile_on_chip(const TileDesc &d, uint64_t stage_cap,
                                             unsigned *err) {
  const bool fits = d.npairs <= (uint32_t)CAP && (uint64_t)d.start + d.npairs <= stage_cap;
  if (!fits && threadIdx.x == 0 &&
      !(d.kind == kTileBucket && d.npairs > (uint32_t)kCap &&
        (uint64_t)d.start + kCap <= stage_cap))
    atomicOr(err, kErrTile);
  return fits;
}

template <int CAP, bool PACKED>
__device__ __forceinline__ void prefetch_tile(CellSmem<CAP, PACKED> &S, int buf,
                                              const TileDesc &d, const CellArgs &C) {
  for (uint32_t e = threadIdx.x; e < d.npairs; e += blockDim.x) {
    cp_async16(&S.rec[buf][e], C.st.rec + d.start + e);
    if (PACKED && d.kind == kTilePacked) cp_async4(&S.alpha[buf][e], C.st.alpha + d.start + e);
  }
  const uint32_t np = d.psi_hi - d.psi_lo;
  if (np <= (uint32_t)kPsiCap)
    for (uint32_t q = threadIdx.x; q < np; q += blockDim.x)
      cp_async8(&S.psik[buf][q], C.psi_list + d.psi_lo + q);
  cp_async_commit();
}

// Target key of record e (bucket and medium tiles share one alpha string).
template <int CAP, bool PACKED>
__device__ __forceinline__ uint64_t rec_key(const CellSmem<CAP, PACKED> &S, int buf, uint32_t e,
                                            bool packed, uint32_t alpha) {
  return pack_key(PACKED && packed ? S.alpha[buf][PACKED ? e : 0] : alpha, S.rec[buf][e].beta);
}
template <int CAP, bool PACKED>
__device__ __forceinline__ uint64_t slot_key(const CellSmem<CAP, PACKED> &S, int buf, uint32_t v,
                                             bool packed, uint32_t alpha) {
  return (v & kPsiBit) ? S.psik[buf][v & ~kPsiBit] : rec_key(S, buf, v, packed, alpha);
}


// |v| as a float for the threshold bound: from the bits (no FP64 instruction),
// +inf when |v| lies above the float range so that the bound always passes.
__device__ __forceinline__ float abs_bound(double v) {
  bool ok;
  const float f = abs_as_float(v, &ok);
  return (ok || fx_exponent(v) < 1023) ? f : __int_as_float(0x7f800000);
}

// Sum of five or more values (list from e through next) in the 128-bit
// fixed-point accumulator anchored to their largest exponent: equal bit for bit
// for any order.  The first walk also sums |v| in float.  |num| <= sum |v|, so
// a target whose bound cannot reach the running threshold tau |E0 - H_ii|
// fails the screen whatever its exact numerator: *reach is cleared and the
// exact sum is skipped.  The test is conservative: a list holds at most kBigCap
// = 4096 values, so the float sum lies within 4095 * 2^-24 < 2.45e-4 below the
// exact sum of the (truncated, hence smaller) terms, which the factor 1.0003
// covers; tau_f is rounded down and den truncated, and the 0.99999 margin
// covers the float product.  Kept out of line: rare, and it would weigh on
// the common path's registers.
__device__ __noinline__ double long_numerator(const StageRec *r, const uint16_t *next,
                                              uint32_t e, float tau_f, float den, int walk_max,
                                              bool *reach, bool *deferred, unsigned long long *fix,
                                              const CellArgs &C) {
  int emax = 1, len = 0;
  float sabs = 0.0f;
  for (uint32_t i = e; i != kEndList; i = next[i]) {
    if (++len > walk_max) {  // a hot target: its warp sums it (warp_numerator)
      *deferred = true;
      return 0.0;
    }
    const int ex = fx_exponent(r[i].v);
    emax = ex > emax ? ex : emax;
    sabs += abs_bound(r[i].v);
  }
  const float df = fabsf(den);
  if (tau_f > 0.0f && df != 0.0f && !(sabs * 1.0003f >= tau_f * df * 0.99999f)) {
    *reach = false;
    return 0.0;
  }
  // The exact sum (several times the walk's cost, and one lane's work that
  // its CTA waits for at the next barrier) is left to k_long_sums when its
  // buffers have room: the values are copied out and the candidate is
  // appended with the list's entry, whose slot the caller fills in.
  if (C.lv) {
    const unsigned long long fi = atomicAdd(C.nfix, 1ull);
    const unsigned long long off = atomicAdd(C.lv_count, (unsigned long long)len);
    if (fi < C.fix_cap) {
      if (off + (unsigned long long)len <= C.lv_cap) {
        unsigned long long j = off;
        for (uint32_t i = e; i != kEndList; i = next[i]) C.lv[j++] = r[i].v;
        C.fix[fi].y = (off << 16) | (unsigned long long)len;
        *fix = fi;
        return 0.0;
      }
      C.fix[fi].y = ~0ull;  // no room for the values: the entry stays unused
    }
  }
  const int frac = fx128_frac_for(emax);
  Fx128 acc = {0, 0};
  unsigned ovf = 0;
  for (uint32_t i = e; i != kEndList; i = next[i]) {
    Fx128 x = fx128_from_double(r[i].v, frac, &ovf);
    fx128_add(acc, x);
  }
  if (ovf) atomicOr(C.err, kErrAccum);
  return fx128_to_double(acc, frac);
}

// The exact sums left by long_numerator: one thread per list, the same
// 128-bit fixed-point rule (so the same value bit for bit), written to the
// candidate's score slot before its exact score is formed.
__global__ void __launch_bounds__(256) k_long_sums(const ulonglong2 *fix,
                                                   const unsigned long long *nfix,
                                                   unsigned long long fix_cap, const double *lv,
                                                   double *cand_score, unsigned *err) {
  const unsigned long long n = *nfix < fix_cap ? *nfix : fix_cap;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const ulonglong2 f = fix[i];
    if (f.y == ~0ull) continue;
    const unsigned long long off = f.y >> 16, len = f.y & 0xffffull;
    int emax = 1;
    for (unsigned long long j = 0; j < len; ++j) {
      const int ex = fx_exponent(lv[off + j]);
      emax = ex > emax ? ex : emax;
    }
    const int frac = fx128_frac_for(emax);
    Fx128 acc = {0, 0};
    unsigned ovf = 0;
    for (unsigned long long j = 0; j < len; ++j) {
      Fx128 x = fx128_from_double(lv[off + j], frac, &ovf);
      fx128_add(acc, x);
    }
    if (ovf) atomicOr(err, kErrAccum);
    cand_score[f.x] = fx128_to_double(acc, frac);
  }
}

// The numerator of a target with more than CAP / 32 records (a hot target),
// formed by the whole warp: the lanes scan the tile's records for the key and
// sum the matching values in the same 128-bit fixed-point accumulator as
// long_numerator, then combine their partial sums (integer addition, so the
// result is the same bit for bit); the float bound of sum |v| is formed the
// same way, in another order, within the same error bound.  The records of
// the target are exactly those with its key: a key met twice or more has no
// singleton record, and screened-out records were never linked.
template <int CAP, bool PACKED>
__device__ __noinline__ double warp_numerator(const CellSmem<CAP, PACKED> &S, int buf, int nrec,
                                              bool packed, uint32_t alpha, bool screened,
                                              uint64_t key, float tau_f, float den, bool *reach,
                                              unsigned *err) {
  const int lane = (int)(threadIdx.x & 31u);
  const StageRec *r = S.rec[buf];
  int emax = 1;
  float sabs = 0.0f;
  for (int i = lane; i < nrec; i += 32)
    if (rec_key(S, buf, (uint32_t)i, packed, alpha) == key && !(screened && is_dropped(r[i].v))) {
      const int ex = fx_exponent(r[i].v);
      emax = ex > emax ? ex : emax;
      sabs += abs_bound(r[i].v);
    }
  for (int o = 16; o; o >>= 1) {
    const int em = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = em > emax ? em : emax;
    sabs += __shfl_xor_sync(0xffffffffu, sabs, o);
  }
  const float df = fabsf(den);
  if (tau_f > 0.0f && df != 0.0f && !(sabs * 1.0003f >= tau_f * df * 0.99999f)) {
    *reach = false;
    return 0.0;
  }
  const int frac = fx128_frac_for(emax);
  Fx128 acc = {0, 0};
  unsigned ovf = 0;
  for (int i = lane; i < nrec; i += 32)
    if (rec_key(S, buf, (uint32_t)i, packed, alpha) == key && !(screened && is_dropped(r[i].v))) {
      Fx128 x = fx128_from_double(r[i].v, frac, &ovf);
      fx128_add(acc, x);
    }
  for (int o = 16; o; o >>= 1) {
    Fx128 t;
    t.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
    t.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
    fx128_add(acc, t);
    ovf |= __shfl_xor_sync(0xffffffffu, ovf, o);
  }
  if (ovf && lane == 0) atomicOr(err, kErrAccum);
  *reach = true;
  return fx128_to_double(acc, frac);
}

// Exact numerator over the record list starting at e (values of screened-out
// records are never inserted); *reach is cleared when a list of five or more
// cannot reach the threshold (its sum is then not formed), and *deferred is
// set for a list longer than walk_max (left to warp_numerator).
template <int CAP, bool PACKED>
__device__ __forceinline__ double list_numerator(const CellSmem<CAP, PACKED> &S, int buf, uint32_t e,
                                                 float tau_f, int walk_max, bool *reach,
                                                 bool *deferred, unsigned long long *fix,
                                                 const CellArgs &C) {
  const StageRec *r = S.rec[buf];
  const uint32_t e2 = S.next[e];
  if (e2 == kEndList) return r[e].v;
  // two records: IEEE addition rounds their exact sum once
  const uint32_t e3 = S.next[e2];
  if (e3 == kEndList) return r[e].v + r[e2].v;
  // three or four: an order-independent FP64 sum; more: the 128-bit
  // fixed-point accumulator anchored to the largest exponent
  const uint32_t e4 = S.next[e3];
  if (e4 == kEndList) return sum4_ordered(0.0, r[e].v, r[e2].v, r[e3].v);
  if (S.next[e4] == kEndList) return sum4_ordered(r[e].v, r[e2].v, r[e3].v, r[e4].v);
  return long_numerator(r, S.next, e, tau_f, r[e].den, walk_max, reach, deferred, fix, C);
}

template <int CAP, int THREADS, bool PACKED>
__global__ void __launch_bounds__(THREADS) k_cells(CellArgs C) {
  using Smem = CellSmem<CAP, PACKED>;
  constexpr int kTab = Smem::kTab;
  constexpr int kRPT = CAP / THREADS;  // records per thread
  // hot targets (lists longer than CAP / 32) are summed by their warp in the
  // large tiles; in kCap tiles one thread walks every list
  constexpr bool kHotWarp = CAP > kCap;
  static_assert(CAP % THREADS == 0 && kRPT <= 32, "records per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int warp_base = (int)(threadIdx.x & ~31u);
  unsigned long long my_unique = 0, my_excl = 0;
  for (int i = threadIdx.x; i < kTab; i += THREADS) S.slot[i] = kEmptySlot;
  for (int i = threadIdx.x; i < kTab / 32; i += THREADS) S.psibit[0][i] = S.psibit[1][i] = 0u;
  for (int i = threadIdx.x; i < Smem::kFilterWords; i += THREADS) S.seen[i] = S.dup[i] = 0u;
  if (threadIdx.x == 0) S.ntargets[0] = S.ntargets[1] = 0;
  // tiles blockIdx.x + k * gridDim.x; descriptors are read one tile ahead of
  // the record copies, which run one tile ahead of the reduction
  uint32_t tile = C.tile0 + blockIdx.x;
  TileDesc d = {0, 0, 0, 0, 0, 0, 0, 0}, dn = {0, 0, 0, 0, 0, 0, 0, 0};
  bool on = false, on_n = false;
  if (tile < C.ntiles) {
    d = C.tiles[tile];
    on = tile_on_chip<CAP>(d, C.st.cap, C.err);
    if (on) prefetch_tile(S, 0, d, C);
  }
  if (tile + gridDim.x < C.ntiles) dn = C.tiles[tile + gridDim.x];
  int buf = 0;
#pragma unroll 1
  for (; tile < C.ntiles; tile += gridDim.x, buf ^= 1) {
    TileDesc dnn = {0, 0, 0, 0, 0, 0, 0, 0};
    if (tile + 2 * gridDim.x < C.ntiles) dnn = C.tiles[tile + 2 * gridDim.x];
    cp_async_wait_all();
    __syncthreads();  // records of this tile in place; the previous tile is done
    if (tile + gridDim.x < C.ntiles) {
      on_n = tile_on_chip<CAP>(dn, C.st.cap, C.err);
      if (on_n) prefetch_tile(S, buf ^ 1, dn, C);
    } else {
      on_n = false;
    }
    // psi bits of the previous tile are read by no one until the next barrier
    for (int i = threadIdx.x; i < kTab / 32; i += THREADS) S.psibit[buf ^ 1][i] = 0u;
    const uint32_t npsi = d.psi_hi - d.psi_lo;
    const bool psi_local = npsi <= (uint32_t)kPsiCap;
    const bool packed = PACKED && d.kind == kTilePacked;
    const int nrec = on ? (int)d.npairs : 0;
    // singleton filter: every key sets its bit; a bit met twice is marked.
    // Thread t holds records t + k THREADS (k < kRPT); their hashes stay in
    // registers for the insert phase, and the filter atomics of all of them
    // are issued before any result is used.
    uint32_t fm[kRPT], old[kRPT];
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int e = (int)threadIdx.x + k * THREADS;
      fm[k] = 0u;
      old[k] = 0u;
      if (e < nrec && !(C.screened && is_dropped(S.rec[buf][e].v))) {
        live |= 1u << k;
        fm[k] = tile_mix(rec_key(S, buf, (uint32_t)e, packed, d.alpha));
      }
    }
#pragma unroll
    for (int k = 0; k < kRPT; ++k)
      if ((live >> k) & 1u) {
        const uint32_t f = fm[k] >> Smem::kFilterShift;
        old[k] = atomicOr(&S.seen[f >> 5], 1u << (f & 31u));
      }
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const uint32_t f = fm[k] >> Smem::kFilterShift, bit = 1u << (f & 31u);
      if (((live >> k) & 1u) && (old[k] & bit)) atomicOr(&S.dup[f >> 5], bit);
    }
    if (on && psi_local)
      for (uint32_t q = threadIdx.x; q < npsi; q += THREADS) {
        const uint32_t f = tile_mix(S.psik[buf][q]) >> Smem::kFilterShift;
        const uint32_t bit = 1u << (f & 31u);
        if (atomicOr(&S.seen[f >> 5], bit) & bit) atomicOr(&S.dup[f >> 5], bit);
      }
    __syncthreads();  // filters complete
    if (on && psi_local) {
      // psi markers: claim a slot, or flag the slot a record already holds
      // (a marker whose filter bit is unmarked meets no record: left out)
      for (uint32_t q = threadIdx.x; q < npsi; q += THREADS) {
        const uint64_t key = S.psik[buf][q];
        const uint32_t mix = tile_mix(key), f = mix >> Smem::kFilterShift;
        if (!((S.dup[f >> 5] >> (f & 31u)) & 1u)) {
          S.psi_slot[q] = kEndList;
          continue;
        }
        uint32_t h = mix & (uint32_t)(kTab - 1);
        uint16_t claimed = kEndList;
        int probe = 0;
        for (; probe < kTab; ++probe) {
          uint32_t cur = S.slot[h];
          if (cur == kEmptySlot) {
            cur = atomicCAS(&S.slot[h], kEmptySlot, kPsiBit | q);
            if (cur == kEmptySlot) {
              claimed = (uint16_t)h;
              break;
            }
          }
          if (slot_key(S, buf, cur, packed, d.alpha) == key) break;
          h = (h + 1) & (kTab - 1);
        }
        if (probe == kTab) atomicOr(C.err, kErrTile);  // cannot happen at load < 3/4
        else atomicOr(&S.psibit[buf][h >> 5], 1u << (h & 31));
        S.psi_slot[q] = claimed;
      }
    }
    if (on) {
      // singletons are scored and appended at once; every other record is
      // linked into its target's list (warps append the slots they claim to
      // the target list with one shared atomic per round)
#pragma unroll
      for (int k = 0; k < kRPT; ++k) {
        const int base = k * THREADS;
        if (base + warp_base >= nrec) break;
        const int e = base + (int)threadIdx.x;
        int claimed = -1;
        bool single = false, pass1 = false;
        uint64_t key = 0;
        double v1 = 0.0;
        const uint32_t mix = fm[k];
        if ((live >> k) & 1u) {
          key = rec_key(S, buf, (uint32_t)e, packed, d.alpha);
          const uint32_t f = mix >> Smem::kFilterShift;
          single = !((S.dup[f >> 5] >> (f & 31u)) & 1u);
          if (single) {
            ++my_unique;
            if (!psi_local && psi_contains(C.psi_ht, C.psi_mask, key, C.err)) {
              ++my_excl;
            } else {
              const StageRec r = S.rec[buf][e];
              v1 = r.v;
              pass1 = true;
              if (C.tau > 0.0) {
                bool okn;
                const float nf = abs_as_float(r.v, &okn);
                const float df = fabsf(r.den);
                if (okn && df != 0.0f) pass1 = nf >= C.tau_f * df * 0.99999f;
              }
            }
          }
        }
        {  // the singletons that pass the threshold
          const unsigned bal = __ballot_sync(0xffffffffu, pass1);
          if (bal) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(C.cand_count, (unsigned long long)__popc(bal));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (pass1) {
              const unsigned long long slotc = b0 + __popc(bal & ((1u << lane) - 1u));
              if (slotc < C.cand_cap) {
                C.cand_key[slotc] = key;
                C.cand_score[slotc] = v1;  // the exact score is formed after the launch
              }
            }
          }
        }
        if (((live >> k) & 1u) && !single) {
          uint32_t h = mix & (uint32_t)(kTab - 1);
          int probe = 0;
          for (; probe < kTab; ++probe) {
            uint32_t cur = S.slot[h];
            if (cur == kEmptySlot) {
              cur = atomicCAS(&S.slot[h], kEmptySlot, (uint32_t)e);
              if (cur == kEmptySlot) {
                S.next[e] = kEndList;
                claimed = (int)h;
                break;
              }
            }
            if (slot_key(S, buf, cur, packed, d.alpha) == key) {
              const uint32_t old = atomicExch(&S.slot[h], (uint32_t)e);
              if (old & kPsiBit) {  // the first record of a psi marker's target
                S.next[e] = kEndList;
                claimed = (int)h;
              } else {
                S.next[e] = (uint16_t)old;
              }
              break;
            }
            h = (h + 1) & (kTab - 1);
          }
          if (probe == kTab) atomicOr(C.err, kErrTile);  // cannot happen at load < 3/4
        }
        const unsigned bal = __ballot_sync(0xffffffffu, claimed >= 0);
        if (bal) {
          uint32_t b0 = 0;
          if (lane == 0) b0 = atomicAdd(&S.ntargets[buf], (uint32_t)__popc(bal));
          b0 = __shfl_sync(0xffffffffu, b0, 0);
          if (claimed >= 0) S.targets[b0 + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)claimed;
        }
      }
    }
    __syncthreads();  // lists complete
    if (threadIdx.x == 0) S.ntargets[buf ^ 1] = 0;  // read by no one until the next barrier
    // the filters are read by no one until the next tile's filter phase
    for (int i = threadIdx.x; i < Smem::kFilterWords; i += THREADS) S.seen[i] = S.dup[i] = 0u;
    if (on) {
      // markers that no record joined are emptied by their inserting thread
      if (psi_local)
        for (uint32_t q = threadIdx.x; q < npsi; q += THREADS) {
          const uint32_t h = S.psi_slot[q];
          if (h != kEndList) {
            const uint32_t v = S.slot[h];
            if (v != kEmptySlot && (v & kPsiBit)) S.slot[h] = kEmptySlot;
          }
        }
      // one target per thread: numerator, exclusion, threshold; the slot is
      // emptied by its owner for the next tile
      const int ntg = (int)S.ntargets[buf];
      const float tau_f = C.tau > 0.0 ? C.tau_f : 0.0f;
#pragma unroll 1
      for (int base = 0; base + warp_base < ntg; base += THREADS) {
        const int idx = base + (int)threadIdx.x;
        bool live = false, deferred = false, reach = true;
        double num = 0.0;
        float den = 0.0f;
        uint64_t key = 0;
        unsigned long long fix = ~0ull;  // the list's k_long_sums entry, if its sum is left there
        if (idx < ntg) {
          const uint32_t h = S.targets[idx];
          const uint32_t e = S.slot[h];
          S.slot[h] = kEmptySlot;
          key = rec_key(S, buf, e, packed, d.alpha);
          ++my_unique;
          const bool in_psi = psi_local ? ((S.psibit[buf][h >> 5] >> (h & 31)) & 1u) != 0u
                                        : psi_contains(C.psi_ht, C.psi_mask, key, C.err);
          if (in_psi) {
            ++my_excl;
          } else {
            live = true;
            den = S.rec[buf][e].den;
            num = list_numerator(S, buf, e, tau_f, kHotWarp ? CAP / 32 : CAP, &reach, &deferred,
                                 &fix, C);
          }
        }
        // hot targets: each summed by the whole warp
        if (kHotWarp)
        for (unsigned m = __ballot_sync(0xffffffffu, deferred); m; m &= m - 1) {
          const int src = __ffs(m) - 1;
          bool r2 = true;
          const double n2 = warp_numerator(S, buf, nrec, packed, d.alpha, C.screened != 0,
                                           __shfl_sync(0xffffffffu, key, src), tau_f,
                                           __shfl_sync(0xffffffffu, den, src), &r2, C.err);
          if (lane == src) {
            num = n2;
            reach = r2;
          }
        }
        bool pass = false;
        if (live) {
          pass = reach;
          if (reach && C.tau > 0.0 && fix == ~0ull) {  // a deferred sum is appended untested
            bool okn;
            const float nf = abs_as_float(num, &okn);
            const float df = fabsf(den);
            if (okn && df != 0.0f) pass = nf >= C.tau_f * df * 0.99999f;  // else the exact test decides
          }
        }
        const double sc = num;  // the exact score is formed after the launch (k_exact_scores)
        const unsigned bal = __ballot_sync(0xffffffffu, pass);
        if (bal) {
          unsigned long long b0 = 0;
          if (lane == 0) b0 = atomicAdd(C.cand_count, (unsigned long long)__popc(bal));
          b0 = __shfl_sync(0xffffffffu, b0, 0);
          if (pass) {
            const unsigned long long slotc = b0 + __popc(bal & ((1u << lane) - 1u));
            if (slotc < C.cand_cap) {
              C.cand_key[slotc] = key;
              C.cand_score[slotc] = sc;
              if (fix != ~0ull) C.fix[fix].x = slotc;
            } else if (fix != ~0ull) {
              C.fix[fix].y = ~0ull;
            }
          }
        }
      }
    }
    d = dn;
    dn = dnn;
    on = on_n;
  }
  cp_async_wait_all();
  for (int dl = 16; dl; dl >>= 1) {
    my_unique += __shfl_xor_sync(0xffffffffu, my_unique, dl);
    my_excl += __shfl_xor_sync(0xffffffffu, my_excl, dl);
  }
  if (lane == 0) {
    if (my_unique) atomicAdd(C.n_unique, my_unique);
    if (my_excl) atomicAdd(C.n_excluded, my_excl);
  }
}

// ---------------------------------------------- oversized hash buckets ---
// A bucket holding more records than one tile is sorted in global memory on
// beta' and its runs are reduced one target per thread.

// Per listed oversized tile: first in-place record, in-place count, target
// alpha string, and its range of the tile-ordered spill list.
__global__ void k_tile_gather(const TileDesc *tiles, const uint32_t *list, uint32_t n,
                              const uint64_t *spill_keys, uint32_t nspill, uint32_t *info) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = list[i];
    const TileDesc d = tiles[t];
    uint32_t lo = 0, hi = nspill;  // first spill key of tile t
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((uint32_t)(spill_keys[mid] >> 32) < t) lo = mid + 1; else hi = mid;
    }
    uint32_t e = lo;
    while (e < nspill && (uint32_t)(spill_keys[e] >> 32) == t) ++e;
    info[5 * i] = d.start;
    info[5 * i + 1] = d.npairs < (uint32_t)kCap ? d.npairs : (uint32_t)kCap;
    info[5 * i + 2] = d.alpha;
    info[5 * i + 3] = lo;
    info[5 * i + 4] = e - lo;
  }
}

// Records of every oversized tile, concatenated (in-place records, then the
// tile's spilled ones): key = (tile position << 32 | beta'), payload =
// position in the concatenation; src = staging index, or spill index with the
// top bit set.
__device__ __forceinline__ const StageRec &big_rec(const StageRec *rec, const StageRec *spill,
                                                   uint64_t src) {
  return (src >> 63) ? spill[(uint32_t)src] : rec[src];
}

__global__ void k_big_gather(const StageRec *rec, const StageRec *spill,
                             const uint64_t *spill_keys, const uint32_t *start,
                             const uint32_t *nin, const uint32_t *slo, const uint32_t *off,
                             uint32_t nt, uint64_t total, uint64_t *keys, uint32_t *idx,
                             uint64_t *src) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nt - 1;  // tile holding record i
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const uint32_t o = (uint32_t)(i - off[lo]);
    const uint64_t sr = o < nin[lo]
                            ? (uint64_t)start[lo] + o
                            : ((1ull << 63) | (uint32_t)spill_keys[slo[lo] + (o - nin[lo])]);
    keys[i] = ((uint64_t)lo << 32) | big_rec(rec, spill, sr).beta;
    idx[i] = (uint32_t)i;
    src[i] = sr;
  }
}

// One CTA per oversized bucket tile of at most kBigCap records: its in-place
// records and its spilled ones (info row: start, in-place count, alpha, first
// entry of the tile-ordered spill list, spilled count) are copied into one
// range of a scratch staging buffer, and its descriptor is rewritten to point
// there (kind, alpha and psi range unchanged).
__global__ void k_big_tile_gather(const TileDesc *tiles, const uint32_t *list,
                                  const uint32_t *info, const uint32_t *off,
                                  const StageRec *rec, const StageRec *spill_rec,
                                  const uint64_t *spill_keys, StageRec *out, TileDesc *out_desc) {
  const uint32_t i = blockIdx.x;
  const uint32_t *r = info + 5 * (size_t)i;
  const uint32_t start = r[0], nin = r[1], slo = r[3], nsp = r[4], o = off[i];
  for (uint32_t e = threadIdx.x; e < nin; e += blockDim.x) out[o + e] = rec[start + e];
  for (uint32_t e = threadIdx.x; e < nsp; e += blockDim.x)
    out[o + nin + e] = spill_rec[(uint32_t)spill_keys[slo + e]];
  if (threadIdx.x == 0) {
    TileDesc d = tiles[list[i]];
    d.start = o;
    d.npairs = nin + nsp;
    out_desc[i] = d;
  }
}

// A target whose numerator is formed: its psi test, the float screen against
// tau and the append, as on chip; counts unique and excluded targets.
__device__ __forceinline__ void big_emit(double num, uint64_t full, float den, const CellArgs &C,
                                         unsigned long long *my_unique,
                                         unsigned long long *my_excl) {
  ++*my_unique;
  if (psi_contains(C.psi_ht, C.psi_mask, full, C.err)) {
    ++*my_excl;
    return;
  }
  bool pass = true;
  if (C.tau > 0.0) {  // float screen first, as on chip
    bool okn;
    const float nf = abs_as_float(num, &okn);
    const float df = fabsf(den);
    if (okn && df != 0.0f) pass = nf >= C.tau_f * df * 0.99999f;
  }
  if (pass) {  // the exact score is formed after the launch (k_exact_scores)
    const unsigned long long slot = atomicAdd(C.cand_count, 1ull);
    if (slot < C.cand_cap) {
      C.cand_key[slot] = full;
      C.cand_score[slot] = num;
    }
  }
}

// Runs (targets) longer than this go to k_big_reduce_long: a CTA per run.
constexpr uint64_t kLongRun = 64;

__global__ void k_big_reduce(const uint64_t *keys, const uint32_t *idx, const uint64_t *src,
                             uint64_t n, const uint32_t *alpha, const StageRec *spill,
                             CellArgs C, uint64_t *long_runs, unsigned *n_long) {
  unsigned long long my_unique = 0, my_excl = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sk = keys[i];
    if (i > 0 && keys[i - 1] == sk) continue;
    if (i + kLongRun < n && keys[i + kLongRun] == sk) {  // sorted: the run is long
      long_runs[atomicAdd(n_long, 1u)] = i;
      continue;
    }
    // the same rule as on chip: one or two values by IEEE addition, three or
    // four by the ordered FP64 sum, more by the 128-bit accumulator
    int emax = 1, live = 0;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint64_t e = i; e < n && keys[e] == sk; ++e) {
      const double v = big_rec(C.st.rec, spill, src[idx[e]]).v;
      if (is_dropped(v)) continue;
      const int ex = fx_exponent(v);
      emax = ex > emax ? ex : emax;
      if (live < 4) w[live] = v;
      ++live;
    }
    if (!live) continue;
    double num;
    if (live == 1) {
      num = w[0];
    } else if (live == 2) {
      num = w[0] + w[1];
    } else if (live <= 4) {
      num = sum4_ordered(w[0], w[1], w[2], w[3]);
    } else {
      const int frac = fx128_frac_for(emax);
      Fx128 acc = {0, 0};
      unsigned ovf = 0;
      for (uint64_t e = i; e < n && keys[e] == sk; ++e) {
        const double v = big_rec(C.st.rec, spill, src[idx[e]]).v;
        if (is_dropped(v)) continue;
        Fx128 x = fx128_from_double(v, frac, &ovf);
        fx128_add(acc, x);
      }
      if (ovf) atomicOr(C.err, kErrAccum);
      num = fx128_to_double(acc, frac);
    }
    const uint64_t full = pack_key(alpha[sk >> 32], (uint32_t)sk);
    big_emit(num, full, big_rec(C.st.rec, spill, src[idx[i]]).den, C, &my_unique, &my_excl);
  }
  for (int dl = 16; dl; dl >>= 1) {
    my_unique += __shfl_xor_sync(0xffffffffu, my_unique, dl);
    my_excl += __shfl_xor_sync(0xffffffffu, my_excl, dl);
  }
  if ((threadIdx.x & 31) == 0) {
    if (my_unique) atomicAdd(C.n_unique, my_unique);
    if (my_excl) atomicAdd(C.n_excluded, my_excl);
  }
}

// Long runs (hot targets with more than kLongRun records), one CTA per run:
// the run's largest exponent and live count by block reductions, then each
// thread's share in the 128-bit fixed-point accumulator anchored to that
// exponent, added exactly across the block: the same value as one thread
// walking the run (the sum is a function of the multiset).  A run with at
// most four live values (the rest dropped by the screen) takes the ordered
// FP64 rule on thread 0.
__global__ void __launch_bounds__(256) k_big_reduce_long(const uint64_t *keys, const uint32_t *idx,
                                                         const uint64_t *src, uint64_t n,
                                                         const uint32_t *alpha,
                                                         const StageRec *spill, CellArgs C,
                                                         const uint64_t *long_runs,
                                                         const unsigned *n_long) {
  __shared__ int s_emax, s_live;
  __shared__ Fx128 part[256];
  unsigned long long my_unique = 0, my_excl = 0;
  const unsigned nl = *n_long;
  for (unsigned r = blockIdx.x; r < nl; r += gridDim.x) {
    const uint64_t i = long_runs[r];
    const uint64_t sk = keys[i];
    if (threadIdx.x == 0) {
      s_emax = 1;
      s_live = 0;
    }
    __syncthreads();
    int emax = 1, live = 0;
    for (uint64_t e = i + threadIdx.x; e < n && keys[e] == sk; e += blockDim.x) {
      const double v = big_rec(C.st.rec, spill, src[idx[e]]).v;
      if (is_dropped(v)) continue;
      const int ex = fx_exponent(v);
      emax = ex > emax ? ex : emax;
      ++live;
    }
    atomicMax(&s_emax, emax);
    atomicAdd(&s_live, live);
    __syncthreads();
    const int frac = fx128_frac_for(s_emax);
    const int nlive = s_live;
    Fx128 acc = {0, 0};
    unsigned ovf = 0;
    if (nlive > 4)
      for (uint64_t e = i + threadIdx.x; e < n && keys[e] == sk; e += blockDim.x) {
        const double v = big_rec(C.st.rec, spill, src[idx[e]]).v;
        if (is_dropped(v)) continue;
        Fx128 x = fx128_from_double(v, frac, &ovf);
        fx128_add(acc, x);
      }
    if (ovf) atomicOr(C.err, kErrAccum);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st; st >>= 1) {
      if ((int)threadIdx.x < st) fx128_add(part[threadIdx.x], part[threadIdx.x + st]);
      __syncthreads();
    }
    if (threadIdx.x == 0 && nlive > 0) {
      double num;
      if (nlive > 4) {
        num = fx128_to_double(part[0], frac);
      } else {  // the rare run whose values the screen dropped: the on-chip rule
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        int k = 0;
        for (uint64_t e = i; e < n && keys[e] == sk && k < 4; ++e) {
          const double v = big_rec(C.st.rec, spill, src[idx[e]]).v;
          if (!is_dropped(v)) w[k++] = v;
        }
        num = nlive == 1 ? w[0]
              : nlive == 2 ? w[0] + w[1]
                           : sum4_ordered(w[0], w[1], w[2], w[3]);
      }
      const uint64_t full = pack_key(alpha[sk >> 32], (uint32_t)sk);
      big_emit(num, full, big_rec(C.st.rec, spill, src[idx[i]]).den, C, &my_unique, &my_excl);
    }
    __syncthreads();  // part[] and the shared counters are reused by the next run
  }
  if (threadIdx.x == 0) {
    if (my_unique) atomicAdd(C.n_unique, my_unique);
    if (my_excl) atomicAdd(C.n_excluded, my_excl);
  }
}

// Linear-probing insert; the table is at most 1/4 full, so a free slot is
// always found, and the probe count is bounded by the table size regardless
// (exceeding it sets *err).
__global__ void k_psi_insert(const uint64_t *keys, size_t n, uint64_t *ht, uint64_t mask,
                             unsigned *err) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    uint64_t h = mix_key(k) & mask;
    uint64_t probe = 0;
    for (; probe <= mask; ++probe) {
      unsigned long long prev =
          atomicCAS((unsigned long long *)&ht[h], ~0ull, (unsigned long long)k);
      if (prev == ~0ull || prev == k) break;
      h = (h + 1) & mask;
    }
    if (probe > mask) atomicOr(err, kErrProbe);
  }
}

__global__ void k_abs_min(const double *s, size_t n, unsigned long long *out) {
  // min |s| as ordered bits (non-negative doubles order like their bit patterns)
  unsigned long long m = ~0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(fabs(s[i]));
    m = b < m ? b : m;
  }
  for (int dl = 16; dl; dl >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, m, dl);
    m = o < m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

inline unsigned grid_for(size_t n, unsigned cap = 152 * 16) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace


// ------------------------------------------------------------ host side ---

int kept_count(const uint32_t *keep, const uint32_t *pos, size_t n, size_t *host_count,
               Arena &arena);

int build_fx(const double *h1, const double *eri, int n, int na, int nb, double ecore, double E0,
             Arena &arena, FxInts *out, int64_t *E0_x) {
  cudaStream_t s = arena.stream();
  double *d3;
  ASCI_TRY(arena.alloc(&d3, 3));
  k_fx_bound<<<1, 256, 0, s>>>(h1, eri, n, d3);
  ASCI_CHECK_LAUNCH();
  double h3[3];
  ASCI_TRY_CUDA(cudaMemcpyAsync(h3, d3, sizeof(h3), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  // B bounds |E0|, every diagonal element and every Fock-like diagonal value:
  // (na+nb) one-body terms, C(na,2)+C(nb,2) same-spin and na*nb opposite-spin
  // pair terms.  With s = 58 - log2(B) a sum of up to 32 such values cannot
  // overflow 64 bits.
  const double nn = (double)(na + nb), pairs_same = 0.5 * (na * (na - 1) + nb * (nb - 1));
  const double B = fabs(ecore) + fabs(E0) + nn * h3[0] + (pairs_same + n) * h3[1] +
                   ((double)na * nb + n) * h3[2] + 1.0;
  int e = 0;
  frexp(B, &e);  // B < 2^e
  int sc = 58 - e;
  if (sc > 60) sc = 60;
  if (sc < 8) {
    record_error("integrals too large for the fixed-point diagonal", __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  int64_t *hh, *jk, *jj;
  ASCI_TRY(arena.alloc(&hh, n));
  ASCI_TRY(arena.alloc(&jk, (size_t)n * n));
  ASCI_TRY(arena.alloc(&jj, (size_t)n * n));
  k_fx_tables<<<(n * n + 255) / 256, 256, 0, s>>>(h1, eri, n, sc, hh, jk, jj);
  ASCI_CHECK_LAUNCH();
  // single excitations: a sum of at most n + 1 table values stays below the
  // bound Bs, and s1 = 61 - log2(Bs) keeps it inside 64 bits
  double *d1;
  ASCI_TRY(arena.alloc(&d1, 1));
  k_fx_single_bound<<<1, 256, 0, s>>>(h1, eri, n, d1);
  ASCI_CHECK_LAUNCH();
  double bs = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&bs, d1, sizeof(bs), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  int e1 = 0;
  frexp(bs + 1e-300, &e1);
  int s1 = 61 - e1;
  if (s1 > 1000) s1 = 1000;
  const size_t n3 = (size_t)n * n * n;
  int64_t *h1x, *ssx, *sox;
  ASCI_TRY(arena.alloc(&h1x, (size_t)n * n));
  ASCI_TRY(arena.alloc(&ssx, n3));
  ASCI_TRY(arena.alloc(&sox, n3));
  k_fx_single_tables<<<(unsigned)std::min<size_t>((n3 + 255) / 256, 4096), 256, 0, s>>>(
      h1, eri, n, s1, h1x, ssx, sox);
  ASCI_CHECK_LAUNCH();
  FxInts X;
  X.n = n;
  X.s = sc;
  X.s1 = s1;
  X.h1x = h1x;
  X.ssx = ssx;
  X.sox = sox;
  X.ecore_x = llrint(ldexp(ecore, sc));
  X.hh = hh;
  X.jk = jk;
  X.jj = jj;
  *out = X;
  *E0_x = llrint(ldexp(E0, sc));
  return ASCI_OK;
}

int core_fock(const FxInts &X, const uint32_t *core_alpha, const uint32_t *core_beta, size_t m,
              int64_t *Dx, int64_t *Fa, int64_t *Fb, Arena &arena) {
  if (!m) return ASCI_OK;
  k_core_fock<<<grid_for(m), 256, 0, arena.stream()>>>(X, core_alpha, core_beta, m, Dx, Fa, Fb);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// Groups (distinct target alpha strings) of the sorted item list.  item_group
// has T + 1 entries; the group tables have G + 1 rows (row G: T and P).
int item_groups(const uint64_t *items, const uint64_t *Wexcl, uint64_t T, uint32_t *item_group,
                uint32_t **g_alpha, uint64_t **g_P0, uint64_t **g_item0, size_t *G,
                Arena &arena) {
  cudaStream_t s = arena.stream();
  ASCI_TRY(scan_item_heads(items, T, item_group, arena));
  uint32_t ng = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&ng, item_group + T, 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  ASCI_TRY(arena.alloc(g_alpha, (size_t)ng + 1));
  ASCI_TRY(arena.alloc(g_P0, (size_t)ng + 1));
  ASCI_TRY(arena.alloc(g_item0, (size_t)ng + 1));
  k_group_tab<<<grid_for(T), 256, 0, s>>>(items, item_group, Wexcl, T, *g_alpha, *g_P0, *g_item0);
  ASCI_CHECK_LAUNCH();
  *G = ng;
  return ASCI_OK;
}

int psi_hash_build(const uint64_t *psi_keys, size_t nd, uint64_t **ht, uint64_t *mask,
                   Arena &arena) {
  uint64_t size = 1024;
  while (size < 4 * (uint64_t)nd) size <<= 1;
  ASCI_TRY(arena.alloc(ht, size));
  cudaStream_t s = arena.stream();
  ASCI_TRY_CUDA(cudaMemsetAsync(*ht, 0xff, size * sizeof(uint64_t), s));
  unsigned *err, herr = 0;
  ASCI_TRY(arena.alloc(&err, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  k_psi_insert<<<grid_for(nd), 256, 0, s>>>(psi_keys, nd, *ht, size - 1, err);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    record_error("psi hash table full", __FILE__, __LINE__);
    return ASCI_ECUDA;
  }
  *mask = size - 1;
  return ASCI_OK;
}


// Stage one batch (items [t0, t1), pairs [P0, P1), groups [gb0, gb1)): plan
// its tiles, count the hash buckets of big classes and emit every record into
// the staging buffer.  The tile table is left in *tiles_out (arena memory).
// Launch of an emission kernel instantiated by (eps screen, precision).
using EmitKernel = void (*)(EmitArgs);
static unsigned emit_grid(EmitKernel k, int threads, size_t smem, size_t ntl, int cap);
static void launch_emit(EmitKernel e0, EmitKernel n0, EmitKernel e1, EmitKernel n1,
                        EmitKernel e2, EmitKernel n2, bool eps, int prec, size_t work,
                        int threads, size_t smem, int cap, cudaStream_t s, const EmitArgs &A) {
  EmitKernel k = prec == 2 ? (eps ? e2 : n2) : prec == 1 ? (eps ? e1 : n1) : (eps ? e0 : n0);
  k<<<emit_grid(k, threads, smem, work, cap), threads, smem, s>>>(A);
}

// Persistent emission grid: as many CTAs as the GPU holds at once (the
// kernel's occupancy at this block size and shared memory, at most `cap` per
// SM when cap > 0), at most `ntl`.
static unsigned emit_grid(EmitKernel k, int threads, size_t smem, size_t ntl, int cap) {
  int dev = 0, sms = 152, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  if (cap > 0 && cap < per) per = cap;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(ntl, (size_t)sms * per));
}

int fused_stage(const FusedCore &F, uint64_t t0, uint64_t t1, uint64_t P0, uint64_t P1,
                uint32_t gb0, uint32_t gb1, const Stage &st, double eps,
                unsigned long long *survivors, unsigned *err,
                void **tiles_out, size_t *ntiles_out, const uint64_t **psi_list_out,
                Spill *spill_out, std::vector<uint32_t> *oversized, Arena &arena) {
  cudaStream_t s = arena.stream();
  const uint32_t ng = gb1 - gb0;
  *psi_list_out = nullptr;
  *spill_out = Spill{nullptr, nullptr, 0};
  *ntiles_out = 0;
  oversized->clear();
  if (P1 <= P0 || ng == 0) return ASCI_OK;
  uint32_t *kind, *nb, *cellbase, *ntile, *tile_base;
  uint64_t *small_pairs, *Ws, *slots, *soff;
  ASCI_TRY(arena.alloc(&slots, ng));
  ASCI_TRY(arena.alloc(&soff, ng));
  ASCI_TRY(arena.alloc(&kind, ng));
  ASCI_TRY(arena.alloc(&nb, ng));
  ASCI_TRY(arena.alloc(&cellbase, ng));
  ASCI_TRY(arena.alloc(&ntile, ng));
  ASCI_TRY(arena.alloc(&tile_base, ng));
  ASCI_TRY(arena.alloc(&small_pairs, ng));
  ASCI_TRY(arena.alloc(&Ws, ng));
  k_group_class<<<grid_for(ng), 256, 0, s>>>(F.g_P0, gb0, gb1, P1, kind, nb, small_pairs,
                                             slots);
  ASCI_CHECK_LAUNCH();
  ASCI_TRACE("stage: classified %u groups", ng);
  ASCI_TRY(scan_exclusive_u64(slots, soff, ng, arena));
  {
    uint64_t last[2];
    ASCI_TRY_CUDA(cudaMemcpyAsync(&last[0], soff + ng - 1, 8, cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaMemcpyAsync(&last[1], slots + ng - 1, 8, cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    if (last[0] + last[1] > st.cap) {
      record_error("staging buffer too small for the batch's hash buckets (lower max_batch_pairs)",
                   __FILE__, __LINE__);
      return ASCI_ENOMEM;
    }
  }
  ASCI_TRY(scan_exclusive_u64(small_pairs, Ws, ng, arena));
  ASCI_TRY(scan_exclusive_u32(nb, cellbase, ng, arena));
  size_t ncells = 0, ntiles = 0;
  ASCI_TRY(kept_count(nb, cellbase, ng, &ncells, arena));
  k_tile_count<<<grid_for(ng), 256, 0, s>>>(ng, kind, nb, Ws, ntile);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(ntile, tile_base, ng, arena));
  ASCI_TRY(kept_count(ntile, tile_base, ng, &ntiles, arena));
  ASCI_TRACE("stage: cells=%zu tiles=%zu", ncells, ntiles);
  if (ncells > P1 - P0 || ntiles > P1 - P0) {
    record_error("inconsistent tile plan", __FILE__, __LINE__);
    return ASCI_ECUDA;
  }

  // work lists of the batch: determinant runs and alpha-double items
  const uint64_t nt = t1 - t0;
  if (nt >= (1ull << 32)) return ASCI_EINVAL;
  uint32_t *rcnt, *roff, *adf, *adpos;
  ASCI_TRY(arena.alloc(&rcnt, nt));
  ASCI_TRY(arena.alloc(&roff, nt));
  ASCI_TRY(arena.alloc(&adf, nt));
  ASCI_TRY(arena.alloc(&adpos, nt));
  const uint32_t npieces =
      (uint32_t)std::max<uint64_t>(1, ((uint64_t)F.E.sb + F.E.dbb + kPiecePairs - 1) / kPiecePairs);
  k_batch_counts<<<grid_for(nt), 256, 0, s>>>(F.items, t0, nt, F.opbits, F.E.sa, npieces,
                                              F.grp_count, rcnt, adf);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(rcnt, roff, nt, arena));
  ASCI_TRY(scan_exclusive_u32(adf, adpos, nt, arena));
  size_t nruns = 0, nad = 0;
  ASCI_TRY(kept_count(rcnt, roff, nt, &nruns, arena));
  ASCI_TRY(kept_count(adf, adpos, nt, &nad, arena));
  uint64_t *runs;
  uint32_t *adl, *adw, *ad_off, *opinfo;
  ASCI_TRY(arena.alloc(&opinfo, nt));
  ASCI_TRY(arena.alloc(&runs, nruns + 1));
  ASCI_TRY(arena.alloc(&adl, nad + 1));
  ASCI_TRY(arena.alloc(&adw, nad + 1));
  ASCI_TRY(arena.alloc(&ad_off, nad + 1));
  k_batch_lists<<<grid_for(nt), 256, 0, s>>>(F.items, t0, nt, F.opbits, F.E.sa, F.grp_count, rcnt,
                                             roff, adpos, runs, adl, adw, F.grp_alpha, F.X.n,
                                             FastDiv(F.E.va ? F.E.va : 1), opinfo);
  ASCI_CHECK_LAUNCH();
  size_t ad_total = 0;
  uint32_t ad_tiles = 0;
  uint32_t *ad_tile_item = nullptr;
  if (nad) {
    ASCI_TRY(scan_exclusive_u32(adw, ad_off, nad, arena));
    ASCI_TRY(kept_count(adw, ad_off, nad, &ad_total, arena));
    if (ad_total > P1 - P0) {
      record_error("alpha-double pairs exceed the batch", __FILE__, __LINE__);
      return ASCI_ECUDA;
    }
    ad_tiles = (uint32_t)((ad_total + kAdTile - 1) / kAdTile);
    ASCI_TRY(arena.alloc(&ad_tile_item, (size_t)ad_tiles + 1));
    k_ad_tile_items<<<grid_for((size_t)ad_tiles + 1), 256, 0, s>>>(
        ad_off, (uint32_t)nad, (uint32_t)ad_total, ad_tiles, ad_tile_item);
    ASCI_CHECK_LAUNCH();
  }
  ASCI_TRACE("stage: runs=%zu alpha-double items=%zu pairs=%zu", nruns, nad, ad_total);

  // tiles: packed and medium classes in place; each bucket of a big class owns
  // kCap slots from its class's first slot on
  TileDesc *tiles;
  unsigned *n_over, *n_spill;
  uint32_t *over_list, *cell_pos0, *cell_tile, *fill, *spill_cell;
  const uint32_t over_cap = (uint32_t)std::min<size_t>(ncells + 1, 1u << 20);
  uint32_t spill_cap = (uint32_t)std::min<uint64_t>(
      std::max<uint64_t>(1ull << 20, (P1 - P0) / 32), 1ull << 30);
  StageRec *spill_rec;
  ASCI_TRY(arena.alloc(&tiles, ntiles + 1));
  ASCI_TRY(arena.alloc(&n_over, 2));
  n_spill = n_over + 1;
  ASCI_TRY(arena.alloc(&over_list, over_cap));
  ASCI_TRY(arena.alloc(&cell_pos0, ncells + 1));
  ASCI_TRY(arena.alloc(&cell_tile, ncells + 1));
  ASCI_TRY(arena.alloc(&fill, ncells + 1));
  ASCI_TRY(arena.alloc(&spill_rec, spill_cap));
  ASCI_TRY(arena.alloc(&spill_cell, spill_cap));
  ASCI_TRY_CUDA(cudaMemsetAsync(tiles, 0, (ntiles + 1) * sizeof(TileDesc), s));
  ASCI_TRY_CUDA(cudaMemsetAsync(n_over, 0, 2 * sizeof(unsigned), s));
  ASCI_TRY_CUDA(cudaMemsetAsync(fill, 0, (ncells + 1) * sizeof(uint32_t), s));
  k_tile_write<<<grid_for(ng), 256, 0, s>>>(gb0, ng, soff, P1, F.g_P0, F.g_alpha, kind, nb, Ws,
                                            tile_base, tiles);
  ASCI_CHECK_LAUNCH();
  if (ncells) {
    k_cell_write<<<grid_for(ncells), 256, 0, s>>>(gb0, ng, (uint32_t)ncells, soff, F.g_alpha,
                                                  tile_base, cellbase, tiles, cell_pos0,
                                                  cell_tile);
    ASCI_CHECK_LAUNCH();
  }
  ASCI_TRACE("stage: tiles written");
  // psi determinants routed to their tiles (entered there as markers)
  uint64_t *psi_list = nullptr;
  if (F.npsi) {
    uint64_t *pk, *pk_alt;
    ASCI_TRY(arena.alloc(&pk, F.npsi));
    ASCI_TRY(arena.alloc(&pk_alt, F.npsi));
    ASCI_TRY(arena.alloc(&psi_list, F.npsi));
    k_psi_route<<<grid_for(F.npsi), 256, 0, s>>>(F.psi_keys, F.npsi, F.g_alpha, gb0, ng, kind, nb,
                                                 Ws, tile_base, pk);
    ASCI_CHECK_LAUNCH();
    int topbit = 1;
    while ((1ull << topbit) <= (uint64_t)ntiles) ++topbit;
    ASCI_TRY(radix_sort_u64(&pk, &pk_alt, F.npsi, 0, 32 + topbit, arena));
    k_psi_ranges<<<grid_for(F.npsi), 256, 0, s>>>(pk, F.npsi, F.psi_keys, psi_list, tiles);
    ASCI_CHECK_LAUNCH();
  }
  *psi_list_out = psi_list;

  EmitArgs A{};
  A.I = F.I;
  A.X = F.X;
  A.E = F.E;
  A.dv_va = FastDiv(F.E.va ? F.E.va : 1);
  A.dv_vb = FastDiv(F.E.vb ? F.E.vb : 1);
  A.dv_pa_p = FastDiv(F.E.pa_p ? F.E.pa_p : 1);
  A.dv_pb_p = FastDiv(F.E.pb_p ? F.E.pb_p : 1);
  A.npd0 = (uint32_t)(F.E.sb + F.E.dbb);
  A.npd1 = 1u + F.E.sb;
  A.npieces = npieces;
  A.items = F.items;
  A.Wexcl = F.Wexcl;
  A.item_group = F.item_group;
  A.t0 = t0;
  A.P0 = P0;
  A.opbits = F.opbits;
  A.grp_alpha = F.grp_alpha;
  A.grp_start = F.grp_start;
  A.grp_count = F.grp_count;
  A.core_beta = F.core_beta;
  A.core_c = F.core_c;
  A.Dx = F.Dx;
  A.Fa = F.Fa;
  A.Fb = F.Fb;
  A.gb0 = gb0;
  A.kind = kind;
  A.nb = nb;
  A.cellbase = cellbase;
  A.soff = soff;
  A.g_P0 = F.g_P0;
  A.cell_pos0 = cell_pos0;
  A.fill = fill;
  A.spill_rec = spill_rec;
  A.spill_cell = spill_cell;
  A.n_spill = n_spill;
  A.spill_cap = spill_cap;
  A.runs = runs;
  A.nruns = nruns;
  A.adl = adl;
  A.opinfo = opinfo;
  A.ad_off = ad_off;
  A.nad = (uint32_t)nad;
  A.ad_total = (uint32_t)ad_total;
  A.ad_tile_item = ad_tile_item;
  A.ad_tiles = ad_tiles;
  A.st = st;
  A.eps = eps;
  A.eps_f = (float)eps;
  A.E0_x = F.E0_x;
  A.inv_scale = ldexp(1.0, -F.X.s);
  A.survivors = survivors;
  A.ncore = F.ncore;
  A.err = err;
  const size_t emit_smem = 2 * (size_t)F.X.n * F.X.n * sizeof(int64_t);
  unsigned long long *run_next;
  ASCI_TRY(arena.alloc(&run_next, 1));
  A.run_next = run_next;
  unsigned long long surv0 = 0;
  if (eps > 0.0) {
    ASCI_TRY_CUDA(cudaMemcpyAsync(&surv0, survivors, sizeof(surv0), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  }
  unsigned hov = 0, hsp = 0;
  for (int attempt = 0;; ++attempt) {
    if (nruns) {
      ASCI_TRY_CUDA(cudaMemsetAsync(run_next, 0, sizeof(unsigned long long), s));
      launch_emit(k_emit_runs<true, 0>, k_emit_runs<false, 0>, k_emit_runs<true, 1>,
                  k_emit_runs<false, 1>, k_emit_runs<true, 2>, k_emit_runs<false, 2>, eps > 0.0,
                  F.prec, (nruns + 7) / 8, kRunThreads, emit_smem, F.ctas_per_sm, s, A);
      ASCI_CHECK_LAUNCH();
    }
    if (ad_tiles) {
      launch_emit(k_emit_ad<true, 0>, k_emit_ad<false, 0>, k_emit_ad<true, 1>,
                  k_emit_ad<false, 1>, k_emit_ad<true, 2>, k_emit_ad<false, 2>, eps > 0.0,
                  F.prec, ad_tiles, kAdThreads, 0, F.ctas_per_sm, s, A);
      ASCI_CHECK_LAUNCH();
    }
    ASCI_TRACE("stage: emission launched");
    if (ncells) {
      k_cell_finish<<<grid_for(ncells), 256, 0, s>>>((uint32_t)ncells, fill, cell_tile, tiles,
                                                     n_over, over_list, over_cap);
      ASCI_CHECK_LAUNCH();
    }
    unsigned hcnt[2] = {0, 0};
    ASCI_TRY_CUDA(cudaMemcpyAsync(hcnt, n_over, sizeof(hcnt), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    hov = hcnt[0];
    hsp = hcnt[1];
    if (hsp <= spill_cap) break;
    if (attempt > 0) {
      record_error("spill list inconsistent between emissions", __FILE__, __LINE__);
      return ASCI_ECUDA;
    }
    // Hot targets overfilled their buckets beyond the spill list.  Bucket fills
    // do not depend on the order of the atomics, so the spill count is exact:
    // size the list to it and emit the batch again.
    ASCI_TRACE("stage: %u spilled records exceed the list (%u); emitting again", hsp, spill_cap);
    spill_cap = hsp;
    ASCI_TRY(arena.alloc(&spill_rec, spill_cap));
    ASCI_TRY(arena.alloc(&spill_cell, spill_cap));
    A.spill_rec = spill_rec;
    A.spill_cell = spill_cell;
    A.spill_cap = spill_cap;
    ASCI_TRY_CUDA(cudaMemsetAsync(n_over, 0, 2 * sizeof(unsigned), s));
    ASCI_TRY_CUDA(cudaMemsetAsync(fill, 0, (ncells + 1) * sizeof(uint32_t), s));
    if (eps > 0.0)
      ASCI_TRY_CUDA(cudaMemcpyAsync(survivors, &surv0, sizeof(surv0), cudaMemcpyDefault, s));
  }
  if (hov > over_cap) {
    record_error("too many oversized hash buckets", __FILE__, __LINE__);
    return ASCI_ENOMEM;
  }
  if (hsp) {  // spilled records in tile order
    uint64_t *sk, *sk_alt;
    ASCI_TRY(arena.alloc(&sk, hsp));
    ASCI_TRY(arena.alloc(&sk_alt, hsp));
    k_spill_keys<<<grid_for(hsp), 256, 0, s>>>(spill_cell, cell_tile, hsp, sk);
    ASCI_CHECK_LAUNCH();
    int topbit = 1;
    while ((1ull << topbit) <= (uint64_t)ntiles) ++topbit;
    ASCI_TRY(radix_sort_u64(&sk, &sk_alt, hsp, 0, 32 + topbit, arena));
    *spill_out = Spill{spill_rec, sk, hsp};
  }
  ASCI_TRACE("stage: oversized buckets=%u spilled records=%u", hov, hsp);
  if (hov) {
    oversized->resize(hov);
    ASCI_TRY_CUDA(cudaMemcpyAsync(oversized->data(), over_list, hov * sizeof(uint32_t),
                                  cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    std::sort(oversized->begin(), oversized->end());
  }
  *tiles_out = tiles;
  *ntiles_out = ntiles;
  return ASCI_OK;
}

size_t tile_capacity() { return (size_t)kCap; }
size_t big_tile_capacity() { return (size_t)kBigCap; }

static CellArgs cell_args(const FusedCore &F, const Stage &st,
                          double tau, uint64_t *cand_key, double *cand_score,
                          unsigned long long *cand_count, unsigned long long cand_cap,
                          unsigned long long *n_unique, unsigned long long *n_excluded,
                          unsigned *err) {
  CellArgs CA;
  memset(&CA, 0, sizeof(CA));
  CA.st = st;
  CA.X = F.X;
  CA.E0_x = F.E0_x;
  CA.inv_scale = ldexp(1.0, -F.X.s);
  CA.tau = tau;
  CA.tau_f = (float)tau;
  if ((double)CA.tau_f > tau) CA.tau_f = nextafterf(CA.tau_f, 0.0f);
  CA.psi_ht = F.psi_ht;
  CA.psi_mask = F.psi_mask;
  CA.cand_key = cand_key;
  CA.cand_score = cand_score;
  CA.cand_count = cand_count;
  CA.cand_cap = cand_cap;
  CA.n_unique = n_unique;
  CA.n_excluded = n_excluded;
  CA.err = err;
  CA.screened = F.screened;
  return CA;
}

// Buffers of the exact sums that the tile kernels leave to k_long_sums, in a
// scratch arena that outlives the launch and the fix-up that follows it,
// sized from the launch's tiles (about seven lists of five or more records a
// tile at (24e,30o), nine records long; with no threshold, as in ASCI-PT2,
// every such list is deferred).  A list that finds no room is summed in the
// tile kernel as before.
static int enable_long_sums(CellArgs &CA, size_t ntiles, Arena &la) {
  const unsigned long long kFixCap =
      std::max<unsigned long long>(1ull << 20, (unsigned long long)ntiles * 8);
  const unsigned long long kLvCap = kFixCap * 12;
  unsigned long long *cnt;
  ASCI_TRY(la.alloc(&CA.lv, (size_t)kLvCap));
  ASCI_TRY(la.alloc(&CA.fix, (size_t)kFixCap));
  ASCI_TRY(la.alloc(&cnt, 2));
  ASCI_TRY_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), la.stream()));
  CA.lv_count = cnt;
  CA.nfix = cnt + 1;
  CA.lv_cap = kLvCap;
  CA.fix_cap = kFixCap;
  return ASCI_OK;
}

static int run_long_sums(const CellArgs &CA, int sms, cudaStream_t s) {
  k_long_sums<<<(unsigned)sms * 4, 256, 0, s>>>(CA.fix, CA.nfix, CA.fix_cap, CA.lv, CA.cand_score,
                                                 CA.err);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// Reduce tiles [tile_begin, tile_end) of a staged batch on chip and append the
// targets with |S| >= tau to the candidate buffer (at most kCap per tile).
int fused_cells(const FusedCore &F, const void *tiles, const uint64_t *psi_list,
                uint32_t tile_begin, uint32_t tile_end, const Stage &st, double tau,
                uint64_t *cand_key, double *cand_score,
                unsigned long long *cand_count, unsigned long long cand_cap,
                unsigned long long *n_unique, unsigned long long *n_excluded, unsigned *err,
                Arena &arena) {
  if (tile_end <= tile_begin) return ASCI_OK;
  cudaStream_t s = arena.stream();
  CellArgs CA = cell_args(F, st, tau, cand_key, cand_score, cand_count, cand_cap, n_unique,
                          n_excluded, err);
  CA.tiles = static_cast<const TileDesc *>(tiles);
  CA.psi_list = psi_list;
  CA.tile0 = tile_begin;
  CA.ntiles = tile_end;
  const size_t cell_smem = sizeof(TileSmem);
  // once (thread-safe static initialisation): attribute and occupancy
  static const int per_sm = [cell_smem]() {
    int p = 0;
    if (cudaFuncSetAttribute(k_cells<kCap, kCellThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cell_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &p, k_cells<kCap, kCellThreads, true>, kCellThreads, cell_smem) !=
            cudaSuccess)
      return 0;
    return p < 1 ? 1 : p;
  }();
  if (!per_sm) {
    record_error("tile kernel: cannot set its shared memory size", __FILE__, __LINE__);
    return ASCI_ECUDA;
  }
  int dev = 0, sms = 152;
  ASCI_TRY_CUDA(cudaGetDevice(&dev));
  ASCI_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per = (F.ctas_per_sm > 0 && F.ctas_per_sm < per_sm) ? F.ctas_per_sm : per_sm;
  const unsigned grid = (unsigned)std::min<size_t>((size_t)sms * per, tile_end - tile_begin);
  ASCI_TRACE("cells: launch grid=%u smem=%zu per_sm=%d", grid, cell_smem, per_sm);
  Arena la(s);
  ASCI_TRY(enable_long_sums(CA, tile_end - tile_begin, la));
  k_cells<kCap, kCellThreads, true><<<grid, kCellThreads, cell_smem, s>>>(CA);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(run_long_sums(CA, sms, s));
  return ASCI_OK;
}

// Per listed tile (start, in-place records, target alpha, first spill entry,
// spilled records): one gather kernel and one copy back.
int tile_info(const void *tiles, const std::vector<uint32_t> &list, const Spill &spill,
              std::vector<uint32_t> *info, cudaStream_t s) {
  const size_t n = list.size();
  info->assign(5 * n, 0u);
  if (!n) return ASCI_OK;
  Arena ta(s);
  uint32_t *d_list, *d_info;
  ASCI_TRY(ta.alloc(&d_list, n));
  ASCI_TRY(ta.alloc(&d_info, 5 * n));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_list, list.data(), n * 4, cudaMemcpyDefault, s));
  k_tile_gather<<<grid_for(n), 256, 0, s>>>(static_cast<const TileDesc *>(tiles), d_list,
                                            (uint32_t)n, spill.keys, spill.n, d_info);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(info->data(), d_info, 5 * n * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  return ASCI_OK;
}

// Launch the tile kernel of one size over tiles [t0, t1) of CA.tiles.
template <int CAP, int THREADS>
static int launch_big_cells(CellArgs CA, uint32_t t0, uint32_t t1, int sms, cudaStream_t s) {
  if (t1 <= t0) return ASCI_OK;
  using Smem = CellSmem<CAP, false>;
  const size_t smem = sizeof(Smem);
  static const int per_sm = [smem]() {
    int p = 0;
    if (cudaFuncSetAttribute(k_cells<CAP, THREADS, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k_cells<CAP, THREADS, false>, THREADS,
                                                      smem) != cudaSuccess)
      return 0;
    return p < 1 ? 1 : p;
  }();
  if (!per_sm) {
    record_error("large tile kernel: cannot set its shared memory size", __FILE__, __LINE__);
    return ASCI_ECUDA;
  }
  CA.tile0 = t0;
  CA.ntiles = t1;
  const unsigned grid = (unsigned)std::min<size_t>((size_t)sms * per_sm, t1 - t0);
  k_cells<CAP, THREADS, false><<<grid, THREADS, smem, s>>>(CA);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// Reduce oversized bucket tiles of at most kBigCap records on chip: list[i]
// is a tile of the batch and info[5i..5i+4] its row from tile_info.  Tiles of
// at most kMidCap records go to the middle-size kernel, the rest to the
// kBigCap one.  Appends at most as many candidates as there are records
// (*nrec_out).
int fused_big_cells(const FusedCore &F, const void *tiles, const uint64_t *psi_list,
                    const uint32_t *list_in, const uint32_t *info_in, size_t nt,
                    const Stage &st, const Spill &spill, double tau, uint64_t *cand_key,
                    double *cand_score, unsigned long long *cand_count,
                    unsigned long long cand_cap, unsigned long long *n_unique,
                    unsigned long long *n_excluded, unsigned *err, uint64_t *nrec_out,
                    Arena &arena) {
  cudaStream_t s = arena.stream();
  *nrec_out = 0;
  if (!nt) return ASCI_OK;
  // middle-size tiles first
  std::vector<uint32_t> list(nt), info(5 * nt), off(nt);
  size_t nmid = 0;
  for (size_t i = 0; i < nt; ++i) {
    const uint32_t *r = info_in + 5 * i;
    if ((uint64_t)r[1] + r[4] <= (uint64_t)kMidCap) ++nmid;
  }
  {
    size_t a = 0, b = nmid;
    for (size_t i = 0; i < nt; ++i) {
      const uint32_t *r = info_in + 5 * i;
      const size_t j = ((uint64_t)r[1] + r[4] <= (uint64_t)kMidCap) ? a++ : b++;
      list[j] = list_in[i];
      for (int w = 0; w < 5; ++w) info[5 * j + w] = r[w];
    }
  }
  uint64_t total = 0;
  for (size_t i = 0; i < nt; ++i) {
    const uint32_t *r = info.data() + 5 * i;
    const uint64_t nrec = (uint64_t)r[1] + r[4];
    if (nrec > (uint64_t)kBigCap || (uint64_t)r[0] + r[1] > st.cap ||
        (uint64_t)r[3] + r[4] > spill.n)
      return ASCI_ECUDA;
    off[i] = (uint32_t)total;
    total += nrec;
  }
  if (total >= (1ull << 32)) return ASCI_ENOMEM;
  *nrec_out = total;
  Arena ta(s);
  uint32_t *d_list, *d_info, *d_off;
  StageRec *big;
  TileDesc *desc;
  ASCI_TRY(ta.alloc(&d_list, nt));
  ASCI_TRY(ta.alloc(&d_info, 5 * nt));
  ASCI_TRY(ta.alloc(&d_off, nt));
  ASCI_TRY(ta.alloc(&big, total));
  ASCI_TRY(ta.alloc(&desc, nt));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_list, list.data(), nt * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_info, info.data(), 5 * nt * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_off, off.data(), nt * 4, cudaMemcpyDefault, s));
  k_big_tile_gather<<<(unsigned)nt, 256, 0, s>>>(static_cast<const TileDesc *>(tiles), d_list,
                                                 d_info, d_off, st.rec, spill.rec, spill.keys,
                                                 big, desc);
  ASCI_CHECK_LAUNCH();
  CellArgs CA = cell_args(F, Stage{big, nullptr, total}, tau, cand_key, cand_score, cand_count,
                          cand_cap, n_unique, n_excluded, err);
  CA.tiles = desc;
  CA.psi_list = psi_list;
  int dev = 0, sms = 152;
  ASCI_TRY_CUDA(cudaGetDevice(&dev));
  ASCI_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ASCI_TRY(enable_long_sums(CA, nt * 4, ta));
  ASCI_TRY((launch_big_cells<kMidCap, kMidThreads>(CA, 0, (uint32_t)nmid, sms, s)));
  ASCI_TRY((launch_big_cells<kBigCap, kBigThreads>(CA, (uint32_t)nmid, (uint32_t)nt, sms, s)));
  ASCI_TRY(run_long_sums(CA, sms, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));  // the host vectors above are read by copies
  return ASCI_OK;
}

// Reduce the oversized bucket tiles described by info[5i..5i+4], i in
// [0, nt), at once: their records are gathered under keys (position << 32 |
// beta'), radix-sorted in global memory and reduced one target per thread.
// Appends at most as many candidates as there are records.
int fused_big_tiles(const FusedCore &F, const uint32_t *info, size_t nt, const Stage &st,
                    const Spill &spill, double tau, uint64_t *cand_key, double *cand_score,
                    unsigned long long *cand_count, unsigned long long cand_cap,
                    unsigned long long *n_unique, unsigned long long *n_excluded, unsigned *err,
                    uint64_t *nrec_out, Arena &arena) {
  cudaStream_t s = arena.stream();
  *nrec_out = 0;
  if (!nt) return ASCI_OK;
  std::vector<uint32_t> start(nt), nin(nt), slo(nt), off(nt + 1), alpha(nt);
  uint64_t total = 0;
  for (size_t i = 0; i < nt; ++i) {
    const uint32_t *r = info + 5 * i;
    if ((uint64_t)r[0] + r[1] > st.cap || (uint64_t)r[3] + r[4] > spill.n) return ASCI_ECUDA;
    start[i] = r[0];
    nin[i] = r[1];
    alpha[i] = r[2];
    slo[i] = r[3];
    off[i] = (uint32_t)total;
    total += (uint64_t)r[1] + r[4];
  }
  if (total >= (1ull << 32)) return ASCI_ENOMEM;
  off[nt] = (uint32_t)total;
  *nrec_out = total;
  Arena ta(s);
  uint32_t *d_start, *d_nin, *d_slo, *d_off, *d_alpha, *i0, *i1;
  uint64_t *k0, *k1, *src;
  ASCI_TRY(ta.alloc(&d_start, nt));
  ASCI_TRY(ta.alloc(&d_nin, nt));
  ASCI_TRY(ta.alloc(&d_slo, nt));
  ASCI_TRY(ta.alloc(&d_off, nt + 1));
  ASCI_TRY(ta.alloc(&d_alpha, nt));
  ASCI_TRY(ta.alloc(&k0, total));
  ASCI_TRY(ta.alloc(&k1, total));
  ASCI_TRY(ta.alloc(&i0, total));
  ASCI_TRY(ta.alloc(&i1, total));
  ASCI_TRY(ta.alloc(&src, total));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_start, start.data(), nt * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_nin, nin.data(), nt * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_slo, slo.data(), nt * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_off, off.data(), (nt + 1) * 4, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(d_alpha, alpha.data(), nt * 4, cudaMemcpyDefault, s));
  k_big_gather<<<grid_for(total), 256, 0, s>>>(st.rec, spill.rec, spill.keys, d_start, d_nin,
                                               d_slo, d_off, (uint32_t)nt, total, k0, i0, src);
  ASCI_CHECK_LAUNCH();
  int topbit = 0;
  while ((1ull << topbit) < (uint64_t)nt) ++topbit;
  ASCI_TRY(radix_sort_u64_u32(&k0, &k1, &i0, &i1, total, 0, 32 + topbit, ta));
  CellArgs CA = cell_args(F, st, tau, cand_key, cand_score, cand_count, cand_cap, n_unique,
                          n_excluded, err);
  uint64_t *long_runs;
  unsigned *n_long;
  ASCI_TRY(ta.alloc(&long_runs, total / kLongRun + 1));
  ASCI_TRY(ta.alloc(&n_long, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(n_long, 0, sizeof(unsigned), s));
  k_big_reduce<<<grid_for(total), 256, 0, s>>>(k0, i0, src, total, d_alpha, spill.rec, CA,
                                               long_runs, n_long);
  ASCI_CHECK_LAUNCH();
  k_big_reduce_long<<<152 * 2, 256, 0, s>>>(k0, i0, src, total, d_alpha, spill.rec, CA,
                                            long_runs, n_long);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));  // the host vectors above are read by the copies
  return ASCI_OK;
}

namespace {


// ASCI-PT2 terms num^2 / (E0 - H_ii) of appended candidates (Alg. 1, last
// step), summed without rounding in a fixed-point grid of 2^-216 held as eight
// signed 32-bit limbs in 64-bit counters (a term of magnitude below 2^40 spans
// at most three limbs; bits below the grid are truncated).  Integer addition
// is exact and associative, so the sum does not depend on the order of the
// terms, on the batches or on the tiles: the result is a function of the set
// of targets.  Per-thread limb sums are reduced over the warp and the block,
// then added to the counters with one atomic per limb and block; a launch
// holds fewer than 2^31 terms, so no counter overflows.
constexpr int kPt2Limbs = 8;
constexpr int kPt2Grid = 216;  // the grid is 2^-216

__device__ __forceinline__ void pt2_add(double t, long long *acc, unsigned *bad) {
  if (t == 0.0) return;
  if (!(fabs(t) < 0x1p40)) {  // also catches NaN and infinities
    *bad = 1u;
    return;
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const int e = (int)((b >> 52) & 0x7ffu);
  unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  int p = (e ? e : 1) - 1075 + kPt2Grid;  // grid position of m's lowest bit
  if (p < 0) {
    if (p <= -64) return;
    m >>= -p;
    p = 0;
  }
  const int k0 = p >> 5, o = p & 31;
  const unsigned long long lo = m << o;
  const unsigned long long hi = o ? (m >> (64 - o)) : 0ull;
  const long long sg = t < 0.0 ? -1 : 1;
  const long long l0 = sg * (long long)(lo & 0xffffffffull), l1 = sg * (long long)(lo >> 32),
                  l2 = sg * (long long)(hi & 0xffffffffull);
  // selects, not indexing, so that acc stays in registers
#pragma unroll
  for (int k = 0; k < kPt2Limbs; ++k)
    acc[k] += k == k0 ? l0 : (k == k0 + 1 ? l1 : (k == k0 + 2 ? l2 : 0ll));
}

// The exact fixed-point H_ii of the 32 targets of a warp (lanes with live
// false take no part), equal bit for bit to fx_diag.  Targets of one tile
// mostly share their alpha string, so the alpha part is formed once per
// distinct alpha string of the warp (at most four; any others take fx_diag):
// D_a = sum_{p in A} h_pp + sum_{p<r in A} jk_pr by the lanes p of A, and
// J_A[q] = sum_{p in A} jj_pq by lane q; each lane then adds its beta part
// sum_{q in B} (h_qq + J_A[q]) + sum_{q<r in B} jk_qr.
__device__ __forceinline__ int64_t warp_diag(const FxInts &X, uint32_t A, uint32_t B,
                                             bool live) {
  const int n = X.n;
  const uint32_t lane = threadIdx.x & 31u;
  int64_t diag = 0;
  uint32_t pending = __ballot_sync(0xffffffffu, live);
  const int nbmax = (int)__reduce_max_sync(0xffffffffu, live ? (unsigned)__popc(B) : 0u);
  for (int round = 0; pending && round < 4; ++round) {
    const uint32_t AL = __shfl_sync(0xffffffffu, A, __ffs(pending) - 1);
    int64_t part = 0, ja = 0;
    if ((int)lane < n) {
      if ((AL >> lane) & 1u) {
        part = X.hh[lane];
        for (uint32_t r = AL & ~((2u << lane) - 1u); r; r &= r - 1)
          part += X.jk[lane * n + __ffs(r) - 1];
      }
      for (uint32_t p = AL; p; p &= p - 1) ja += X.jj[(__ffs(p) - 1) * n + lane];
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const bool mine = live && A == AL && ((pending >> lane) & 1u);
    const uint32_t group = __ballot_sync(0xffffffffu, mine);
    // each lane reads J_A[q] from lane q for the occupied beta orbitals q of
    // its own B (every round is taken by the whole warp)
    int64_t cross = 0;
    uint32_t mB = B;
    for (int it = 0; it < nbmax; ++it) {
      const bool has = mB != 0u;
      const int q = has ? __ffs(mB) - 1 : 0;
      mB &= mB - 1u;
      const int64_t t = __shfl_sync(0xffffffffu, ja, q);
      if (mine && has) cross += t;
    }
    if (mine) {
      int64_t s = X.ecore_x + part + cross;
      for (uint32_t m = B; m; m &= m - 1) {
        const int q = __ffs(m) - 1;
        s += X.hh[q];
        for (uint32_t r = m & (m - 1); r; r &= r - 1) s += X.jk[q * n + __ffs(r) - 1];
      }
      diag = s;
    }
    pending &= ~group;
  }
  if (live && ((pending >> lane) & 1u)) diag = fx_diag(X, A, B);
  return diag;
}

// Exact scores of appended candidates, which hold their numerator:
// S = num / (E0 - H_ii), with H_ii summed in fixed point (exact; warp_diag
// shares the alpha part among the warp's candidates, which come from a few
// tiles and mostly share their alpha string) and E0 - H_ii rounded once to a
// double.
__global__ void __launch_bounds__(256) k_exact_scores(const uint64_t *key, double *score, size_t n,
                                                      FxInts X, int64_t E0_x, double inv_scale) {
  // warp-uniform loop: warp_diag needs every lane
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const size_t i = base + (threadIdx.x & 31u);
    const bool live = i < n;
    const uint64_t k = live ? key[i] : 0ull;
    const int64_t dg = warp_diag(X, key_alpha(k), (uint32_t)(k >> 32), live);
    if (live) score[i] = score[i] / (__ll2double_rn(E0_x - dg) * inv_scale);
  }
}

__global__ void __launch_bounds__(256) k_pt2_terms(const uint64_t *key, const double *num,
                                                   size_t n, FxInts X, int64_t E0_x,
                                                   double inv_scale, long long *limbs,
                                                   unsigned *err) {
  __shared__ long long red[8][kPt2Limbs];
  long long acc[kPt2Limbs];
  for (int k = 0; k < kPt2Limbs; ++k) acc[k] = 0;
  unsigned bad = 0;
  // warp-uniform loop: warp_diag needs every lane
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const size_t i = base + (threadIdx.x & 31u);
    const bool live = i < n;
    const uint64_t k = live ? key[i] : 0ull;
    const int64_t dg = warp_diag(X, key_alpha(k), (uint32_t)(k >> 32), live);
    if (!live) continue;
    const double den = __ll2double_rn(E0_x - dg) * inv_scale;
    const double v = num[i];
    const double r = (fabs(den) >= 1e-30 && fabs(den) <= 1e30) ? recip_fast(den) : 1.0 / den;
    pt2_add(v * v * r, acc, &bad);
  }
  if (bad) atomicOr(err, kErrAccum);
  for (int k = 0; k < kPt2Limbs; ++k)
    for (int o = 16; o; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < kPt2Limbs; ++k) red[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < kPt2Limbs) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    if (t) atomicAdd((unsigned long long *)&limbs[threadIdx.x], (unsigned long long)t);
  }
}

// The counters as one double: the limbs in a fixed order, low to high.
__global__ void k_pt2_value(const long long *limbs, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double x = 0.0;
  for (int k = 0; k < kPt2Limbs; ++k) x += ldexp((double)limbs[k], 32 * k - kPt2Grid);
  *out = x;
}

}  // namespace

int pt2_terms(const FusedCore &F, const uint64_t *key, const double *num, size_t n,
              long long *limbs, unsigned *err, cudaStream_t s) {
  if (!n) return ASCI_OK;
  k_pt2_terms<<<grid_for(n, 152 * 8), 256, 0, s>>>(key, num, n, F.X, F.E0_x,
                                                   ldexp(1.0, -F.X.s), limbs, err);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

int pt2_value(const long long *limbs, double *out, cudaStream_t s) {
  k_pt2_value<<<1, 32, 0, s>>>(limbs, out);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

int exact_scores(const FusedCore &F, const uint64_t *key, double *score, size_t n,
                 cudaStream_t s) {
  if (!n) return ASCI_OK;
  k_exact_scores<<<grid_for(n, 152 * 32), 256, 0, s>>>(key, score, n, F.X, F.E0_x,
                                                      ldexp(1.0, -F.X.s));
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// Smallest |score| among n candidates (host result), used as the threshold.
int abs_min(const double *s, size_t n, double *host_min, Arena &arena) {
  unsigned long long *d;
  ASCI_TRY(arena.alloc(&d, 1));
  cudaStream_t st = arena.stream();
  ASCI_TRY_CUDA(cudaMemsetAsync(d, 0xff, sizeof(unsigned long long), st));
  k_abs_min<<<grid_for(n), 256, 0, st>>>(s, n, d);
  ASCI_CHECK_LAUNCH();
  unsigned long long h = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDefault, st));
  ASCI_TRY_CUDA(cudaStreamSynchronize(st));
  double v;
  memcpy(&v, &h, sizeof(v));
  *host_min = v;
  return ASCI_OK;
}

}  // namespace asci
