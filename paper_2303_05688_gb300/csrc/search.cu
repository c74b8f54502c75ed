// Host orchestration of the ASCI search and the C ABI (include/asci.h).
//
// Pipeline of one search (Algorithm 2, batched by constraints of Sec. 2.2):
//   prepare   stage inputs, validate, sort psi's keys, select the core
//             (largest |c|, ties by key), group the core by alpha string
//   plan      build the items (group, alpha operation) with their target alpha
//             strings, sort them by that string, weigh them (pairs per item),
//             and cut the item list into batches at constraint-class
//             boundaries, refining heavy classes level by level (triplets,
//             quadruplets, ... up to single alpha strings)
//   per batch generate pairs -> sort -> accumulate -> exclude psi, H_ii, score
//             -> merge into a running candidate pool (pruned to the top N)
//   select    top N of the pool (radix select on |S|, key tie-break)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "asci_internal.cuh"
#include "fused.cuh"

namespace asci {

int make_items(const ExcCounts &X, int n, const uint32_t *grp_alpha, uint32_t ngroups,
               uint32_t o_begin, uint32_t nops, int opbits, uint64_t *items,
               uint64_t *varying, Arena &arena);
int compact_u64(const uint64_t *in, const uint32_t *keep, const uint32_t *pos, size_t n,
                uint64_t *out, Arena &arena);
int compact_f64(const double *in, const uint32_t *keep, const uint32_t *pos, size_t n, double *out,
                Arena &arena);
int kept_count(const uint32_t *keep, const uint32_t *pos, size_t n, size_t *host_count,
               Arena &arena);

int build_fx(const double *h1, const double *eri, int n, int na, int nb, double ecore, double E0,
             Arena &arena, FxInts *out, int64_t *E0_x);
int core_fock(const FxInts &X, const uint32_t *core_alpha, const uint32_t *core_beta, size_t m,
              int64_t *Dx, int64_t *Fa, int64_t *Fb, Arena &arena);
int item_groups(const uint64_t *items, const uint64_t *Wexcl, uint64_t T, uint32_t *item_group,
                uint32_t **g_alpha, uint64_t **g_P0, uint64_t **g_item0, size_t *G,
                Arena &arena);
int psi_hash_build(const uint64_t *psi_keys, size_t nd, uint64_t **ht, uint64_t *mask,
                   Arena &arena);
int fused_stage(const FusedCore &F, uint64_t t0, uint64_t t1, uint64_t P0, uint64_t P1,
                uint32_t gb0, uint32_t gb1, const Stage &st, double eps,
                unsigned long long *survivors, unsigned *err,
                void **tiles_out, size_t *ntiles_out, const uint64_t **psi_list_out,
                Spill *spill_out, std::vector<uint32_t> *oversized, Arena &arena);
int tile_info(const void *tiles, const std::vector<uint32_t> &list, const Spill &spill,
              std::vector<uint32_t> *info, cudaStream_t s);
int fused_big_cells(const FusedCore &F, const void *tiles, const uint64_t *psi_list,
                    const uint32_t *list, const uint32_t *info, size_t nt, const Stage &st,
                    const Spill &spill, double tau, uint64_t *cand_key, double *cand_score,
                    unsigned long long *cand_count, unsigned long long cand_cap,
                    unsigned long long *n_unique, unsigned long long *n_excluded, unsigned *err,
                    uint64_t *nrec_out, Arena &arena);
int fused_big_tiles(const FusedCore &F, const uint32_t *info, size_t nt, const Stage &st,
                    const Spill &spill, double tau,
                    uint64_t *cand_key, double *cand_score, unsigned long long *cand_count,
                    unsigned long long cand_cap, unsigned long long *n_unique,
                    unsigned long long *n_excluded, unsigned *err, uint64_t *nrec_out,
                    Arena &arena);
int fused_cells(const FusedCore &F, const void *tiles, const uint64_t *psi_list,
                uint32_t tile_begin, uint32_t tile_end, const Stage &st, double tau,
                uint64_t *cand_key, double *cand_score,
                unsigned long long *cand_count, unsigned long long cand_cap,
                unsigned long long *n_unique, unsigned long long *n_excluded, unsigned *err,
                Arena &arena);
size_t tile_capacity();
size_t big_tile_capacity();
int exact_scores(const FusedCore &F, const uint64_t *key, double *score, size_t n,
                 cudaStream_t s);
int abs_min(const double *s, size_t n, double *host_min, Arena &arena);
int pt2_terms(const FusedCore &F, const uint64_t *key, const double *num, size_t n,
              long long *limbs, unsigned *err, cudaStream_t s);
int pt2_value(const long long *limbs, double *out, cudaStream_t s);

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Pool allocations left before an injected failure; negative: none pending.
static std::atomic<long long> g_alloc_fault{-1};

bool injected_alloc_failure() {
  if (g_alloc_fault.load(std::memory_order_relaxed) < 0) return false;
  return g_alloc_fault.fetch_sub(1, std::memory_order_relaxed) == 0;
}

bool trace_on() {
  static const bool on = [] {
    const char *v = getenv("ASCI_TRACE");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

void record_error(const char *what, const char *file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", what, file, line);
}

void clear_last_error() { g_last_error[0] = 0; }

namespace {

inline unsigned grid_for(size_t n, unsigned cap = 152 * 16) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

// ------------------------------ kernels ------------------------------------

enum : uint32_t {
  kBadRange = 1u,     // bits at or above norb
  kBadCount = 2u,     // electron counts differ from the first determinant
  kBadValue = 4u,     // non-finite coefficient or integral
  kDuplicate = 8u,    // repeated determinant
};

__global__ void k_prepare_psi(const asci_det *dets, const double *c, size_t nd, int norb, int na,
                              int nb, uint64_t *keys, uint32_t *idx, unsigned *err) {
  const uint64_t hi = ~((1ull << norb) - 1ull);  // norb <= 32
  unsigned e = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (size_t)gridDim.x * blockDim.x) {
    asci_det d = dets[i];
    if ((d.alpha & hi) || (d.beta & hi)) e |= kBadRange;
    if (na >= 0 && (__popcll(d.alpha) != na || __popcll(d.beta) != nb)) e |= kBadCount;
    if (!isfinite(c[i])) e |= kBadValue;
    keys[i] = pack_key((uint32_t)d.alpha, (uint32_t)d.beta);
    idx[i] = (uint32_t)i;
  }
  if (e) atomicOr(err, e);
}

__global__ void k_check_finite(const double *x, size_t n, unsigned *err) {
  unsigned e = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) e = kBadValue;
  if (e) atomicOr(err, e);
}

__global__ void k_check_dups(const uint64_t *sorted, size_t n, unsigned *err) {
  unsigned e = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (sorted[i] == sorted[i - 1]) e = kDuplicate;
  if (e) atomicOr(err, e);
}

// key for the core order: ~bits(|c|) ascending = |c| descending
__global__ void k_abs_keys(const uint32_t *idx, const double *c, size_t n, uint64_t *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = ~(uint64_t)__double_as_longlong(fabs(c[idx[i]]));
}

// gather the core: alpha as the sort key (low word), payload = core position
__global__ void k_gather_core(const uint32_t *core_idx, const uint64_t *psi_keys_by_input,
                              const double *c, size_t m, uint64_t *alpha_keys, uint32_t *pos,
                              uint64_t *core_keys, double *core_c) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (size_t)gridDim.x * blockDim.x) {
    uint32_t i = core_idx[j];
    uint64_t k = psi_keys_by_input[i];
    core_keys[j] = k;
    core_c[j] = c[i];
    alpha_keys[j] = (uint64_t)key_alpha(k);
    pos[j] = (uint32_t)j;
  }
}

__global__ void k_low_words(const uint64_t *in, size_t n, uint32_t *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)in[i];
}

__global__ void k_input_keys(const asci_det *dets, size_t nd, uint64_t *keys) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (size_t)gridDim.x * blockDim.x)
    keys[i] = pack_key((uint32_t)dets[i].alpha, (uint32_t)dets[i].beta);
}

// As k_input_keys for keys not validated before: a word with a bit at or
// above 32 does not fit the packed key and sets *bad.
__global__ void k_input_keys_checked(const asci_det *dets, size_t nd, uint64_t *keys,
                                     unsigned *bad) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (size_t)gridDim.x * blockDim.x) {
    const asci_det d = dets[i];
    if ((d.alpha | d.beta) >> 32) *bad = 1u;
    keys[i] = pack_key((uint32_t)d.alpha, (uint32_t)d.beta);
  }
}

// core sorted by alpha: group heads, per-det beta and coefficient in that order
__global__ void k_group_heads(const uint64_t *alpha_sorted, const uint32_t *pos,
                              const uint64_t *core_keys, const double *core_c, size_t m,
                              uint32_t *head, uint32_t *beta_sorted, double *c_sorted) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (size_t)gridDim.x * blockDim.x) {
    head[j] = (j == 0 || alpha_sorted[j] != alpha_sorted[j - 1]) ? 1u : 0u;
    uint32_t p = pos[j];
    beta_sorted[j] = key_beta(core_keys[p]);
    c_sorted[j] = core_c[p];
  }
}

__global__ void k_group_table(const uint32_t *head, const uint32_t *gid, const uint64_t *alpha_sorted,
                              size_t m, uint32_t *grp_alpha, uint32_t *grp_start) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (size_t)gridDim.x * blockDim.x)
    if (head[j]) {
      grp_alpha[gid[j]] = (uint32_t)alpha_sorted[j];
      grp_start[gid[j]] = (uint32_t)j;
    }
}

__global__ void k_group_count(const uint32_t *grp_start, uint32_t ngroups, uint32_t m,
                              uint32_t *grp_count) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
       g += gridDim.x * blockDim.x)
    grp_count[g] = ((g + 1 < ngroups) ? grp_start[g + 1] : m) - grp_start[g];
}

__device__ __forceinline__ uint32_t top_bits(uint32_t x, int L) {
  for (int drop = __popc(x) - L; drop > 0; --drop) x &= x - 1u;
  return x;
}

// class starts at level L inside target groups [s, e)
__global__ void k_class_heads(const uint32_t *g_alpha, uint64_t s, uint64_t e, int L,
                              uint32_t *head) {
  for (uint64_t g = s + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < e;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t cur = top_bits(g_alpha[g], L);
    head[g - s] = (g == s || cur != top_bits(g_alpha[g - 1], L)) ? 1u : 0u;
  }
}

// each class's first group, first item and first pair
__global__ void k_class_list(const uint32_t *head, const uint32_t *pos, uint64_t s, uint64_t cnt,
                             const uint64_t *g_item0, const uint64_t *g_P0, uint64_t *gstarts,
                             uint64_t *istarts, uint64_t *wstarts) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (head[i]) {
      gstarts[pos[i]] = s + i;
      istarts[pos[i]] = g_item0[s + i];
      wstarts[pos[i]] = g_P0[s + i];
    }
}

__global__ void k_unpack(const uint64_t *keys, size_t n, asci_det *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    asci_det d;
    d.alpha = key_alpha(keys[i]);
    d.beta = key_beta(keys[i]);
    out[i] = d;
  }
}

// ------------------------------- timing ------------------------------------

// ---------------------------------------------------------- sharding ---
// Shard of each target alpha class (Sec. 2.2, Alg. 3): light classes by a
// hash of their alpha string, heavy ones by the greedy placement on the host.

__device__ __forceinline__ uint32_t class_hash(uint32_t a) {
  uint32_t x = a * 0x9E3779B1u;
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  return x;
}

// Light classes: shard by hash, loads summed per block; heavy classes listed.
__global__ void k_class_shard(const uint32_t *g_alpha, const uint64_t *g_P0, size_t G,
                              uint64_t Pend, uint64_t heavy, int32_t W, int32_t *shard,
                              unsigned long long *light_load, uint32_t *heavy_ids,
                              unsigned *n_heavy, uint32_t heavy_cap) {
  extern __shared__ unsigned long long sload[];
  for (int i = threadIdx.x; i < W; i += blockDim.x) sload[i] = 0;
  __syncthreads();
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
       g += (size_t)gridDim.x * blockDim.x) {
    const uint64_t wg = (g + 1 < G ? g_P0[g + 1] : Pend) - g_P0[g];
    if (wg >= heavy) {
      const unsigned k = atomicAdd(n_heavy, 1u);
      if (k < heavy_cap) heavy_ids[k] = (uint32_t)g;
      shard[g] = -1;
    } else {
      const int32_t r = (int32_t)(class_hash(g_alpha[g]) % (uint32_t)W);
      shard[g] = r;
      atomicAdd(&sload[r], (unsigned long long)wg);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < W; i += blockDim.x)
    if (sload[i]) atomicAdd(&light_load[i], sload[i]);
}

__global__ void k_heavy_set(const uint32_t *ids, const int32_t *sh, uint32_t n, int32_t *shard) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    shard[ids[i]] = sh[i];
}

__global__ void k_keep_items(const uint32_t *item_group, const int32_t *shard, uint64_t T,
                             int32_t r, uint32_t *keep) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (uint64_t)gridDim.x * blockDim.x)
    keep[t] = shard[item_group[t]] == r ? 1u : 0u;
}

__global__ void k_compact_items(const uint64_t *in, const uint32_t *keep, const uint32_t *pos,
                                uint64_t T, uint64_t *out) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (uint64_t)gridDim.x * blockDim.x)
    if (keep[t]) out[pos[t]] = in[t];
}

// Keep the items of shard r's classes: *items (sorted by target alpha, T
// entries, weights summing to P with exclusive prefix Wexcl) is compacted in
// place into *T_out entries.
int shard_items(uint64_t **items, uint64_t **items_alt, const uint64_t *Wexcl, uint64_t T,
                uint64_t P, int32_t r, int32_t W, uint64_t *T_out, Arena &arena) {
  cudaStream_t s = arena.stream();
  Arena sa(s);
  uint32_t *item_group, *g_alpha;
  uint64_t *g_P0, *g_item0;
  size_t G = 0;
  ASCI_TRY(sa.alloc(&item_group, T + 1));
  ASCI_TRY(item_groups(*items, Wexcl, T, item_group, &g_alpha, &g_P0, &g_item0, &G, sa));
  const uint64_t heavy = std::max<uint64_t>(1, P / (64ull * (uint64_t)W));
  const uint32_t heavy_cap = (uint32_t)std::min<uint64_t>(G, 64ull * W + 1);
  int32_t *shard;
  unsigned long long *light;
  uint32_t *heavy_ids;
  unsigned *n_heavy;
  ASCI_TRY(sa.alloc(&shard, G));
  ASCI_TRY(sa.alloc(&light, (size_t)W));
  ASCI_TRY(sa.alloc(&heavy_ids, heavy_cap));
  ASCI_TRY(sa.alloc(&n_heavy, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(light, 0, (size_t)W * sizeof(unsigned long long), s));
  ASCI_TRY_CUDA(cudaMemsetAsync(n_heavy, 0, sizeof(unsigned), s));
  k_class_shard<<<grid_for(G), 256, (size_t)W * sizeof(unsigned long long), s>>>(
      g_alpha, g_P0, G, P, heavy, W, shard, light, heavy_ids, n_heavy, heavy_cap);
  ASCI_CHECK_LAUNCH();
  unsigned nh = 0;
  std::vector<uint64_t> loads((size_t)W);
  ASCI_TRY_CUDA(cudaMemcpyAsync(&nh, n_heavy, sizeof(nh), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(loads.data(), light, (size_t)W * 8, cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (nh > heavy_cap) return ASCI_ECUDA;  // at most 64 W classes reach the threshold
  if (nh) {
    std::vector<uint32_t> ids(nh);
    std::vector<uint64_t> p0(nh), p1(nh), wts(nh);
    ASCI_TRY_CUDA(cudaMemcpyAsync(ids.data(), heavy_ids, nh * 4, cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    std::sort(ids.begin(), ids.end());  // placement independent of the listing order
    for (unsigned i = 0; i < nh; ++i) {
      ASCI_TRY_CUDA(cudaMemcpyAsync(&p0[i], g_P0 + ids[i], 8, cudaMemcpyDefault, s));
      if (ids[i] + 1 < G)
        ASCI_TRY_CUDA(cudaMemcpyAsync(&p1[i], g_P0 + ids[i] + 1, 8, cudaMemcpyDefault, s));
      else
        p1[i] = P;
    }
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    for (unsigned i = 0; i < nh; ++i) wts[i] = p1[i] - p0[i];
    std::vector<int32_t> sh(nh);
    ASCI_TRY(asci_shard_assign(wts.data(), nh, W, loads.data(), sh.data()));
    uint32_t *d_ids;
    int32_t *d_sh;
    ASCI_TRY(sa.alloc(&d_ids, nh));
    ASCI_TRY(sa.alloc(&d_sh, nh));
    ASCI_TRY_CUDA(cudaMemcpyAsync(d_ids, ids.data(), nh * 4, cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaMemcpyAsync(d_sh, sh.data(), nh * 4, cudaMemcpyDefault, s));
    k_heavy_set<<<grid_for(nh), 256, 0, s>>>(d_ids, d_sh, nh, shard);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));  // the host vectors above are read by the copies
  }
  uint32_t *keep, *pos;
  ASCI_TRY(sa.alloc(&keep, T));
  ASCI_TRY(sa.alloc(&pos, T));
  k_keep_items<<<grid_for(T), 256, 0, s>>>(item_group, shard, T, r, keep);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(keep, pos, T, sa));
  size_t kept = 0;
  ASCI_TRY(kept_count(keep, pos, T, &kept, sa));
  k_compact_items<<<grid_for(T), 256, 0, s>>>(*items, keep, pos, T, *items_alt);
  ASCI_CHECK_LAUNCH();
  std::swap(*items, *items_alt);
  *T_out = kept;
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  return ASCI_OK;
}


int bits_for(uint32_t v) {
  int b = 0;
  while ((1ull << b) < (uint64_t)v) ++b;
  return b < 1 ? 1 : b;
}

struct Batch {
  uint64_t t0, t1, P0, P1;
};

// Cut items [0, T) into batches of at most bmax pairs at class boundaries
// (Sec. 2.2 constraints; Alg. 3's work counts h are the class weights).  A
// class is a set of target alpha strings, so the classes are found on the
// table of distinct target strings (groups; row G holds T and P).
class Planner {
 public:
  Planner(const uint32_t *g_alpha, const uint64_t *g_item0, const uint64_t *g_P0, uint64_t G,
          uint64_t bmax, uint64_t first_cap, int lmax, Arena &arena)
      : ga_(g_alpha), gi_(g_item0), gp_(g_P0), G_(G), bmax_(bmax), first_cap_(first_cap),
        lmax_(lmax), arena_(arena) {}

  // The pairs of each class of level L, in constraint order.
  int class_weights(int L, std::vector<uint64_t> *w) {
    std::vector<uint64_t> gst, ist, wst;
    ASCI_TRY(query(0, G_, L, &gst, &ist, &wst));
    uint64_t P = 0;
    ASCI_TRY_CUDA(cudaMemcpyAsync(&P, gp_ + G_, 8, cudaMemcpyDefault, arena_.stream()));
    ASCI_TRY_CUDA(cudaStreamSynchronize(arena_.stream()));
    w->resize(wst.size());
    for (size_t i = 0; i < wst.size(); ++i) (*w)[i] = (i + 1 < wst.size() ? wst[i + 1] : P) - wst[i];
    return ASCI_OK;
  }

  int run(uint64_t T, uint64_t P, int L0, std::vector<Batch> *out, int *max_level) {
    batches_.clear();
    cur_open_ = false;
    max_level_ = L0;
    ASCI_TRY(visit(0, G_, T, P, L0));
    flush();
    *out = batches_;
    *max_level = max_level_;
    return ASCI_OK;
  }

 private:
  int query(uint64_t s, uint64_t e, int L, std::vector<uint64_t> *gst, std::vector<uint64_t> *ist,
            std::vector<uint64_t> *wst) {
    uint64_t cnt = e - s;
    Arena qa(arena_.stream());  // released when the query returns
    uint32_t *head, *pos;
    ASCI_TRY(qa.alloc(&head, cnt));
    ASCI_TRY(qa.alloc(&pos, cnt));
    cudaStream_t st = qa.stream();
    k_class_heads<<<grid_for(cnt), 256, 0, st>>>(ga_, s, e, L, head);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY(scan_exclusive_u32(head, pos, cnt, qa));
    size_t nc = 0;
    ASCI_TRY(kept_count(head, pos, cnt, &nc, qa));
    uint64_t *dg, *di, *dw;
    ASCI_TRY(qa.alloc(&dg, nc));
    ASCI_TRY(qa.alloc(&di, nc));
    ASCI_TRY(qa.alloc(&dw, nc));
    k_class_list<<<grid_for(cnt), 256, 0, st>>>(head, pos, s, cnt, gi_, gp_, dg, di, dw);
    ASCI_CHECK_LAUNCH();
    gst->resize(nc);
    ist->resize(nc);
    wst->resize(nc);
    ASCI_TRY_CUDA(cudaMemcpyAsync(gst->data(), dg, nc * 8, cudaMemcpyDefault, st));
    ASCI_TRY_CUDA(cudaMemcpyAsync(ist->data(), di, nc * 8, cudaMemcpyDefault, st));
    ASCI_TRY_CUDA(cudaMemcpyAsync(wst->data(), dw, nc * 8, cudaMemcpyDefault, st));
    ASCI_TRY_CUDA(cudaStreamSynchronize(st));
    return ASCI_OK;
  }

  void flush() {
    if (cur_open_ && cur_.P1 > cur_.P0) batches_.push_back(cur_);
    cur_open_ = false;
  }

  void add(uint64_t cs, uint64_t ce, uint64_t ws, uint64_t we) {
    const uint64_t cap = batches_.empty() ? first_cap_ : bmax_;
    if (cur_open_ && (we - cur_.P0) > cap) flush();
    if (!cur_open_) {
      cur_ = Batch{cs, ce, ws, we};
      cur_open_ = true;
    } else {
      cur_.t1 = ce;
      cur_.P1 = we;
    }
  }

  // groups [gs, ge), whose items end at ie and pairs at we, split at level L
  int visit(uint64_t gs, uint64_t ge, uint64_t ie, uint64_t we, int L) {
    if (L > max_level_) max_level_ = L;
    std::vector<uint64_t> gst, ist, wst;
    ASCI_TRY(query(gs, ge, L, &gst, &ist, &wst));
    for (size_t c = 0; c < gst.size(); ++c) {
      const bool last = c + 1 == gst.size();
      const uint64_t g0 = gst[c], g1 = last ? ge : gst[c + 1];
      const uint64_t i0 = ist[c], i1 = last ? ie : ist[c + 1];
      const uint64_t w0 = wst[c], w1 = last ? we : wst[c + 1];
      if (w1 - w0 > bmax_ && L < lmax_ && g1 - g0 > 1) {
        flush();
        ASCI_TRY(visit(g0, g1, i1, w1, L + 1));
      } else {
        add(i0, i1, w0, w1);
      }
    }
    return ASCI_OK;
  }

  const uint32_t *ga_;
  const uint64_t *gi_;
  const uint64_t *gp_;
  uint64_t G_;
  uint64_t bmax_;
  uint64_t first_cap_;
  int lmax_;
  Arena &arena_;
  std::vector<Batch> batches_;
  Batch cur_{};
  bool cur_open_ = false;
  int max_level_ = 0;
};

}  // namespace

// Per-device memory pool that keeps the search scratch cached between calls.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

int device_pool(int dev, cudaMemPool_t *pool) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 64) return ASCI_ECUDA;
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    ASCI_TRY_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
    uint64_t thr = ~0ull;
    ASCI_TRY_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
  }
  *pool = g_pools[dev];
  return ASCI_OK;
}

// A request for the pair counts of the constraint classes of one level
// (asci_constraint_classes): the search stops once its items are weighed.
struct ClassQuery {
  int level;
  uint64_t *out;     // host or device, capacity entries
  size_t capacity;
  size_t n;          // classes found
};

// The search proper.  All pointers resolved; `arena` owns the scratch.
// With pt2_out set, the same pipeline runs without a threshold and, instead
// of keeping candidates, folds every unique target outside psi into the
// ASCI-PT2 sum num^2 / (E0 - H_ii) (N must be 0).
static int search_impl(const asci_det *dets_in, const double *coeffs_in, size_t nd, double E0,
                       const asci_ints *ints, size_t C, size_t N, const asci_opts &o,
                       asci_det *out_dets, double *out_scores, size_t *out_n, asci_stats *st,
                       cudaStream_t stream, double *pt2_out = nullptr,
                       ClassQuery *cq = nullptr) {
  Arena arena(stream);
  double tl[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // per-stage device milliseconds
  uint64_t tile_launches = 0, staged_records = 0, oversized_records = 0, big_records = 0;
  StageTimer tm(stream), total_tm(stream), ktm(stream);
  total_tm.start();
  tm.start();
  const int n = ints->norb;
  const asci_det *dets;
  const double *coeffs, *h1, *eri;
  ASCI_TRY(to_device(dets_in, nd, &dets, arena));
  ASCI_TRY(to_device(coeffs_in, nd, &coeffs, arena));
  ASCI_TRY(to_device(ints->h1, (size_t)n * n, &h1, arena));
  ASCI_TRY(to_device(ints->eri, (size_t)n * n * n * n, &eri, arena));

  ASCI_TRACE("search: ndets=%zu norb=%d C=%zu N=%zu eps=%g", nd, n, C, N, o.eps_search);
  // electron counts from the first determinant
  asci_det d0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&d0, dets, sizeof(d0), cudaMemcpyDefault, stream));
  ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
  const int na = __builtin_popcountll(d0.alpha), nb = __builtin_popcountll(d0.beta);
  if (na > n || nb > n) return ASCI_EINVAL;

  unsigned *derr;
  ASCI_TRY(arena.alloc(&derr, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(derr, 0, sizeof(unsigned), stream));
  uint64_t *pkeys, *pkeys_alt, *absk, *absk_alt;
  uint32_t *pidx, *pidx_alt;
  ASCI_TRY(arena.alloc(&pkeys, nd));
  ASCI_TRY(arena.alloc(&pkeys_alt, nd));
  ASCI_TRY(arena.alloc(&pidx, nd));
  ASCI_TRY(arena.alloc(&pidx_alt, nd));
  k_prepare_psi<<<grid_for(nd), 256, 0, stream>>>(dets, coeffs, nd, n, na, nb, pkeys, pidx, derr);
  ASCI_CHECK_LAUNCH();
  k_check_finite<<<grid_for((size_t)n * n * n * n), 256, 0, stream>>>(eri, (size_t)n * n * n * n,
                                                                       derr);
  ASCI_CHECK_LAUNCH();
  k_check_finite<<<grid_for((size_t)n * n), 256, 0, stream>>>(h1, (size_t)n * n, derr);
  ASCI_CHECK_LAUNCH();
  // psi keys sorted (exclusion table) with input positions
  ASCI_TRY(radix_sort_u64_u32(&pkeys, &pkeys_alt, &pidx, &pidx_alt, nd, 0, 64, arena));
  k_check_dups<<<grid_for(nd), 256, 0, stream>>>(pkeys, nd, derr);
  ASCI_CHECK_LAUNCH();
  unsigned herr = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDefault, stream));
  ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
  if (herr) {
    record_error(herr & kDuplicate   ? "duplicate determinants in psi"
                 : herr & kBadCount  ? "determinants with different electron counts"
                 : herr & kBadRange  ? "determinant bits at or above norb"
                                     : "non-finite coefficient or integral",
                 __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  const uint64_t *psi_sorted = pkeys;
  // the psi key buffer stays live; reuse the alternates for the core order
  ASCI_TRY(arena.alloc(&absk, nd));
  ASCI_TRY(arena.alloc(&absk_alt, nd));
  k_abs_keys<<<grid_for(nd), 256, 0, stream>>>(pidx, coeffs, nd, absk);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(radix_sort_u64_u32(&absk, &absk_alt, &pidx, &pidx_alt, nd, 0, 64, arena));
  const size_t m = std::min(C, nd);
  // keys of psi by input position (for gathering the core)
  uint64_t *in_keys;
  ASCI_TRY(arena.alloc(&in_keys, nd));
  k_input_keys<<<grid_for(nd), 256, 0, stream>>>(dets, nd, in_keys);
  ASCI_CHECK_LAUNCH();
  uint64_t *core_keys, *alpha_k, *alpha_k_alt;
  double *core_c;
  uint32_t *cpos, *cpos_alt;
  ASCI_TRY(arena.alloc(&core_keys, m));
  ASCI_TRY(arena.alloc(&core_c, m));
  ASCI_TRY(arena.alloc(&alpha_k, m));
  ASCI_TRY(arena.alloc(&alpha_k_alt, m));
  ASCI_TRY(arena.alloc(&cpos, m));
  ASCI_TRY(arena.alloc(&cpos_alt, m));
  k_gather_core<<<grid_for(m), 256, 0, stream>>>(pidx, in_keys, coeffs, m, alpha_k, cpos, core_keys,
                                                 core_c);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(radix_sort_u64_u32(&alpha_k, &alpha_k_alt, &cpos, &cpos_alt, m, 0, 32, arena));
  uint32_t *ghead, *gid, *core_beta;
  double *core_c_sorted;
  ASCI_TRY(arena.alloc(&ghead, m));
  ASCI_TRY(arena.alloc(&gid, m));
  ASCI_TRY(arena.alloc(&core_beta, m));
  ASCI_TRY(arena.alloc(&core_c_sorted, m));
  k_group_heads<<<grid_for(m), 256, 0, stream>>>(alpha_k, cpos, core_keys, core_c, m, ghead,
                                                 core_beta, core_c_sorted);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(ghead, gid, m, arena));
  size_t ngroups = 0;
  ASCI_TRY(kept_count(ghead, gid, m, &ngroups, arena));
  uint32_t *grp_alpha, *grp_start, *grp_count;
  ASCI_TRY(arena.alloc(&grp_alpha, ngroups));
  ASCI_TRY(arena.alloc(&grp_start, ngroups));
  ASCI_TRY(arena.alloc(&grp_count, ngroups));
  k_group_table<<<grid_for(m), 256, 0, stream>>>(ghead, gid, alpha_k, m, grp_alpha, grp_start);
  ASCI_CHECK_LAUNCH();
  k_group_count<<<grid_for(ngroups), 256, 0, stream>>>(grp_start, (uint32_t)ngroups, (uint32_t)m,
                                                       grp_count);
  ASCI_CHECK_LAUNCH();

  ASCI_TRACE("prepared: core=%zu groups=%zu", m, ngroups);
  DevInts I;
  ASCI_TRY(build_tables(h1, eri, n, na, nb, ints->ecore, o.precision != ASCI_FP64, arena, &I));
  const ExcCounts X = exc_counts(n, na, nb);
  if (st) {
    st->ncore = m;
    st->generated = (uint64_t)m * X.total;
  }
  tm.stop(&tl[0]);

  // ------------------------------- plan ------------------------------------
  tm.start();
  const uint64_t npd0 = (uint64_t)X.sb + X.dbb;
  const uint32_t nops = 1u + X.sa + (uint32_t)X.daa;
  const uint32_t o_begin = npd0 > 0 ? 0u : 1u;
  const int opbits = bits_for(nops);
  if (opbits >= 32 || (uint64_t)ngroups >= (1ull << (32 - opbits))) {
    record_error("too many distinct core alpha strings for the item format", __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  // pairs of one item must index in 32 bits
  {
    uint32_t maxc = 0;
    // conservative bound: the whole core in one group
    maxc = (uint32_t)m;
    if ((uint64_t)maxc * std::max<uint64_t>(npd0, 1ull + X.sb) >= (1ull << 32)) {
      record_error("core too large for one alpha group", __FILE__, __LINE__);
      return ASCI_EINVAL;
    }
  }
  uint64_t T = (uint64_t)ngroups * (nops - o_begin);
  const int32_t W = o.shard_count > 1 ? o.shard_count : 1;
  std::vector<Batch> batches;
  int max_level = 0;
  uint64_t *items = nullptr, *items_alt = nullptr, *Wexcl = nullptr;
  uint64_t P = 0;
  if (T > 0) {
    ASCI_TRY(arena.alloc(&items, T));
    ASCI_TRY(arena.alloc(&items_alt, T));
    uint64_t varying = 0;  // bits in which the target strings differ
    ASCI_TRY(make_items(X, n, grp_alpha, (uint32_t)ngroups, o_begin, nops, opbits, items, &varying,
                        arena));
    ASCI_TRY(radix_sort_u64_varying(&items, &items_alt, T, 32, 32 + n, varying, arena));
    ASCI_TRY(arena.alloc(&Wexcl, T + 1));
    ASCI_TRY(scan_item_weights(items, T, opbits, grp_count, X, Wexcl, arena));
    ASCI_TRY_CUDA(cudaMemcpyAsync(&P, Wexcl + T, 8, cudaMemcpyDefault, stream));
    ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
    if (P != (uint64_t)m * X.total) {
      record_error("pair count does not match the closed form", __FILE__, __LINE__);
      return ASCI_ECUDA;
    }
    if (W > 1) {  // this shard's classes only
      uint64_t T1 = 0;
      ASCI_TRY(shard_items(&items, &items_alt, Wexcl, T, P, o.shard_index, W, &T1, arena));
      ASCI_TRACE("shard %d of %d: items %llu of %llu", o.shard_index, W,
                 (unsigned long long)T1, (unsigned long long)T);
      T = T1;
      P = 0;
      if (T) {
        ASCI_TRY(scan_item_weights(items, T, opbits, grp_count, X, Wexcl, arena));
        ASCI_TRY_CUDA(cudaMemcpyAsync(&P, Wexcl + T, 8, cudaMemcpyDefault, stream));
        ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
      }
    }
  }
  // the distinct target alpha strings (groups) of the items
  uint32_t *item_group = nullptr;
  uint32_t *g_alpha = nullptr;
  uint64_t *g_P0 = nullptr, *g_item0 = nullptr;
  size_t G = 0;
  if (T > 0) {
    ASCI_TRY(arena.alloc(&item_group, T + 1));
    ASCI_TRY(item_groups(items, Wexcl, T, item_group, &g_alpha, &g_P0, &g_item0, &G, arena));
  }
  if (cq) {  // the classes of one level, in constraint order, and their pairs
    cq->n = 0;
    if (T > 0 && P > 0) {
      Planner pl(g_alpha, g_item0, g_P0, G, P, P, na, arena);
      std::vector<uint64_t> w;
      ASCI_TRY(pl.class_weights(std::min(cq->level, na), &w));
      cq->n = w.size();
      if (cq->capacity >= cq->n && cq->n) {
        ASCI_TRY_CUDA(cudaMemcpyAsync(cq->out, w.data(), cq->n * 8, cudaMemcpyDefault, stream));
        ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
      }
    }
    if (st) st->generated = P;
    return ASCI_OK;
  }
  if (T > 0 && P > 0) {
    uint64_t bmax = o.max_batch_pairs;
    if (bmax == 0) {
      size_t fr = 0, tot = 0;
      ASCI_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
      bmax = (uint64_t)(fr / 2) / 40;  // staging: 1.5 slots of 20 bytes per pair
      bmax = std::max<uint64_t>(bmax, 1ull << 20);
      bmax = std::min<uint64_t>(bmax, 1ull << 31);
    }
    const int lmax = (o.max_constraint_level > 0) ? std::min(o.max_constraint_level, na) : na;
    const int L0 = std::min(3, lmax);
    // a small first batch fixes the selection threshold early
    const uint64_t first_cap = std::min<uint64_t>(bmax, std::max<uint64_t>(1ull << 22, P / 64));
    Planner planner(g_alpha, g_item0, g_P0, G, bmax, first_cap, lmax, arena);
    ASCI_TRY(planner.run(T, P, L0, &batches, &max_level));
  }
  uint64_t bcap = 0;
  for (auto &b : batches) bcap = std::max(bcap, b.P1 - b.P0);
  if (st) st->generated = P;  // C n_exc, or this shard's part of it
  ASCI_TRACE("planned: items=%llu pairs=%llu batches=%zu max_batch=%llu level=%d",
             (unsigned long long)T, (unsigned long long)P, batches.size(),
             (unsigned long long)bcap, max_level);
  if (st) {
    st->batches = batches.size();
    st->max_batch = bcap;
    st->max_level = (uint64_t)max_level;
  }
  if (bcap >= (1ull << 32) - 1) {
    record_error("a constraint batch exceeds 2^32 pairs", __FILE__, __LINE__);
    return ASCI_ENOMEM;
  }
  tm.stop(&tl[1]);

  // --------------------------- batches -------------------------------------
  // per-search tables of the constraint-tile kernels
  tm.start();
  FusedCore F;
  F.I = I;
  F.E = X;
  F.items = items;
  F.Wexcl = Wexcl;
  F.opbits = opbits;
  F.grp_alpha = grp_alpha;
  F.grp_start = grp_start;
  F.grp_count = grp_count;
  F.core_beta = core_beta;
  F.core_c = core_c_sorted;
  uint64_t *psi_ht = nullptr;
  uint64_t psi_mask = 0;
  ASCI_TRY(psi_hash_build(psi_sorted, nd, &psi_ht, &psi_mask, arena));
  F.psi_ht = psi_ht;
  F.psi_keys = psi_sorted;
  F.npsi = nd;
  F.psi_mask = psi_mask;
  F.ncore = (uint32_t)m;
  F.prec = o.precision == ASCI_FP32_INT_COMP_ACC ? 2 : (o.precision == ASCI_FP32_INT_FP64_ACC ? 1 : 0);
  F.screened = o.eps_search > 0.0 ? 1 : 0;
  F.ctas_per_sm = o.ctas_per_sm;
  ASCI_TRY(build_fx(h1, eri, n, na, nb, ints->ecore, E0, arena, &F.X, &F.E0_x));
  if (st) st->diag_grid_bits = (uint64_t)F.X.s;
  {
    uint32_t *core_alpha32;
    int64_t *Dx, *Fa, *Fb;
    ASCI_TRY(arena.alloc(&core_alpha32, m));
    ASCI_TRY(arena.alloc(&Dx, m));
    ASCI_TRY(arena.alloc(&Fa, m * n));
    ASCI_TRY(arena.alloc(&Fb, m * n));
    k_low_words<<<grid_for(m), 256, 0, stream>>>(alpha_k, m, core_alpha32);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY(core_fock(F.X, core_alpha32, core_beta, m, Dx, Fa, Fb, arena));
    F.Dx = Dx;
    F.Fa = Fa;
    F.Fb = Fb;
  }
  F.item_group = item_group;
  F.g_alpha = g_alpha;
  F.g_P0 = g_P0;
  tm.stop(&tl[1]);
  ASCI_TRACE("tables: fixed-point scale 2^-%d, target groups=%zu", F.X.s, G);

  int dev = 0, sms = 152;
  ASCI_TRY_CUDA(cudaGetDevice(&dev));
  ASCI_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t cap_extra =
      std::max<size_t>(tile_capacity() * (size_t)sms * 16, std::min<uint64_t>(bcap, 1ull << 29));
  const size_t pool_cap = N + cap_extra;
  // staging: pairs of classes that fit a tile in place, kCap slots per hash
  // bucket of a big class (expected fill about 13/16)
  const uint64_t scap = std::min<uint64_t>(bcap + bcap / 2 + (1u << 16), 0xfff00000ull);
  Stage stg = {nullptr, nullptr, scap};
  uint64_t *pool_k[2] = {nullptr, nullptr};
  double *pool_s[2] = {nullptr, nullptr};
  unsigned long long *dcount = nullptr;  // [0] candidates, [1] unique, [2] excluded, [3] survivors
  unsigned *derr2 = nullptr;
  if (bcap) {
    ASCI_TRY(arena.alloc(&stg.rec, scap));
    ASCI_TRY(arena.alloc(&stg.alpha, scap));
    for (int i = 0; i < 2; ++i) {
      ASCI_TRY(arena.alloc(&pool_k[i], pool_cap));
      ASCI_TRY(arena.alloc(&pool_s[i], pool_cap));
    }
    ASCI_TRY(arena.alloc(&dcount, 4));
    ASCI_TRY(arena.alloc(&derr2, 1));
    ASCI_TRY_CUDA(cudaMemsetAsync(dcount, 0, 4 * sizeof(unsigned long long), stream));
    ASCI_TRY_CUDA(cudaMemsetAsync(derr2, 0, sizeof(unsigned), stream));
  }
  size_t pool_n = 0;
  int pcur = 0;
  double tau = 0.0;
  long long *pt2_limbs = nullptr;  // ASCI-PT2 fixed-point counters
  if (pt2_out) {
    ASCI_TRY(arena.alloc(&pt2_limbs, 8));
    ASCI_TRY_CUDA(cudaMemsetAsync(pt2_limbs, 0, 8 * sizeof(long long), stream));
  }
  // Candidates [pool_n, c) were appended with their numerators: form their
  // exact scores, or (PT2) add their terms and drop them.
  auto consume = [&](unsigned long long c) -> int {
    if (pt2_out) {
      ASCI_TRY(pt2_terms(F, pool_k[pcur] + pool_n, pool_s[pcur] + pool_n, (size_t)c - pool_n,
                         pt2_limbs, derr2, stream));
      const unsigned long long keep = pool_n;
      ASCI_TRY_CUDA(cudaMemcpyAsync(dcount, &keep, sizeof(keep), cudaMemcpyHostToDevice, stream));
      ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
      return ASCI_OK;
    }
    ASCI_TRY(exact_scores(F, pool_k[pcur] + pool_n, pool_s[pcur] + pool_n, (size_t)c - pool_n,
                          stream));
    pool_n = (size_t)c;
    return ASCI_OK;
  };
  // Prune the pool to the top N and raise tau to its N-th |S| (a lower bound of
  // the final cutoff, so nothing that can still be selected is ever dropped).
  auto prune = [&](Arena &pa) -> int {
    size_t m2 = 0;
    ASCI_TRY(select_topn_packed(pool_k[pcur], pool_s[pcur], pool_n, N, pool_k[pcur ^ 1],
                                pool_s[pcur ^ 1], &m2, pa));
    pcur ^= 1;
    pool_n = m2;
    if (m2 >= N && N > 0) ASCI_TRY(abs_min(pool_s[pcur], pool_n, &tau, pa));
    unsigned long long c = pool_n;
    ASCI_TRY_CUDA(cudaMemcpyAsync(dcount, &c, sizeof(c), cudaMemcpyDefault, stream));
    ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
    return ASCI_OK;
  };
  for (const Batch &b : batches) {
    Arena ba(stream);  // scratch of this batch, released when the batch ends
    uint32_t gg[2];
    ASCI_TRY_CUDA(cudaMemcpyAsync(&gg[0], item_group + b.t0, 4, cudaMemcpyDefault, stream));
    ASCI_TRY_CUDA(cudaMemcpyAsync(&gg[1], item_group + b.t1 - 1, 4, cudaMemcpyDefault, stream));
    ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
    tm.start();
    void *tiles = nullptr;
    size_t ntiles = 0;
    if ((size_t)gg[1] + 1 > G || gg[0] > gg[1]) {
      record_error("batch group range outside the group table", __FILE__, __LINE__);
      return ASCI_ECUDA;
    }
    ASCI_TRACE("batch: items [%llu,%llu) pairs [%llu,%llu) groups [%u,%u)",
               (unsigned long long)b.t0, (unsigned long long)b.t1, (unsigned long long)b.P0,
               (unsigned long long)b.P1, gg[0], gg[1] + 1);
    std::vector<uint32_t> oversized;
    const uint64_t *psi_list = nullptr;
    Spill spill{nullptr, nullptr, 0};
    ASCI_TRY(fused_stage(F, b.t0, b.t1, b.P0, b.P1, gg[0], gg[1] + 1, stg, o.eps_search,
                         dcount + 3, derr2, &tiles, &ntiles, &psi_list, &spill, &oversized, ba));
    ASCI_TRACE("staged: tiles=%zu oversized=%zu", ntiles, oversized.size());
    tm.stop(&tl[2]);
    staged_records += b.P1 - b.P0;
    tm.start();
    size_t t = 0;
    while (t < ntiles) {
      // tiles that can append at most the free capacity
      size_t room = (pool_cap - pool_n) / tile_capacity();
      if (room == 0) {
        tm.stop(&tl[5]);
        tm.start();
        ASCI_TRY(prune(ba));
        tm.stop(&tl[6]);
        tm.start();
        room = (pool_cap - pool_n) / tile_capacity();
        if (room == 0) return ASCI_ENOMEM;
      }
      const size_t t1 = std::min(ntiles, t + room);
      ASCI_TRACE("cells: tiles [%zu,%zu) tau=%.6g pool=%zu", t, t1, tau, pool_n);
      ktm.start();
      ASCI_TRY(fused_cells(F, tiles, psi_list, (uint32_t)t, (uint32_t)t1, stg, tau,
                           pool_k[pcur], pool_s[pcur], dcount, pool_cap, dcount + 1, dcount + 2,
                           derr2, ba));
      ktm.stop(&tl[3]);
      ++tile_launches;
      unsigned long long c = 0;
      unsigned he = 0;
      ASCI_TRY_CUDA(cudaMemcpyAsync(&c, dcount, sizeof(c), cudaMemcpyDefault, stream));
      ASCI_TRY_CUDA(cudaMemcpyAsync(&he, derr2, sizeof(he), cudaMemcpyDefault, stream));
      ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
      if (he) {
        char msg[96];
        snprintf(msg, sizeof(msg), "constraint-tile kernel check failed (flags 0x%x)", he);
        record_error(msg, __FILE__, __LINE__);
        return ASCI_ECUDA;
      }
      if (c > pool_cap) return ASCI_ECUDA;  // cannot happen: room bounds the appends
      ASCI_TRY(consume(c));
      t = t1;
      if (pool_n > N && (pool_cap - pool_n) < pool_cap / 2) {
        tm.stop(&tl[5]);
        tm.start();
        ASCI_TRY(prune(ba));
        tm.stop(&tl[6]);
        tm.start();
      }
    }
    // buckets too large for one tile: those of at most big_tile_capacity()
    // records on chip in the large tile kernel, the rest by global sorts; each
    // launch takes as many of them as the free candidate capacity allows
    // (every record may become one)
    if (!oversized.empty()) {
      std::vector<uint32_t> info;  // 5 words per oversized tile
      ASCI_TRY(tile_info(tiles, oversized, spill, &info, stream));
      std::vector<uint32_t> big_list, big_info, glob_info;
      for (size_t k = 0; k < oversized.size(); ++k) {
        const bool on_chip = (uint64_t)info[5 * k + 1] + info[5 * k + 4] <= big_tile_capacity();
        if (on_chip) big_list.push_back(oversized[k]);
        auto &dst = on_chip ? big_info : glob_info;
        dst.insert(dst.end(), info.begin() + 5 * k, info.begin() + 5 * k + 5);
      }
      ASCI_TRACE("oversized buckets: %zu on chip, %zu by global sort", big_info.size() / 5,
                 glob_info.size() / 5);
      for (int pass = 0; pass < 2; ++pass) {
        const std::vector<uint32_t> &inf = pass == 0 ? big_info : glob_info;
        const size_t cnt = inf.size() / 5;
        auto recs = [&](size_t k) { return (uint64_t)inf[5 * k + 1] + inf[5 * k + 4]; };
        size_t i = 0;
        while (i < cnt) {
          if ((uint64_t)(pool_cap - pool_n) < recs(i)) {
            tm.stop(&tl[5]);
            tm.start();
            ASCI_TRY(prune(ba));
            tm.stop(&tl[6]);
            tm.start();
            if ((uint64_t)(pool_cap - pool_n) < recs(i)) return ASCI_ENOMEM;
          }
          uint64_t room = pool_cap - pool_n, total = 0;
          size_t j = i;
          while (j < cnt && total + recs(j) <= room) total += recs(j++);
          uint64_t nrec = 0;
          ktm.start();
          if (pass == 0)
            ASCI_TRY(fused_big_cells(F, tiles, psi_list, big_list.data() + i, inf.data() + 5 * i,
                                     j - i, stg, spill, tau, pool_k[pcur], pool_s[pcur], dcount,
                                     pool_cap, dcount + 1, dcount + 2, derr2, &nrec, ba));
          else
            ASCI_TRY(fused_big_tiles(F, inf.data() + 5 * i, j - i, stg, spill, tau, pool_k[pcur],
                                     pool_s[pcur], dcount, pool_cap, dcount + 1, dcount + 2,
                                     derr2, &nrec, ba));
          ktm.stop(&tl[4]);
          oversized_records += nrec;
          if (pass == 0) big_records += nrec;
          unsigned long long c = 0;
          unsigned he = 0;
          ASCI_TRY_CUDA(cudaMemcpyAsync(&c, dcount, sizeof(c), cudaMemcpyDefault, stream));
          ASCI_TRY_CUDA(cudaMemcpyAsync(&he, derr2, sizeof(he), cudaMemcpyDefault, stream));
          ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
          if (he) {
            char msg[96];
            snprintf(msg, sizeof(msg), "oversized-tile reduction check failed (flags 0x%x)", he);
            record_error(msg, __FILE__, __LINE__);
            return ASCI_ECUDA;
          }
          if (c > pool_cap) return ASCI_ECUDA;
          ASCI_TRY(consume(c));
          ASCI_TRACE("oversized tiles (%s): [%zu,%zu) %llu records, pool=%zu",
                     pass == 0 ? "on chip" : "global", i, j, (unsigned long long)nrec, pool_n);
          i = j;
        }
      }
    }
    tm.stop(&tl[5]);
    if (pool_n > N) {  // tighten tau before the next batch
      tm.start();
      ASCI_TRY(prune(ba));
      tm.stop(&tl[6]);
    }
  }
  uint64_t unique = 0, excluded = 0, surviving = P;
  if (bcap) {
    unsigned long long hc[4];
    ASCI_TRY_CUDA(cudaMemcpyAsync(hc, dcount, sizeof(hc), cudaMemcpyDefault, stream));
    ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
    unique = hc[1];
    excluded = hc[2];
    if (o.eps_search > 0.0) surviving = hc[3];
  }
  if (pt2_out) {
    double v = 0.0;
    unsigned he = 0;
    if (bcap) {
      double *dv;
      ASCI_TRY(arena.alloc(&dv, 1));
      ASCI_TRY(pt2_value(pt2_limbs, dv, stream));
      ASCI_TRY_CUDA(cudaMemcpyAsync(&v, dv, sizeof(v), cudaMemcpyDeviceToHost, stream));
      ASCI_TRY_CUDA(cudaMemcpyAsync(&he, derr2, sizeof(he), cudaMemcpyDeviceToHost, stream));
      ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
    }
    if (he) {
      record_error("a PT2 term is not finite or exceeds 2^40 (E0 equals or nearly equals a "
                   "target's H_ii)", __FILE__, __LINE__);
      return ASCI_EINVAL;
    }
    *pt2_out = v;
    *out_n = 0;
    if (st) {
      st->surviving = surviving;
      st->unique = unique;
      st->excluded = excluded;
      st->selected = 0;
    }
    total_tm.stop(&tl[7]);
    if (st) {
      memcpy(st->t_stage, tl, sizeof(tl));
      st->tile_launches = tile_launches;
      st->oversized_records = oversized_records;
      st->big_tile_records = big_records;
      st->tile_records = staged_records - oversized_records;
    }
    return ASCI_OK;
  }
  ASCI_TRACE("select: pool=%zu N=%zu", pool_n, N);
  // ------------------------------ select -----------------------------------
  tm.start();
  size_t nsel = 0;
  uint64_t *sel_k = nullptr;
  double *sel_s = nullptr;
  const size_t nout = std::min(N, pool_n);
  if (nout) {
    ASCI_TRY(arena.alloc(&sel_k, nout));
    ASCI_TRY(arena.alloc(&sel_s, nout));
    ASCI_TRY(select_topn_packed(pool_k[pcur], pool_s[pcur], pool_n, N, sel_k, sel_s, &nsel, arena));
    if (o.sort_output && nsel > 1) {
      uint64_t *k2;
      double *s2;
      ASCI_TRY(arena.alloc(&k2, nsel));
      ASCI_TRY(arena.alloc(&s2, nsel));
      ASCI_TRY(radix_sort_u64_f64(&sel_k, &k2, &sel_s, &s2, nsel, 0, 64, arena));
    }
    asci_det *dout = out_dets;
    double *sout = out_scores;
    const bool host_out = !is_device_ptr(out_dets);
    const bool host_sc = !is_device_ptr(out_scores);
    if (host_out) ASCI_TRY(arena.alloc(&dout, nsel));
    if (host_sc) sout = sel_s;
    k_unpack<<<grid_for(nsel), 256, 0, stream>>>(sel_k, nsel, dout);
    ASCI_CHECK_LAUNCH();
    if (host_out)
      ASCI_TRY_CUDA(cudaMemcpyAsync(out_dets, dout, nsel * sizeof(asci_det),
                                    cudaMemcpyDefault, stream));
    if (host_sc)
      ASCI_TRY_CUDA(cudaMemcpyAsync(out_scores, sout, nsel * sizeof(double),
                                    cudaMemcpyDefault, stream));
    else
      ASCI_TRY_CUDA(cudaMemcpyAsync(out_scores, sel_s, nsel * sizeof(double),
                                    cudaMemcpyDefault, stream));
  }
  ASCI_TRY_CUDA(cudaStreamSynchronize(stream));
  tm.stop(&tl[6]);
  *out_n = nsel;
  if (st) {
    st->surviving = surviving;
    st->unique = unique;
    st->excluded = excluded;
    st->selected = nsel;
  }
  (void)g_item0;
  (void)G;
  total_tm.stop(&tl[7]);
  if (st) {
    memcpy(st->t_stage, tl, sizeof(tl));
    st->tile_launches = tile_launches;
    st->oversized_records = oversized_records;
    st->big_tile_records = big_records;
    st->tile_records = staged_records - oversized_records;
  }
  return ASCI_OK;
}

}  // namespace asci

using namespace asci;

// Inputs of the component entry points may be host or device memory; outputs
// are written through a device staging buffer when they are host memory.
static int stage_ints(const asci_ints *ints, Arena &arena, const double **h1, const double **eri) {
  const size_t n = (size_t)ints->norb;
  ASCI_TRY(to_device(ints->h1, n * n, h1, arena));
  ASCI_TRY(to_device(ints->eri, n * n * n * n, eri, arena));
  return ASCI_OK;
}

extern "C" {

void asci_default_opts(asci_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->eps_search = 0.0;
  o->max_constraint_level = 0;
  o->precision = ASCI_FP64;
  o->max_batch_pairs = 0;
  o->sort_output = 0;
}

const char *asci_version(void) { return "libasci 0.1 (sm_103a)"; }

const char *asci_strerror(int code) {
  switch (code) {
    case ASCI_OK: return "ok";
    case ASCI_EINVAL: return "invalid argument";
    case ASCI_ENOMEM: return "out of device memory";
    case ASCI_ECUDA: return "CUDA error";
    case ASCI_ETIMEOUT: return "a bounded wait or an iteration limit ran out";
    default: return "unknown error";
  }
}

const char *asci_last_error(void) { return g_last_error; }

unsigned long long asci_launch_count(void) { return g_launches.load(); }

void asci_debug_fail_allocation(int64_t after) { g_alloc_fault.store(after < 0 ? -1 : after); }

void asci_trim_cache(void) {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && device_pool(dev, &pool) == ASCI_OK)
    cudaMemPoolTrimTo(pool, 0);
}

static int begin_call(void *cuda_stream, cudaStream_t *s) {
  g_last_error[0] = 0;
  *s = (cudaStream_t)cuda_stream;
  int dev = 0;
  ASCI_TRY_CUDA(cudaGetDevice(&dev));
  (void)dev;
  return ASCI_OK;
}

int asci_search(const asci_det *dets, const double *coeffs, size_t ndets, double E0,
                const asci_ints *ints, size_t C, size_t N, const asci_opts *opts,
                asci_det *out_dets, double *out_scores, size_t *out_n, asci_stats *stats,
                void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!dets || !coeffs || !ints || !ints->h1 || !ints->eri || !out_n) return ASCI_EINVAL;
  if ((N > 0) && (!out_dets || !out_scores)) return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32 || ndets == 0 || C == 0) return ASCI_EINVAL;
  if (!std::isfinite(E0) || !std::isfinite(ints->ecore)) return ASCI_EINVAL;
  if (ndets >= (1ull << 32)) return ASCI_EINVAL;
  asci_opts o;
  asci_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.eps_search >= 0.0) || !std::isfinite(o.eps_search)) return ASCI_EINVAL;
  if (o.precision < ASCI_FP64 || o.precision > ASCI_FP32_INT_COMP_ACC) return ASCI_EINVAL;
  if (o.ctas_per_sm < 0 || o.ctas_per_sm > 64) return ASCI_EINVAL;
  if (o.shard_count < 0 || o.shard_count > 1024 ||
      (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count)))
    return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  int r = search_impl(dets, coeffs, ndets, E0, ints, C, N, o, out_dets, out_scores, out_n, stats,
                      s);
  if (r != ASCI_OK) *out_n = 0;
  return r;
}

int asci_pt2(const asci_det *dets, const double *coeffs, size_t ndets, double E0,
             const asci_ints *ints, size_t C, const asci_opts *opts, double *e_pt2,
             asci_stats *stats, void *cuda_stream) {
  if (e_pt2) *e_pt2 = 0.0;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!dets || !coeffs || !ints || !ints->h1 || !ints->eri || !e_pt2) return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32 || ndets == 0 || C == 0) return ASCI_EINVAL;
  if (!std::isfinite(E0) || !std::isfinite(ints->ecore)) return ASCI_EINVAL;
  if (ndets >= (1ull << 32)) return ASCI_EINVAL;
  asci_opts o;
  asci_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.eps_search >= 0.0) || !std::isfinite(o.eps_search)) return ASCI_EINVAL;
  if (o.precision < ASCI_FP64 || o.precision > ASCI_FP32_INT_COMP_ACC) return ASCI_EINVAL;
  if (o.ctas_per_sm < 0 || o.ctas_per_sm > 64) return ASCI_EINVAL;
  if (o.shard_count < 0 || o.shard_count > 1024 ||
      (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count)))
    return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  size_t n_out = 0;
  double v = 0.0;
  int r = search_impl(dets, coeffs, ndets, E0, ints, C, 0, o, nullptr, nullptr, &n_out, stats, s,
                      &v);
  if (r == ASCI_OK) *e_pt2 = v;
  return r;
}

int asci_excitations(const asci_ints *ints, const asci_det *core, const double *coeffs,
                     size_t ncore, asci_det *out_targets, double *out_values, size_t capacity,
                     size_t *out_n, void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!ints || !ints->h1 || !ints->eri || !core || !coeffs || !out_targets || !out_values || !out_n)
    return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32 || ncore == 0) return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  const int n = ints->norb;
  const asci_det *dcore;
  const double *dc, *h1, *eri;
  ASCI_TRY(to_device(core, ncore, &dcore, arena));
  ASCI_TRY(to_device(coeffs, ncore, &dc, arena));
  ASCI_TRY(stage_ints(ints, arena, &h1, &eri));
  asci_det d0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&d0, dcore, sizeof(d0), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  const int na = __builtin_popcountll(d0.alpha), nb = __builtin_popcountll(d0.beta);
  if (na > n || nb > n || (n < 64 && ((d0.alpha | d0.beta) >> n))) return ASCI_EINVAL;
  const ExcCounts X = exc_counts(n, na, nb);
  const uint64_t total = (uint64_t)ncore * X.total;
  if (total > capacity) return ASCI_EINVAL;
  // every core det must have the same electron counts and no bits >= norb
  {
    unsigned *derr;
    uint64_t *tk;
    uint32_t *ti;
    double *tc;
    ASCI_TRY(arena.alloc(&derr, 1));
    ASCI_TRY(arena.alloc(&tk, ncore));
    ASCI_TRY(arena.alloc(&ti, ncore));
    ASCI_TRY(arena.alloc(&tc, ncore));
    ASCI_TRY_CUDA(cudaMemsetAsync(derr, 0, sizeof(unsigned), s));
    ASCI_TRY_CUDA(cudaMemsetAsync(tc, 0, ncore * sizeof(double), s));
    k_prepare_psi<<<grid_for(ncore), 256, 0, s>>>(dcore, tc, ncore, n, na, nb, tk, ti, derr);
    ASCI_CHECK_LAUNCH();
    unsigned herr = 0;
    ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr & (kBadRange | kBadCount)) return ASCI_EINVAL;
  }
  DevInts I;
  ASCI_TRY(build_tables(h1, eri, n, na, nb, ints->ecore, false, arena, &I));
  uint64_t *ck, *ok;
  double *ov;
  asci_det *dt;
  ASCI_TRY(arena.alloc(&ck, ncore));
  ASCI_TRY(arena.alloc(&ok, total));
  ASCI_TRY(out_buffer(out_values, total, &ov, arena));
  ASCI_TRY(out_buffer(out_targets, total, &dt, arena));
  k_input_keys<<<grid_for(ncore), 256, 0, s>>>(dcore, ncore, ck);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(emit_fixed_order(I, ck, dc, ncore, ok, ov, arena));
  k_unpack<<<grid_for(total), 256, 0, s>>>(ok, total, dt);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(finish_out(out_values, ov, total, s));
  ASCI_TRY(finish_out(out_targets, dt, total, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = total;
  return ASCI_OK;
}

int asci_diagonal(const asci_ints *ints, const asci_det *dets, size_t n, double *out_haa,
                  void *cuda_stream) {
  if (!ints || !ints->h1 || !ints->eri || !dets || !out_haa) return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32) return ASCI_EINVAL;
  if (n == 0) return ASCI_OK;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  const asci_det *dd;
  const double *h1, *eri;
  double *dout;
  ASCI_TRY(to_device(dets, n, &dd, arena));
  ASCI_TRY(stage_ints(ints, arena, &h1, &eri));
  ASCI_TRY(out_buffer(out_haa, n, &dout, arena));
  {
    // no bits at or above norb (they would index past the integral tables)
    unsigned *derr;
    uint64_t *tk;
    uint32_t *ti;
    double *tc;
    ASCI_TRY(arena.alloc(&derr, 1));
    ASCI_TRY(arena.alloc(&tk, n));
    ASCI_TRY(arena.alloc(&ti, n));
    ASCI_TRY(arena.alloc(&tc, n));
    ASCI_TRY_CUDA(cudaMemsetAsync(derr, 0, sizeof(unsigned), s));
    ASCI_TRY_CUDA(cudaMemsetAsync(tc, 0, n * sizeof(double), s));
    k_prepare_psi<<<grid_for(n), 256, 0, s>>>(dd, tc, n, ints->norb, -1, -1, tk, ti, derr);
    ASCI_CHECK_LAUNCH();
    unsigned herr = 0;
    ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr & kBadRange) return ASCI_EINVAL;
  }
  DevInts I;
  ASCI_TRY(build_tables(h1, eri, ints->norb, 0, 0, ints->ecore, false, arena, &I));
  uint64_t *k;
  ASCI_TRY(arena.alloc(&k, n));
  k_input_keys<<<grid_for(n), 256, 0, s>>>(dd, n, k);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(diagonal_packed(I, k, n, dout, arena));
  ASCI_TRY(finish_out(out_haa, dout, n, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  return ASCI_OK;
}

int asci_sort_accumulate(const asci_det *keys, const double *values, size_t n,
                         asci_det *out_keys, double *out_sums, size_t *out_n,
                         void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!keys || !values || !out_keys || !out_sums || !out_n) return ASCI_EINVAL;
  if (n == 0) return ASCI_OK;
  if (n >= (1ull << 32)) return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  const asci_det *dk;
  const double *dv;
  ASCI_TRY(to_device(keys, n, &dk, arena));
  ASCI_TRY(to_device(values, n, &dv, arena));
  uint64_t *k0, *k1, *uk;
  double *v0, *v1, *us;
  asci_det *dok;
  ASCI_TRY(arena.alloc(&k0, n));
  ASCI_TRY(arena.alloc(&k1, n));
  ASCI_TRY(arena.alloc(&uk, n));
  ASCI_TRY(arena.alloc(&v0, n));
  ASCI_TRY(arena.alloc(&v1, n));
  ASCI_TRY(out_buffer(out_sums, n, &us, arena));
  ASCI_TRY(out_buffer(out_keys, n, &dok, arena));
  unsigned *bad, hbad = 0;
  ASCI_TRY(arena.alloc(&bad, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
  k_input_keys_checked<<<grid_for(n), 256, 0, s>>>(dk, n, k0, bad);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (hbad) {
    record_error("asci_sort_accumulate: a key word has bits at or above 32", __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  ASCI_TRY_CUDA(cudaMemcpyAsync(v0, dv, n * sizeof(double), cudaMemcpyDefault, s));
  size_t u = 0;
  ASCI_TRY(sort_accumulate(&k0, &k1, &v0, &v1, n, uk, us, &u, arena));
  k_unpack<<<grid_for(u), 256, 0, s>>>(uk, u, dok);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(finish_out(out_sums, us, u, s));
  ASCI_TRY(finish_out(out_keys, dok, u, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = u;
  return ASCI_OK;
}

int asci_search_many(asci_problem *problems, size_t count, const asci_opts *opts,
                     int32_t streams) {
  g_last_error[0] = 0;
  if (streams < 1 || (count > 0 && !problems)) return ASCI_EINVAL;
  if (!count) return ASCI_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ASCI_ECUDA;
  std::atomic<size_t> next{0};
  std::mutex mu;
  size_t first_bad = count;
  std::string first_msg;
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    const bool own = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    for (;;) {
      const size_t i = next.fetch_add(1);
      if (i >= count) break;
      asci_problem &p = problems[i];
      p.status = own ? asci_search(p.dets, p.coeffs, p.ndets, p.E0, p.ints, p.C, p.N, opts,
                                   p.out_dets, p.out_scores, p.out_n, p.stats, s)
                     : ASCI_ECUDA;
      if (p.status != ASCI_OK) {
        std::lock_guard<std::mutex> lk(mu);
        if (i < first_bad) {
          first_bad = i;
          first_msg = own ? g_last_error : "cannot create a CUDA stream";
        }
      }
    }
    if (own) cudaStreamDestroy(s);
  };
  const size_t nt = std::min<size_t>((size_t)streams, count);
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto &t : pool) t.join();
  if (first_bad < count) {
    snprintf(g_last_error, sizeof(g_last_error), "problem %zu: %s", first_bad, first_msg.c_str());
    return problems[first_bad].status;
  }
  return ASCI_OK;
}

int asci_constraint_classes(const asci_det *dets, const double *coeffs, size_t ndets,
                            const asci_ints *ints, size_t C, int32_t level, uint64_t *out_pairs,
                            size_t capacity, size_t *out_n, void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!dets || !coeffs || !ints || !ints->h1 || !ints->eri || !out_n) return ASCI_EINVAL;
  if (capacity > 0 && !out_pairs) return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32 || ndets == 0 || C == 0 || level < 1) return ASCI_EINVAL;
  if (!std::isfinite(ints->ecore) || ndets >= (1ull << 32)) return ASCI_EINVAL;
  asci_opts o;
  asci_default_opts(&o);
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  ClassQuery q{level, out_pairs, capacity, 0};
  size_t dummy = 0;
  const int r = search_impl(dets, coeffs, ndets, 0.0, ints, C, 0, o, nullptr, nullptr, &dummy,
                            nullptr, s, nullptr, &q);
  if (r != ASCI_OK) return r;
  *out_n = q.n;
  return ASCI_OK;
}

int asci_shard_assign(const uint64_t *weights, size_t n, int32_t shards,
                      const uint64_t *initial_loads, int32_t *shard_out) {
  if (shards < 1 || (n > 0 && (!weights || !shard_out))) return ASCI_EINVAL;
  std::vector<size_t> order(n);
  std::iota(order.begin(), order.end(), (size_t)0);
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t b) { return weights[a] > weights[b]; });
  using Load = std::pair<uint64_t, int32_t>;  // (load, shard): smallest first
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> q;
  for (int32_t i = 0; i < shards; ++i) q.push({initial_loads ? initial_loads[i] : 0ull, i});
  for (size_t c : order) {
    Load l = q.top();
    q.pop();
    shard_out[c] = l.second;
    l.first += weights[c];
    q.push(l);
  }
  return ASCI_OK;
}

int asci_select_begin(uint64_t total, uint64_t N, asci_select_state *st) {
  if (!st) return ASCI_EINVAL;
  memset(st, 0, sizeof(*st));
  st->remaining = N;
  if (total <= N) {  // every entry is selected
    st->threshold[0] = st->threshold[1] = ~0ull;
    st->digit = -1;
    st->done = 1;
    return ASCI_OK;
  }
  st->digit = 15;
  return ASCI_OK;
}

int asci_select_step(asci_select_state *st, const uint64_t hist[256]) {
  if (!st || !hist || st->done || st->digit < 0 || st->digit > 15 || st->remaining == 0)
    return ASCI_EINVAL;
  // the byte value d whose bucket holds the remaining-th entry of the class
  uint64_t below = 0;
  int d = 0;
  for (; d < 256; ++d) {
    if (below + hist[d] >= st->remaining) break;
    below += hist[d];
  }
  if (d == 256) {
    record_error("asci_select_step: the histogram holds fewer entries than remain", __FILE__,
                 __LINE__);
    return ASCI_EINVAL;
  }
  st->remaining -= below;
  const int word = st->digit >= 8 ? 0 : 1;
  const int shift = 8 * (st->digit >= 8 ? st->digit - 8 : st->digit);
  st->prefix[word] |= (uint64_t)d << shift;
  st->mask[word] |= 0xffull << shift;
  if (hist[d] == st->remaining) {  // the whole bucket is selected: lower bits are free
    st->threshold[0] = st->prefix[0] | ~st->mask[0];
    st->threshold[1] = st->prefix[1] | ~st->mask[1];
    st->digit = -1;
    st->done = 1;
    return ASCI_OK;
  }
  st->threshold[0] = st->prefix[0];
  st->threshold[1] = st->prefix[1];
  if (--st->digit < 0) st->done = 1;  // every byte fixed: threshold is the N-th word
  return ASCI_OK;
}

int asci_select_histogram(const asci_det *keys, const double *scores, size_t n, int32_t digit,
                          const uint64_t prefix[2], const uint64_t mask[2], uint64_t hist[256],
                          void *cuda_stream) {
  if ((n && (!keys || !scores)) || !prefix || !mask || !hist || digit < 0 || digit > 15)
    return ASCI_EINVAL;
  if (n >= (1ull << 32)) return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  uint64_t *k = nullptr;
  const double *ds = nullptr;
  if (n) {
    const asci_det *dk;
    ASCI_TRY(to_device(keys, n, &dk, arena));
    ASCI_TRY(to_device(scores, n, &ds, arena));
    ASCI_TRY(arena.alloc(&k, n));
    k_input_keys<<<grid_for(n), 256, 0, s>>>(dk, n, k);
    ASCI_CHECK_LAUNCH();
  }
  return select_histogram(k, ds, n, digit, prefix, mask, hist, arena);
}

int asci_select_below(const asci_det *keys, const double *scores, size_t n,
                      const uint64_t threshold[2], asci_det *out_keys, double *out_scores,
                      size_t *out_n, void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!out_n || !threshold || (n && (!keys || !scores || !out_keys || !out_scores)))
    return ASCI_EINVAL;
  if (n >= (1ull << 32)) return ASCI_EINVAL;
  if (n == 0) return ASCI_OK;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  const asci_det *dk;
  const double *ds;
  ASCI_TRY(to_device(keys, n, &dk, arena));
  ASCI_TRY(to_device(scores, n, &ds, arena));
  uint64_t *k, *ok;
  double *os;
  asci_det *dok;
  ASCI_TRY(arena.alloc(&k, n));
  ASCI_TRY(arena.alloc(&ok, n));
  ASCI_TRY(out_buffer(out_scores, n, &os, arena));
  ASCI_TRY(out_buffer(out_keys, n, &dok, arena));
  k_input_keys<<<grid_for(n), 256, 0, s>>>(dk, n, k);
  ASCI_CHECK_LAUNCH();
  size_t m = 0;
  ASCI_TRY(select_below(k, ds, n, threshold, ok, os, &m, arena));
  k_unpack<<<grid_for(m), 256, 0, s>>>(ok, m, dok);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(finish_out(out_scores, os, m, s));
  ASCI_TRY(finish_out(out_keys, dok, m, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = m;
  return ASCI_OK;
}

int asci_select_topn(const asci_det *keys, const double *scores, size_t n, size_t N,
                     asci_det *out_keys, double *out_scores, size_t *out_n,
                     void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!keys || !scores || !out_n || (N && (!out_keys || !out_scores))) return ASCI_EINVAL;
  if (n == 0 || N == 0) return ASCI_OK;
  if (n >= (1ull << 32)) return ASCI_EINVAL;
  cudaStream_t s;
  ASCI_TRY(begin_call(cuda_stream, &s));
  Arena arena(s);
  const asci_det *dk;
  const double *ds;
  ASCI_TRY(to_device(keys, n, &dk, arena));
  ASCI_TRY(to_device(scores, n, &ds, arena));
  const size_t m0 = std::min(n, N);
  uint64_t *k, *ok;
  double *os;
  asci_det *dok;
  ASCI_TRY(arena.alloc(&k, n));
  ASCI_TRY(arena.alloc(&ok, m0));
  ASCI_TRY(out_buffer(out_scores, m0, &os, arena));
  ASCI_TRY(out_buffer(out_keys, m0, &dok, arena));
  k_input_keys<<<grid_for(n), 256, 0, s>>>(dk, n, k);
  ASCI_CHECK_LAUNCH();
  size_t m = 0;
  ASCI_TRY(select_topn_packed(k, ds, n, N, ok, os, &m, arena));
  k_unpack<<<grid_for(m), 256, 0, s>>>(ok, m, dok);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(finish_out(out_scores, os, m, s));
  ASCI_TRY(finish_out(out_keys, dok, m, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = m;
  return ASCI_OK;
}

}  // extern "C"
