// Internal declarations of libasci (GPU path).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "asci.h"

namespace asci {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------

void record_error(const char *what, const char *file, int line);
// Allocation fault injection for tests of the error path (asci_debug_fail_allocation):
// true when this allocation is to fail.
bool injected_alloc_failure();
void clear_last_error();

// Stage tracing to stderr, enabled by the environment variable ASCI_TRACE=1.
bool trace_on();
#define ASCI_TRACE(...)                                \
  do {                                                 \
    if (::asci::trace_on()) {                          \
      fprintf(stderr, "[asci] " __VA_ARGS__);          \
      fputc('\n', stderr);                             \
      fflush(stderr);                                  \
    }                                                  \
  } while (0)

// Library-owned stream-ordered memory pool of a device (kept cached between calls).
int device_pool(int dev, cudaMemPool_t *pool);

#define ASCI_TRY_CUDA(expr)                                 \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) {                               \
      ::asci::record_error(cudaGetErrorString(e__), __FILE__, __LINE__); \
      return (e__ == cudaErrorMemoryAllocation) ? ASCI_ENOMEM : ASCI_ECUDA; \
    }                                                       \
  } while (0)

#define ASCI_TRY(expr)              \
  do {                              \
    int r__ = (expr);               \
    if (r__ != ASCI_OK) return r__; \
  } while (0)

// Every kernel launch is followed by ASCI_CHECK_LAUNCH, which also counts it
// (asci_launch_count() reports the total, for launch accounting by callers).
void count_launch();
#define ASCI_CHECK_LAUNCH()  \
  do {                       \
    ::asci::count_launch();  \
    ASCI_TRY_CUDA(cudaGetLastError()); \
  } while (0)

// Stream-ordered scratch arena: every allocation is released when the arena
// goes out of scope (cudaFreeAsync on the same stream).
class Arena {
 public:
  explicit Arena(cudaStream_t s) : stream_(s) {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && device_pool(dev, &pool_) != ASCI_OK) pool_ = nullptr;
  }
  // Bump mode: every allocation is carved, 256-byte aligned, from the given
  // device region; nothing is allocated or freed.  Exhaustion returns ASCI_ENOMEM.
  Arena(cudaStream_t s, void *region, size_t bytes)
      : stream_(s), bump_base_(static_cast<char *>(region)), bump_cap_(bytes) {}
  ~Arena() { release(); }
  Arena(const Arena &) = delete;
  Arena &operator=(const Arena &) = delete;
  template <typename T>
  int alloc(T **p, size_t count) {
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 256;
    if (bump_base_) {
      const size_t off = (bump_off_ + 255) & ~(size_t)255;
      if (off > bump_cap_ || bytes > bump_cap_ - off) {
        record_error("fixed scratch region exhausted", __FILE__, __LINE__);
        *p = nullptr;
        return ASCI_ENOMEM;
      }
      bump_off_ = off + bytes;
      *p = reinterpret_cast<T *>(bump_base_ + off);
      return ASCI_OK;
    }
    if (injected_alloc_failure()) {
      record_error("injected allocation failure", __FILE__, __LINE__);
      *p = nullptr;
      return ASCI_ENOMEM;
    }
    cudaError_t e = pool_ ? cudaMallocFromPoolAsync(&q, bytes, pool_, stream_)
                          : cudaMallocAsync(&q, bytes, stream_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      record_error(cudaGetErrorString(e), __FILE__, __LINE__);
      *p = nullptr;
      return ASCI_ENOMEM;
    }
    ptrs_.push_back(q);
    *p = static_cast<T *>(q);
    return ASCI_OK;
  }
  void release() {
    for (void *q : ptrs_) cudaFreeAsync(q, stream_);
    ptrs_.clear();
    bump_off_ = 0;
  }
  cudaStream_t stream() const { return stream_; }

 private:
  cudaStream_t stream_;
  cudaMemPool_t pool_ = nullptr;
  std::vector<void *> ptrs_;
  char *bump_base_ = nullptr;
  size_t bump_cap_ = 0, bump_off_ = 0;
};

// Host or device memory: inputs are used in place when on the device and
// staged through the arena otherwise; outputs that are host memory are written
// through a device buffer and copied out at the end of the call.
inline bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
int to_device(const T *src, size_t count, const T **dst, Arena &arena) {
  if (is_device_ptr(src)) {
    *dst = src;
    return ASCI_OK;
  }
  T *d = nullptr;
  ASCI_TRY(arena.alloc(&d, count));
  if (count)
    ASCI_TRY_CUDA(cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyDefault,
                                  arena.stream()));
  *dst = d;
  return ASCI_OK;
}

template <typename T>
int out_buffer(T *user, size_t count, T **dev, Arena &arena) {
  if (is_device_ptr(user)) {
    *dev = user;
    return ASCI_OK;
  }
  return arena.alloc(dev, count);
}

template <typename T>
int finish_out(T *user, const T *dev, size_t count, cudaStream_t s) {
  if ((const T *)user != dev && count)
    ASCI_TRY_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDefault, s));
  return ASCI_OK;
}

// Device time between start() and stop() on one stream, added to *acc in
// milliseconds (stop() waits for the stream to reach the end event).
struct StageTimer {
  cudaStream_t s;
  cudaEvent_t ev[2];
  bool ok = false;
  explicit StageTimer(cudaStream_t st) : s(st) {
    ok = cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess;
  }
  ~StageTimer() {
    if (ok) {
      cudaEventDestroy(ev[0]);
      cudaEventDestroy(ev[1]);
    }
  }
  void start() {
    if (ok) cudaEventRecord(ev[0], s);
  }
  void stop(double *acc) {
    if (!ok) return;
    cudaEventRecord(ev[1], s);
    cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *acc += ms;
  }
};

// ---------------------------------------------------------------------------
// determinants and keys
// ---------------------------------------------------------------------------

// Packed 64-bit key of a determinant (norb <= 32): beta word high, alpha word
// low, so that unsigned order equals the 128-bit key order.
__host__ __device__ inline uint64_t pack_key(uint32_t a, uint32_t b) {
  return ((uint64_t)b << 32) | (uint64_t)a;
}
__host__ __device__ inline uint32_t key_alpha(uint64_t k) { return (uint32_t)k; }
__host__ __device__ inline uint32_t key_beta(uint64_t k) { return (uint32_t)(k >> 32); }

// Sign of the single p -> q on string s: (-1)^popc(s & bits strictly between).
__device__ __forceinline__ int single_parity(uint32_t s, int p, int q) {
  int lo = p < q ? p : q, hi = p < q ? q : p;
  uint32_t between = ((hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u)) & ~((2u << lo) - 1u);
  return __popc(s & between) & 1;
}

// Position of the k-th (0-based) set bit of w; w must hold more than k bits.
__device__ __forceinline__ int nth_set_bit(uint32_t w, int k) {
  int pos = 0, c;
  c = __popc(w & 0xffffu);
  if (k >= c) { k -= c; w >>= 16; pos += 16; }
  c = __popc(w & 0xffu);
  if (k >= c) { k -= c; w >>= 8; pos += 8; }
  c = __popc(w & 0xfu);
  if (k >= c) { k -= c; w >>= 4; pos += 4; }
  c = __popc(w & 0x3u);
  if (k >= c) { k -= c; w >>= 2; pos += 2; }
  c = (int)(w & 1u);
  if (k >= c) pos += 1;
  return pos;
}

// Colex unranking of a pair x < y: r = y(y-1)/2 + x.
__device__ __forceinline__ void unrank_pair(uint32_t r, int *x, int *y) {
  int yy = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)r)) * 0.5f);
  while ((uint32_t)(yy * (yy - 1) / 2) > r) --yy;
  while ((uint32_t)((yy + 1) * yy / 2) <= r) ++yy;
  *y = yy;
  *x = (int)(r - (uint32_t)(yy * (yy - 1) / 2));
}

// Division by a loop-invariant divisor with a multiply-high and two shifts
// (the round-up method of Granlund and Montgomery, 1994); exact for every
// 32-bit dividend and divisors 1 <= d < 2^31.
struct FastDiv {
  uint32_t d, m, s1, s2;
  __host__ __device__ FastDiv() : d(1), m(1), s1(0), s2(0) {}
  __host__ explicit FastDiv(uint32_t div) : d(div) {
    uint32_t l = 0;
    while ((1ull << l) < (uint64_t)div) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - div)) / div) + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 0 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    uint32_t t = __umulhi(n, m);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// ---------------------------------------------------------------------------
// integral tables resident on the device for one search
// ---------------------------------------------------------------------------

struct DevInts {
  int n, na, nb;
  double ecore;
  const double *h1;     // n*n
  const double *eri;    // n^4, (pq|rs)
  const double *asym;   // n^4, [((i*n+a)*n+j)*n+b] = (ia|jb) - (ib|ja)
  const double *s_same; // n^3, [(i*n+a)*n+k] = (ia|kk) - (ik|ka)
  const double *s_opp;  // n^3, [(i*n+a)*n+k] = (ia|kk)
  const double *jk;     // n*n, (pp|qq) - (pq|qp)
  const double *jj;     // n*n, (pp|qq)
  const float *eri32;   // n^4 FP32 copy (precision variants)
  const float *asym32;  // n^4 FP32 copy
  // the asym values again, laid out [((j*n+b)*n+i)*n+a] (equal bit for bit):
  // the beta doubles of one warp's chunk vary a fastest, so this layout puts
  // a chunk's gathers in a few contiguous rows
  const double *asymT;
  const float *asymT32;
};

// Slater-Condon pieces shared by the excitation generator and the
// Hamiltonian build.  Single i -> a on the string s (other spin o), without
// its sign: h_ia + sum_{k in s} ((ia|kk) - (ik|ka)) + sum_{k in o} (ia|kk).
__device__ __forceinline__ double single_value(const DevInts &I, uint32_t s, uint32_t o, int i,
                                               int a) {
  const int n = I.n;
  const double *ss = I.s_same + ((size_t)i * n + a) * n;
  const double *so = I.s_opp + ((size_t)i * n + a) * n;
  double v = I.h1[i * n + a];
  for (uint32_t m = s; m; m &= m - 1) v += ss[__ffs(m) - 1];
  for (uint32_t m = o; m; m &= m - 1) v += so[__ffs(m) - 1];
  return v;
}

__device__ __forceinline__ double eri4(const double *t, int n, int i, int a, int j, int b) {
  return t[(((size_t)i * n + a) * n + j) * n + b];
}

// Sign bit of the same-spin double i<j -> a<b on s, taken as i -> a, then j -> b.
__device__ __forceinline__ int double_parity(uint32_t s, int i, int j, int a, int b) {
  int p1 = single_parity(s, i, a);
  uint32_t s1 = s ^ (1u << i) ^ (1u << a);
  return p1 ^ single_parity(s1, j, b);
}

__device__ __forceinline__ uint32_t full_mask(int n) {
  return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// 1/x to FP64 accuracy from the FP32 estimate __frcp_rn and two
// Newton-Raphson steps y <- y(2 - xy) (each squares the relative error:
// 2^-23 -> 2^-46 -> 2^-92), for |x| in [1e-30, 1e30].  GB300 has little FP64
// throughput, and this avoids the longer FP64 division sequence.
__device__ __forceinline__ double recip_fast(double x) {
  double y = (double)__frcp_rn((float)x);
  y = y * fma(-x, y, 2.0);
  return y * fma(-x, y, 2.0);
}

// Counts of one determinant's excitations (Sec. 2.1: singles and doubles).
struct ExcCounts {
  uint32_t na, nb, va, vb;
  uint32_t sa, sb;      // singles per spin: n v
  uint32_t pa_h, pa_p;  // C(na,2), C(va,2)
  uint32_t pb_h, pb_p;  // C(nb,2), C(vb,2)
  uint64_t daa, dbb, dab, total;
};

ExcCounts exc_counts(int n, int na, int nb);

// Host-side build of the derived integral tables from h1 / eri already on the device.
int build_tables(const double *h1_dev, const double *eri_dev, int n, int na, int nb, double ecore,
                 bool want_fp32, Arena &arena, DevInts *out);

// ---------------------------------------------------------------------------
// primitives (sort.cu)
// ---------------------------------------------------------------------------

// Exclusive prefix sum, device-wide; in and out may alias.
int scan_exclusive_u32(const uint32_t *in, uint32_t *out, size_t n, Arena &arena);
int scan_exclusive_u64(const uint64_t *in, uint64_t *out, size_t n, Arena &arena);
// Exclusive scan of the pairs of each item of the constraint-batched
// generation (group in the bits above opbits, alpha operation below): writes
// T + 1 entries, the last one the total.
int scan_item_weights(const uint64_t *items, uint64_t T, int opbits, const uint32_t *grp_count,
                      const ExcCounts &X, uint64_t *Wexcl, Arena &arena);
// Exclusive scan of the flags "item i starts a new target alpha string" of a
// sorted item list: T + 1 entries, the last one the number of strings.
int scan_item_heads(const uint64_t *items, uint64_t T, uint32_t *excl, Arena &arena);

// Stable LSD radix sort of 64-bit keys on bits [begin_bit, end_bit), with an
// optional payload.  The sorted data ends in *keys / *vals (the two buffers of
// each pair are swapped as passes proceed).  n < 2^32.
int radix_sort_u64(uint64_t **keys, uint64_t **keys_alt, size_t n, int begin_bit, int end_bit,
                   Arena &arena);
int radix_sort_u64_u32(uint64_t **keys, uint64_t **keys_alt, uint32_t **vals, uint32_t **vals_alt,
                       size_t n, int begin_bit, int end_bit, Arena &arena);
int radix_sort_u64_f64(uint64_t **keys, uint64_t **keys_alt, double **vals, double **vals_alt,
                       size_t n, int begin_bit, int end_bit, Arena &arena);
// The same keys-only sort when the caller knows which bits vary among the
// keys (a digit with no varying bit is skipped; varying bits outside the mask
// would be left unsorted).
int radix_sort_u64_varying(uint64_t **keys, uint64_t **keys_alt, size_t n, int begin_bit,
                           int end_bit, uint64_t varying, Arena &arena);

// Bits in which the keys differ (OR of key ^ keys[0]); result on the host.
int varying_bits_u64(const uint64_t *keys, size_t n, uint64_t *host_mask, Arena &arena);

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------

// Sort-and-accumulate of packed (key, value) pairs: sorts in place (buffers
// may be swapped) and writes unique keys and sums.  Returns U on the host.
int sort_accumulate(uint64_t **keys, uint64_t **keys_alt, double **vals, double **vals_alt,
                    size_t n, uint64_t *ukeys, double *usums, size_t *host_u, Arena &arena);

// H_ii of packed keys.
int diagonal_packed(const DevInts &I, const uint64_t *keys, size_t n, double *out, Arena &arena);

// Top-N by |score| with key tie-break; compacts into out arrays (may not alias
// the inputs).  Returns the count on the host.
int select_topn_packed(const uint64_t *keys, const double *scores, size_t n, size_t N,
                       uint64_t *out_keys, double *out_scores, size_t *host_out_n, Arena &arena);

// Histogram of byte `digit` of the rank word (~bits(|S|), key) over entries
// matching pre on the bits of msk ({hi, lo}); hist is host memory.
int select_histogram(const uint64_t *keys, const double *scores, size_t n, int digit,
                     const uint64_t pre[2], const uint64_t msk[2], uint64_t hist[256],
                     Arena &arena);
// Entries whose rank word is at most thr ({hi, lo}), compacted.
int select_below(const uint64_t *keys, const double *scores, size_t n, const uint64_t thr[2],
                 uint64_t *out_keys, double *out_scores, size_t *host_out_n, Arena &arena);

// Excitation emission in the fixed per-determinant order (component entry).
int emit_fixed_order(const DevInts &I, const uint64_t *core_keys, const double *core_c,
                     size_t ncore, uint64_t *out_keys, double *out_vals, Arena &arena);

}  // namespace asci
