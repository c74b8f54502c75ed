// Device-wide primitives: exclusive scan and a stable LSD radix sort.
//
// The sort is the "sort" of the paper's sort-and-accumulate (Sec. 2.2); it is
// written for this library: 8-bit digits, one histogram (upsweep) kernel, a
// device-wide scan of the digit-major histogram, and a scatter (downsweep)
// kernel that ranks each tile's keys stably with warp ballots.
#include "asci_internal.cuh"

namespace asci {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *total) {
  __shared__ T warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  T warp_prefix = warp ? warp_sums[warp - 1] : T(0);
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

// Scan inputs: an array, or a value computed from each index.
template <typename T>
struct ArrayIn {
  const T *p;
  __device__ T operator()(size_t i) const { return p[i]; }
};

// Pairs of item i (the constraint-batched generation's item format, alpha
// operation in the low opbits, group above it): the beta singles and doubles
// for o = 0, the single itself and its alpha-beta doubles for an alpha
// single, one pair for an alpha double; times the group's core determinants.
// Index T (one past the end) is 0, so the scan's last entry is the total.
struct ItemWeightIn {
  const uint64_t *items;
  const uint32_t *grp_count;
  uint64_t T, npd0, npd1;
  uint32_t omask, sa;
  int opbits;
  __device__ uint64_t operator()(size_t i) const {
    if (i >= T) return 0;
    const uint32_t lo = (uint32_t)items[i];
    const uint32_t k = lo >> opbits, o = lo & omask;
    const uint64_t npd = (o == 0) ? npd0 : (o <= sa ? npd1 : 1ull);
    return npd * grp_count[k];
  }
};

// 1 where item i starts a new target alpha string (its high word changes);
// index T (one past the end) is 0, so the scan's last entry is the count.
struct ItemHeadIn {
  const uint64_t *items;
  uint64_t T;
  __device__ uint32_t operator()(size_t i) const {
    if (i >= T) return 0u;
    return (i == 0 || (items[i] >> 32) != (items[i - 1] >> 32)) ? 1u : 0u;
  }
};

template <typename T, typename In>
__global__ void k_tile_reduce(In in, size_t n, T *partial) {
  size_t base = (size_t)blockIdx.x * kScanTile;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t idx = base + (size_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s += in(idx);
  }
  T total;
  block_exclusive_scan<T>(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Shared-memory index of tile element e, padded by one element per 128 bytes
// so that the transposed pass (thread t on elements 16t .. 16t+15) falls on
// distinct banks: without the pad every thread of a warp hits one or two banks.
template <typename T>
__device__ __forceinline__ int scan_pad(int e) {
  return e + e / (int)(128 / sizeof(T));
}

template <typename T, typename In>
__global__ void k_tile_scan(In in, T *out, size_t n, const T *partial) {
  __shared__ T tile[kScanTile + kScanTile / (128 / sizeof(T))];
  size_t base = (size_t)blockIdx.x * kScanTile;
  // coalesced load into shared memory
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t idx = base + (size_t)i * kScanThreads + threadIdx.x;
    tile[scan_pad<T>(i * kScanThreads + threadIdx.x)] = idx < n ? in(idx) : T(0);
  }
  __syncthreads();
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = tile[scan_pad<T>(threadIdx.x * kScanItems + i)];
    s += v[i];
  }
  T pre = block_exclusive_scan<T>(s, nullptr);
  if (partial) pre += partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    tile[scan_pad<T>(threadIdx.x * kScanItems + i)] = pre;
    pre += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t idx = base + (size_t)i * kScanThreads + threadIdx.x;
    if (idx < n) out[idx] = tile[scan_pad<T>(i * kScanThreads + threadIdx.x)];
  }
}

template <typename T, typename In>
int scan_exclusive_by(In in, T *out, size_t n, Arena &arena) {
  if (n == 0) return ASCI_OK;
  size_t nb = (n + kScanTile - 1) / kScanTile;
  cudaStream_t s = arena.stream();
  if (nb == 1) {
    k_tile_scan<T, In><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    ASCI_CHECK_LAUNCH();
    return ASCI_OK;
  }
  T *partial = nullptr;
  ASCI_TRY(arena.alloc(&partial, nb));
  k_tile_reduce<T, In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, partial);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_by<T>(ArrayIn<T>{partial}, partial, nb, arena));
  k_tile_scan<T, In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, partial);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

template <typename T>
int scan_exclusive(const T *in, T *out, size_t n, Arena &arena) {
  return scan_exclusive_by<T>(ArrayIn<T>{in}, out, n, arena);
}

// ----------------------------- radix sort ---------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;  // per thread
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

__global__ void k_digit_hist(const uint64_t *keys, size_t n, int shift, uint32_t *hist,
                             uint32_t ntiles) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int i = 0; i < kSortItems; ++i) {
    size_t idx = base + (size_t)i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Shared memory of the scatter: the tile's keys (and values) in digit order,
// per-warp digit counters, and each digit's tile start and global offset.
template <typename V, bool kHasVals>
constexpr size_t scatter_smem() {
  return (size_t)kSortTile * sizeof(uint64_t) + (kHasVals ? (size_t)kSortTile * sizeof(V) : 0) +
         (size_t)(kSortWarps + 2) * kRadix * sizeof(uint32_t);
}

// Stable scatter of one tile.  Warp w owns elements [w*32*kSortItems, ...) of
// the tile in rounds of 32 consecutive elements, so tile order is preserved.
// The tile is first placed in shared memory in digit order; each digit's run
// is then written to its global position with consecutive threads on
// consecutive addresses.
template <typename V, bool kHasVals>
__global__ void __launch_bounds__(kSortThreads, 4)
    k_digit_scatter(const uint64_t *keys_in, const V *vals_in, uint64_t *keys_out, V *vals_out,
                    size_t n, int shift, const uint32_t *offsets, uint32_t ntiles) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sm);
  V *sv = reinterpret_cast<V *>(sk + kSortTile);
  uint32_t *wb = reinterpret_cast<uint32_t *>(sm + (size_t)kSortTile * sizeof(uint64_t) +
                                              (kHasVals ? (size_t)kSortTile * sizeof(V) : 0));
  uint32_t *dstart = wb + kSortWarps * kRadix;  // digit start within the tile
  uint32_t *dglob = dstart + kRadix;            // digit start in the output
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) wb[i] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kSortTile;
  const size_t wbase = base + (size_t)warp * 32 * kSortItems;
  // the tile's keys stay in registers (four CTAs of 256 threads per SM); a
  // key's digit is recomputed where it is needed, out-of-range slots get the
  // digit kRadix, which no counter holds
  uint64_t k[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const size_t idx = wbase + (size_t)r * 32 + lane;
    k[r] = idx < n ? keys_in[idx] : 0ull;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool ok = wbase + (size_t)r * 32 + lane < n;
    const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & 0xffu) : (uint32_t)kRadix;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == __ffs(peers) - 1) wb[warp * kRadix + d] += __popc(peers);
  }
  __syncthreads();
  {
    // per digit: offsets of the warps within the digit's run, the run's start
    // in the tile (scan over digits) and in the output
    const int dig = threadIdx.x;  // kSortThreads == kRadix
    uint32_t cnt = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wb[w * kRadix + dig];
      wb[w * kRadix + dig] = cnt;
      cnt += c;
    }
    dstart[dig] = block_exclusive_scan<uint32_t>(cnt, nullptr);
    dglob[dig] = offsets[(size_t)dig * ntiles + blockIdx.x];
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const size_t idx = wbase + (size_t)r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & 0xffu) : (uint32_t)kRadix;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t pos = 0;
    if (ok) pos = dstart[d] + wb[warp * kRadix + d] + __popc(peers & lt);
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wb[warp * kRadix + d] += __popc(peers);
    __syncwarp();
    if (ok) {
      sk[pos] = k[r];
      if (kHasVals) sv[pos] = vals_in[idx];
    }
  }
  __syncthreads();
  const uint32_t tn = (uint32_t)((n - base) < (size_t)kSortTile ? (n - base) : (size_t)kSortTile);
  for (uint32_t i = threadIdx.x; i < tn; i += kSortThreads) {
    const uint64_t key = sk[i];
    const uint32_t dg = (uint32_t)((key >> shift) & 0xffu);
    const uint32_t gpos = dglob[dg] + (i - dstart[dg]);
    keys_out[gpos] = key;
    if (kHasVals) vals_out[gpos] = sv[i];
  }
}

template <typename V, bool kHasVals>
int radix_sort_impl(uint64_t **keys, uint64_t **keys_alt, V **vals, V **vals_alt, size_t n,
                    int begin_bit, int end_bit, Arena &arena, const uint64_t *known_mask = nullptr) {
  if (n <= 1 || begin_bit >= end_bit) return ASCI_OK;
  if (n >= (1ull << 32)) return ASCI_EINVAL;
  cudaStream_t s = arena.stream();
  uint32_t ntiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
  uint32_t *hist = nullptr;
  ASCI_TRY(arena.alloc(&hist, (size_t)kRadix * ntiles));
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_digit_scatter<V, kHasVals>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)scatter_smem<V, kHasVals>());
  ASCI_TRY_CUDA(attr);
  uint64_t mask = 0;
  if (known_mask) mask = *known_mask;  // the caller knows which bits vary
  else ASCI_TRY(varying_bits_u64(*keys, n, &mask, arena));
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    uint64_t dmask = (0xffull << shift);
    if (end_bit - shift < 8) dmask &= ((end_bit >= 64) ? ~0ull : ((1ull << end_bit) - 1));
    if ((mask & dmask) == 0) continue;  // digit constant over the input
    k_digit_hist<<<ntiles, kSortThreads, 0, s>>>(*keys, n, shift, hist, ntiles);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY(scan_exclusive<uint32_t>(hist, hist, (size_t)kRadix * ntiles, arena));
    k_digit_scatter<V, kHasVals><<<ntiles, kSortThreads, scatter_smem<V, kHasVals>(), s>>>(
        *keys, kHasVals ? *vals : nullptr, *keys_alt, kHasVals ? *vals_alt : nullptr, n, shift,
        hist, ntiles);
    ASCI_CHECK_LAUNCH();
    uint64_t *t = *keys;
    *keys = *keys_alt;
    *keys_alt = t;
    if (kHasVals) {
      V *tv = *vals;
      *vals = *vals_alt;
      *vals_alt = tv;
    }
  }
  return ASCI_OK;
}

__global__ void k_varying(const uint64_t *keys, size_t n, unsigned long long *out) {
  uint64_t k0 = keys[0], acc = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    acc |= keys[i] ^ k0;
  for (int d = 16; d; d >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, (unsigned long long)acc);
}

}  // namespace

int scan_exclusive_u32(const uint32_t *in, uint32_t *out, size_t n, Arena &arena) {
  return scan_exclusive<uint32_t>(in, out, n, arena);
}
int scan_exclusive_u64(const uint64_t *in, uint64_t *out, size_t n, Arena &arena) {
  return scan_exclusive<uint64_t>(in, out, n, arena);
}

int scan_item_weights(const uint64_t *items, uint64_t T, int opbits, const uint32_t *grp_count,
                      const ExcCounts &X, uint64_t *Wexcl, Arena &arena) {
  ItemWeightIn in{items, grp_count, T, (uint64_t)X.sb + X.dbb, 1ull + X.sb,
                  (1u << opbits) - 1u, X.sa, opbits};
  return scan_exclusive_by<uint64_t>(in, Wexcl, (size_t)T + 1, arena);
}

int scan_item_heads(const uint64_t *items, uint64_t T, uint32_t *excl, Arena &arena) {
  return scan_exclusive_by<uint32_t>(ItemHeadIn{items, T}, excl, (size_t)T + 1, arena);
}

int varying_bits_u64(const uint64_t *keys, size_t n, uint64_t *host_mask, Arena &arena) {
  *host_mask = 0;
  if (n == 0) return ASCI_OK;
  unsigned long long *d = nullptr;
  ASCI_TRY(arena.alloc(&d, 1));
  cudaStream_t s = arena.stream();
  ASCI_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_varying<<<blocks, 256, 0, s>>>(keys, n, d);
  ASCI_CHECK_LAUNCH();
  unsigned long long h = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *host_mask = h;
  return ASCI_OK;
}

int radix_sort_u64(uint64_t **keys, uint64_t **keys_alt, size_t n, int begin_bit, int end_bit,
                   Arena &arena) {
  return radix_sort_impl<uint32_t, false>(keys, keys_alt, nullptr, nullptr, n, begin_bit, end_bit,
                                          arena);
}
int radix_sort_u64_varying(uint64_t **keys, uint64_t **keys_alt, size_t n, int begin_bit,
                           int end_bit, uint64_t varying, Arena &arena) {
  return radix_sort_impl<uint32_t, false>(keys, keys_alt, nullptr, nullptr, n, begin_bit, end_bit,
                                          arena, &varying);
}
int radix_sort_u64_u32(uint64_t **keys, uint64_t **keys_alt, uint32_t **vals, uint32_t **vals_alt,
                       size_t n, int begin_bit, int end_bit, Arena &arena) {
  return radix_sort_impl<uint32_t, true>(keys, keys_alt, vals, vals_alt, n, begin_bit, end_bit,
                                         arena);
}
int radix_sort_u64_f64(uint64_t **keys, uint64_t **keys_alt, double **vals, double **vals_alt,
                       size_t n, int begin_bit, int end_bit, Arena &arena) {
  return radix_sort_impl<double, true>(keys, keys_alt, vals, vals_alt, n, begin_bit, end_bit,
                                       arena);
}

}  // namespace asci
