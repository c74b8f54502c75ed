// Sort-and-accumulate (Sec. 2.2), the diagonal H_ii and the score of Eq. 1,
// exclusion of psi, and the top-N selection that replaces a full sort.
#include "asci_internal.cuh"

namespace asci {

namespace {

// ------------------------- segmented accumulate ----------------------------

__global__ void k_heads(const uint64_t *keys, size_t n, uint32_t *head) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_head_index(const uint32_t *head, const uint32_t *pos, size_t n,
                             uint32_t *head_idx) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (head[i]) head_idx[pos[i]] = (uint32_t)i;
}

// Sum of each run of equal keys, in input order (deterministic).
__global__ void k_segment_sum(const uint64_t *keys, const double *vals, size_t n,
                              const uint32_t *head_idx, size_t u, uint64_t *ukeys,
                              double *usums) {
  for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < u;
       s += (size_t)gridDim.x * blockDim.x) {
    size_t b = head_idx[s], e = (s + 1 < u) ? head_idx[s + 1] : n;
    double acc = 0.0;
    for (size_t i = b; i < e; ++i) acc += vals[i];
    ukeys[s] = keys[b];
    usums[s] = acc;
  }
}

// ------------------------------- diagonal ----------------------------------

__device__ double diag_value(const DevInts &I, uint32_t A, uint32_t B) {
  const int n = I.n;
  double s = I.ecore;
  for (uint32_t m = A; m; m &= m - 1) {
    const int p = __ffs(m) - 1;
    const double *jkp = I.jk + p * n, *jjp = I.jj + p * n;
    s += I.h1[p * n + p];
    for (uint32_t r = m & (m - 1); r; r &= r - 1) s += jkp[__ffs(r) - 1];
    for (uint32_t r = B; r; r &= r - 1) s += jjp[__ffs(r) - 1];
  }
  for (uint32_t m = B; m; m &= m - 1) {
    const int p = __ffs(m) - 1;
    const double *jkp = I.jk + p * n;
    s += I.h1[p * n + p];
    for (uint32_t r = m & (m - 1); r; r &= r - 1) s += jkp[__ffs(r) - 1];
  }
  return s;
}

__global__ void k_diag(DevInts I, const uint64_t *keys, size_t n, double *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    out[i] = diag_value(I, key_alpha(k), key_beta(k));
  }
}

template <typename T>
__global__ void k_compact(const T *in, const uint32_t *keep, const uint32_t *pos, size_t n,
                          T *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (keep[i]) out[pos[i]] = in[i];
}

// ------------------------------ selection ----------------------------------
//
// The rank of an entry is the 128-bit word R = (~bits(|S|), key): ascending R
// is |S| descending, then key ascending.  Keys are distinct, so R is too, and
// the top N are exactly the entries with R <= R_N.  R_N is found digit by digit
// from the most significant end (a radix select).

__device__ __forceinline__ void rank_words(uint64_t key, double s, uint64_t *hi, uint64_t *lo) {
  *hi = ~((uint64_t)__double_as_longlong(fabs(s)));
  *lo = key;
}

__global__ void k_select_hist(const uint64_t *keys, const double *scores, size_t n, int digit,
                              uint64_t pre_hi, uint64_t pre_lo, uint64_t m_hi, uint64_t m_lo,
                              unsigned long long *hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    uint64_t hi, lo;
    rank_words(keys[i], scores[i], &hi, &lo);
    if (((hi & m_hi) == pre_hi) && ((lo & m_lo) == pre_lo)) {
      uint32_t d = digit >= 8 ? (uint32_t)(hi >> ((digit - 8) * 8)) & 0xffu
                              : (uint32_t)(lo >> (digit * 8)) & 0xffu;
      atomicAdd(&h[d], 1u);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void k_select_flags(const uint64_t *keys, const double *scores, size_t n,
                               uint64_t t_hi, uint64_t t_lo, uint32_t *flag) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    uint64_t hi, lo;
    rank_words(keys[i], scores[i], &hi, &lo);
    flag[i] = (hi < t_hi || (hi == t_hi && lo <= t_lo)) ? 1u : 0u;
  }
}

inline unsigned grid_for(size_t n, unsigned cap = 152 * 16) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

int compact_u64(const uint64_t *in, const uint32_t *keep, const uint32_t *pos, size_t n,
                uint64_t *out, Arena &arena) {
  if (!n) return ASCI_OK;
  k_compact<uint64_t><<<grid_for(n), 256, 0, arena.stream()>>>(in, keep, pos, n, out);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

int compact_f64(const double *in, const uint32_t *keep, const uint32_t *pos, size_t n, double *out,
                Arena &arena) {
  if (!n) return ASCI_OK;
  k_compact<double><<<grid_for(n), 256, 0, arena.stream()>>>(in, keep, pos, n, out);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// Number of kept entries = pos[n-1] + keep[n-1] (host read).
int kept_count(const uint32_t *keep, const uint32_t *pos, size_t n, size_t *host_count,
               Arena &arena) {
  *host_count = 0;
  if (!n) return ASCI_OK;
  uint32_t h[2];
  cudaStream_t s = arena.stream();
  ASCI_TRY_CUDA(cudaMemcpyAsync(&h[0], pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(&h[1], keep + n - 1, 4, cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *host_count = (size_t)h[0] + h[1];
  return ASCI_OK;
}

int sort_accumulate(uint64_t **keys, uint64_t **keys_alt, double **vals, double **vals_alt,
                    size_t n, uint64_t *ukeys, double *usums, size_t *host_u, Arena &arena) {
  *host_u = 0;
  if (!n) return ASCI_OK;
  ASCI_TRY(radix_sort_u64_f64(keys, keys_alt, vals, vals_alt, n, 0, 64, arena));
  uint32_t *head, *pos, *head_idx;
  ASCI_TRY(arena.alloc(&head, n));
  ASCI_TRY(arena.alloc(&pos, n));
  cudaStream_t s = arena.stream();
  k_heads<<<grid_for(n), 256, 0, s>>>(*keys, n, head);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(head, pos, n, arena));
  size_t u = 0;
  ASCI_TRY(kept_count(head, pos, n, &u, arena));
  ASCI_TRY(arena.alloc(&head_idx, u));
  k_head_index<<<grid_for(n), 256, 0, s>>>(head, pos, n, head_idx);
  ASCI_CHECK_LAUNCH();
  k_segment_sum<<<grid_for(u), 256, 0, s>>>(*keys, *vals, n, head_idx, u, ukeys, usums);
  ASCI_CHECK_LAUNCH();
  *host_u = u;
  return ASCI_OK;
}

int diagonal_packed(const DevInts &I, const uint64_t *keys, size_t n, double *out, Arena &arena) {
  if (!n) return ASCI_OK;
  k_diag<<<grid_for(n), 256, 0, arena.stream()>>>(I, keys, n, out);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

int select_topn_packed(const uint64_t *keys, const double *scores, size_t n, size_t N,
                       uint64_t *out_keys, double *out_scores, size_t *host_out_n,
                       Arena &arena) {
  *host_out_n = 0;
  if (!n || !N) return ASCI_OK;
  cudaStream_t s = arena.stream();
  uint32_t *flag, *pos;
  ASCI_TRY(arena.alloc(&flag, n));
  ASCI_TRY(arena.alloc(&pos, n));
  uint64_t t_hi = ~0ull, t_lo = ~0ull;  // select everything when N >= n
  if (N < n) {
    unsigned long long *dhist;
    ASCI_TRY(arena.alloc(&dhist, 256));
    uint64_t pre_hi = 0, pre_lo = 0, m_hi = 0, m_lo = 0;
    uint64_t remaining = N;
    for (int digit = 15; digit >= 0; --digit) {
      ASCI_TRY_CUDA(cudaMemsetAsync(dhist, 0, 256 * sizeof(unsigned long long), s));
      k_select_hist<<<grid_for(n), 256, 0, s>>>(keys, scores, n, digit, pre_hi, pre_lo, m_hi,
                                                m_lo, dhist);
      ASCI_CHECK_LAUNCH();
      unsigned long long h[256];
      ASCI_TRY_CUDA(cudaMemcpyAsync(h, dhist, sizeof(h), cudaMemcpyDeviceToHost, s));
      ASCI_TRY_CUDA(cudaStreamSynchronize(s));
      uint64_t cum = 0;
      int d = 0;
      for (; d < 256; ++d) {
        if (cum + h[d] >= remaining) break;
        cum += h[d];
      }
      if (d == 256) return ASCI_ECUDA;  // inconsistent histogram
      remaining -= cum;
      uint64_t dv = (uint64_t)d;
      if (digit >= 8) {
        pre_hi |= dv << ((digit - 8) * 8);
        m_hi |= 0xffull << ((digit - 8) * 8);
      } else {
        pre_lo |= dv << (digit * 8);
        m_lo |= 0xffull << (digit * 8);
      }
      if (h[d] == remaining) {
        // the whole bucket is selected: threshold = prefix with all lower bits set
        t_hi = pre_hi | ~m_hi;
        t_lo = pre_lo | ~m_lo;
        break;
      }
      t_hi = pre_hi;
      t_lo = pre_lo;
    }
  }
  k_select_flags<<<grid_for(n), 256, 0, s>>>(keys, scores, n, t_hi, t_lo, flag);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(flag, pos, n, arena));
  size_t m = 0;
  ASCI_TRY(kept_count(flag, pos, n, &m, arena));
  ASCI_TRY(compact_u64(keys, flag, pos, n, out_keys, arena));
  ASCI_TRY(compact_f64(scores, flag, pos, n, out_scores, arena));
  *host_out_n = m;
  return ASCI_OK;
}

// Building blocks of a selection across ranks: the histogram of one byte of
// the rank word over the entries that match a prefix, and the entries at or
// below a rank threshold.
int select_histogram(const uint64_t *keys, const double *scores, size_t n, int digit,
                     const uint64_t pre[2], const uint64_t msk[2], uint64_t hist[256],
                     Arena &arena) {
  cudaStream_t s = arena.stream();
  unsigned long long *dhist;
  ASCI_TRY(arena.alloc(&dhist, 256));
  ASCI_TRY_CUDA(cudaMemsetAsync(dhist, 0, 256 * sizeof(unsigned long long), s));
  if (n) {
    k_select_hist<<<grid_for(n), 256, 0, s>>>(keys, scores, n, digit, pre[0], pre[1], msk[0],
                                              msk[1], dhist);
    ASCI_CHECK_LAUNCH();
  }
  ASCI_TRY_CUDA(cudaMemcpyAsync(hist, dhist, 256 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  return ASCI_OK;
}

int select_below(const uint64_t *keys, const double *scores, size_t n, const uint64_t thr[2],
                 uint64_t *out_keys, double *out_scores, size_t *host_out_n, Arena &arena) {
  *host_out_n = 0;
  if (!n) return ASCI_OK;
  cudaStream_t s = arena.stream();
  uint32_t *flag, *pos;
  ASCI_TRY(arena.alloc(&flag, n));
  ASCI_TRY(arena.alloc(&pos, n));
  k_select_flags<<<grid_for(n), 256, 0, s>>>(keys, scores, n, thr[0], thr[1], flag);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(flag, pos, n, arena));
  size_t m = 0;
  ASCI_TRY(kept_count(flag, pos, n, &m, arena));
  ASCI_TRY(compact_u64(keys, flag, pos, n, out_keys, arena));
  ASCI_TRY(compact_f64(scores, flag, pos, n, out_scores, arena));
  *host_out_n = m;
  return ASCI_OK;
}

}  // namespace asci
