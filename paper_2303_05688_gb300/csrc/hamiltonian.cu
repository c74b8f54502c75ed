// The variational step of the ASCI loop (Algorithm 1, "diagonalize the
// Hamiltonian in the selected determinant space"; Sec. 2.3).
//
//  * H over a determinant list (Sec. 2.3, CSR): the paper's double loop over
//    determinant pairs, pruned by the structure of the keys.  In key order
//    (beta word high) each beta string's determinants are one group; a row
//    visits only the groups whose beta string is within two excitations (a
//    group graph built by a tiled double loop over the beta strings), tests
//    the alpha distance against 4 - popc(beta_i ^ beta_j), and for groups a
//    beta double away looks its own alpha string up by binary search.
//    Connected pairs get H_ij by the Slater-Condon rules, evaluated 32 at a
//    time from a per-warp queue; nonzero elements are stored, each row's
//    columns ascending.  A counting pass and a scan give the row pointers, the
//    filling pass the elements; rows in the caller's order come from one sort
//    of the key-ordered entries.
//  * y = H x (Algorithm 6 on one device): a warp per row, lanes strided over
//    the row, a fixed shuffle tree: the same bits on every call.
//  * Davidson (Algorithm 5): basis V and products W = H V resident on the
//    device, the subspace matrix V^T H V grown one column per product, its
//    eigenpairs by parallel-order Jacobi in one CTA (FP32 sweeps refined by
//    FP64 sweeps), the shifted Jacobi
//    preconditioner, two passes of classical Gram-Schmidt, a thick restart
//    (the four lowest Ritz vectors) at the subspace limit.  Every reduction
//    has a fixed order.
//  * The ASCI loop itself: search, merge, build, diagonalise, repeat.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "asci_internal.cuh"

namespace asci {
namespace {

constexpr int kRowThreads = 256;   // rows per CTA of the build
constexpr int kColStage = 2048;    // column keys staged in shared memory at a time
constexpr int kMaxSub = 32;        // largest Davidson subspace (shared-memory Jacobi)
constexpr int kDotBlocks = 296;    // fixed partial-sum grid of the dot products
constexpr int kKeep = 4;           // Ritz vectors kept by a Davidson restart
constexpr int kDotThreads = 256;

inline unsigned blocks_for(size_t n, unsigned threads, unsigned cap = 152 * 16) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

// ------------------------------ validation ---------------------------------

enum : uint32_t { kBadRange = 1u, kBadCount = 2u, kDuplicate = 4u, kBadValue = 8u };

__global__ void k_det_keys(const asci_det *dets, size_t n, int norb, int na, int nb,
                           uint64_t *keys, unsigned *err) {
  const uint64_t hi = ~((1ull << norb) - 1ull);
  unsigned e = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const asci_det d = dets[i];
    if ((d.alpha & hi) || (d.beta & hi)) e |= kBadRange;
    if (__popcll(d.alpha) != na || __popcll(d.beta) != nb) e |= kBadCount;
    keys[i] = pack_key((uint32_t)d.alpha, (uint32_t)d.beta);
  }
  if (e) atomicOr(err, e);
}

__global__ void k_adjacent_equal(const uint64_t *sorted, size_t n, unsigned *err) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (sorted[i] == sorted[i - 1]) atomicOr(err, kDuplicate);
}

__global__ void k_finite(const double *x, size_t n, unsigned *err) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(err, kBadValue);
}

__global__ void k_keys_to_dets(const uint64_t *keys, size_t n, asci_det *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    asci_det d;
    d.alpha = key_alpha(keys[i]);
    d.beta = key_beta(keys[i]);
    out[i] = d;
  }
}

// ------------------------------ the build ----------------------------------

// <D_i|H|D_j> for distinct determinants within two excitations: the holes are
// the ket's orbitals missing from the bra, the particles the bra's orbitals
// missing from the ket, ascending.
__device__ double offdiag_element(const DevInts &I, uint32_t ai, uint32_t bi, uint32_t aj,
                                  uint32_t bj) {
  const uint32_t xa = ai ^ aj, xb = bi ^ bj;
  const int da = __popc(xa), db = __popc(xb);
  if (db == 0 && da == 2) {
    const int h = __ffs(aj & xa) - 1, p = __ffs(ai & xa) - 1;
    const double v = single_value(I, aj, bj, h, p);
    return single_parity(aj, h, p) ? -v : v;
  }
  if (da == 0 && db == 2) {
    const int h = __ffs(bj & xb) - 1, p = __ffs(bi & xb) - 1;
    const double v = single_value(I, bj, aj, h, p);
    return single_parity(bj, h, p) ? -v : v;
  }
  if (da == 2) {  // opposite-spin double
    const int ha = __ffs(aj & xa) - 1, pa = __ffs(ai & xa) - 1;
    const int hb = __ffs(bj & xb) - 1, pb = __ffs(bi & xb) - 1;
    const double v = eri4(I.eri, I.n, ha, pa, hb, pb);
    return (single_parity(aj, ha, pa) ^ single_parity(bj, hb, pb)) ? -v : v;
  }
  // same-spin double (da == 4 or db == 4)
  const uint32_t ket = da ? aj : bj, x = da ? xa : xb, bra = da ? ai : bi;
  uint32_t hm = ket & x, pm = bra & x;
  const int h1 = __ffs(hm) - 1;
  hm &= hm - 1;
  const int h2 = __ffs(hm) - 1;
  const int p1 = __ffs(pm) - 1;
  pm &= pm - 1;
  const int p2 = __ffs(pm) - 1;
  const double v = eri4(I.asym, I.n, h1, p1, h2, p2);
  return double_parity(ket, h1, h2, p1, p2) ? -v : v;
}

// The build works on determinants in key order (beta word high), so that
// every beta string's determinants form one contiguous group.  Two
// determinants are within two excitations iff
//   popc(alpha_i ^ alpha_j) + popc(beta_i ^ beta_j) <= 4,
// so a row only has to visit the groups whose beta string is within two
// excitations of its own (the group graph, built once per list by a tiled
// double loop over the G group strings), and inside such a group only the
// alpha test remains, with the threshold 4 - popc(beta_i ^ beta_j) (for beta
// strings a double apart, alpha_j must equal alpha_i: a binary search in the
// alpha-sorted group).  A warp takes a row and walks its neighbour groups in
// ascending order, 32 columns at a time; a ballot places the hits, so each
// row's columns come out ascending.  A counting pass gives the row lengths, a scan the row
// pointers, and the filling pass writes (never past a row's counted end).

// head[i] = 1 where a new beta string starts (keys sorted)
__global__ void k_beta_heads(const uint64_t *keys, uint32_t n, uint32_t *head) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    head[i] = (i == 0 || key_beta(keys[i]) != key_beta(keys[i - 1])) ? 1u : 0u;
}

// group of each row; start and beta string of each group (gid: exclusive scan of head)
__global__ void k_beta_groups(const uint64_t *keys, uint32_t n, const uint32_t *head,
                              const uint32_t *gid, uint32_t *of_row, uint32_t *gstart,
                              uint32_t *gbeta) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t g = gid[i] + head[i] - 1u;
    of_row[i] = g;
    if (head[i]) {
      gstart[g] = i;
      gbeta[g] = key_beta(keys[i]);
    }
    if (i == n - 1) gstart[g + 1] = n;  // end of the last group
  }
}

// Group graph: count (kFill false) or list (kFill true) the groups g2 with
// popc(beta_g1 ^ beta_g2) <= 4, for the groups g1 = [blockIdx.x * 256, +256)
// (one per thread) against the groups [blockIdx.y * chunk, +chunk) staged in
// shared memory.
template <bool kFill>
__global__ void __launch_bounds__(kRowThreads) k_beta_pairs(const uint32_t *gbeta, uint32_t G,
                                                            uint32_t chunk, uint32_t nchunks,
                                                            uint64_t *cnt_off, uint32_t *nbr) {
  __shared__ uint32_t sb[kColStage];
  const uint32_t g1 = blockIdx.x * kRowThreads + threadIdx.x;
  const bool live = g1 < G;
  const uint32_t b1 = live ? gbeta[g1] : 0u;
  const uint32_t c0 = blockIdx.y * chunk;
  const uint32_t c1 = min(G, c0 + chunk);
  const size_t slot = (size_t)g1 * nchunks + blockIdx.y;
  uint64_t cnt = 0, pos = 0, end = 0;
  if (kFill && live) {
    pos = cnt_off[slot];
    end = cnt_off[slot + 1];
  }
  for (uint32_t s = c0; s < c1; s += kColStage) {
    const uint32_t m = min((uint32_t)kColStage, c1 - s);
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < m; t += kRowThreads) sb[t] = gbeta[s + t];
    __syncthreads();
    if (!live) continue;
#pragma unroll 4
    for (uint32_t t = 0; t < m; ++t) {
      if (__popc(b1 ^ sb[t]) > 4) continue;
      if (kFill) {
        if (pos < end) nbr[pos] = s + t;
        ++pos;
      } else {
        ++cnt;
      }
    }
  }
  if (!kFill && live) cnt_off[slot] = cnt;
}

// Row lengths (kFill false: rp[r] = count) or elements (kFill true: rp holds
// the row pointers) of rows r = warp, warp + warps, ...  The diagonal is
// always stored; off-diagonal elements when nonzero.  The columns that pass
// the excitation test are queued in shared memory (in column order) and
// evaluated 32 at a time, one per lane, so that the Slater-Condon work runs
// on full warps rather than on the one or two lanes that hit in a step.
constexpr int kRowWarps = 8;

template <bool kFill>
__device__ __forceinline__ void flush_queue(const DevInts &I, const uint64_t *keys, uint32_t r,
                                            uint32_t ai, uint32_t bi, const double *diag,
                                            uint32_t *q, int k, uint32_t lane, uint32_t below,
                                            int64_t &pos, int64_t end, int64_t &cnt, int32_t *col,
                                            double *val) {
  double v = 0.0;
  uint32_t j = 0;
  bool nz = false;
  if ((int)lane < k) {
    j = q[lane];
    if (j == r) {
      v = diag[r];
      nz = true;
    } else {
      const uint64_t kj = keys[j];
      v = offdiag_element(I, ai, bi, key_alpha(kj), key_beta(kj));
      nz = v != 0.0;
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, nz);
  if (kFill) {
    if (nz) {
      const int64_t p = pos + __popc(bal & below);
      if (p < end) {
        col[p] = (int32_t)j;
        val[p] = v;
      }
    }
    pos += __popc(bal);
  } else {
    cnt += __popc(bal);
  }
}

template <bool kFill>
__global__ void __launch_bounds__(kRowWarps * 32) k_ham_rows(
    DevInts I, const uint64_t *__restrict__ keys, uint32_t n, const uint32_t *__restrict__ of_row,
    const uint32_t *__restrict__ gstart, const uint32_t *__restrict__ gbeta,
    const int64_t *__restrict__ nbr_ptr, const uint32_t *__restrict__ nbr,
    const double *__restrict__ diag, int64_t *rp, int32_t *col, double *val) {
  __shared__ uint32_t queue[kRowWarps][64];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t below = (1u << lane) - 1u;
  uint32_t *q = queue[threadIdx.x >> 5];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const uint64_t ki = keys[r];
    const uint32_t ai = key_alpha(ki), bi = key_beta(ki);
    const uint32_t g = of_row[r];
    int64_t pos = 0, end = 0, cnt = 0;
    if (kFill) {
      pos = rp[r];
      end = rp[r + 1];
    }
    int qn = 0;  // queued columns (warp-uniform, < 64)
    // 32 neighbour groups at a time: lane k holds group k's first column,
    // length and alpha threshold; their columns are walked as one
    // concatenated range, 32 columns per step, each lane finding its group
    // by a binary search over the lanes' offsets
    const int64_t e1 = nbr_ptr[g + 1];
    for (int64_t e0 = nbr_ptr[g]; e0 < e1; e0 += 32) {
      uint32_t gs = 0, len = 0;
      int thr = -1;
      if (e0 + lane < e1) {
        const uint32_t g2 = nbr[e0 + lane];
        gs = gstart[g2];
        len = gstart[g2 + 1] - gs;
        thr = 4 - __popc(bi ^ gbeta[g2]);
        if (thr == 0) {
          // beta strings a double apart: only alpha_j == alpha_i connects, and
          // the group is sorted by alpha, so one binary search replaces the
          // walk (the group becomes that one column, or nothing)
          uint32_t lo = gs, hi = gs + len;
          while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (key_alpha(keys[mid]) < ai) lo = mid + 1;
            else hi = mid;
          }
          const bool found = lo < gs + len && key_alpha(keys[lo]) == ai;
          gs = lo;
          len = found ? 1u : 0u;
        }
      }
      uint32_t off = len;  // inclusive scan of the lengths
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, off, o);
        if ((int)lane >= o) off += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, off, 31);
      off -= len;  // exclusive
      for (uint32_t c = 0; c < total; c += 32) {
        const uint32_t idx = c + lane;
        int k = 0;  // the last lane whose offset is <= idx
        for (int step = 16; step; step >>= 1) {
          const uint32_t o2 = __shfl_sync(0xffffffffu, off, k + step);
          if (o2 <= idx) k += step;
        }
        const uint32_t j = __shfl_sync(0xffffffffu, gs, k) + (idx - __shfl_sync(0xffffffffu, off, k));
        const int t = __shfl_sync(0xffffffffu, thr, k);
        const bool hit = idx < total && __popc(ai ^ key_alpha(keys[idx < total ? j : r])) <= t;
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) q[qn + __popc(bal & below)] = j;
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
          flush_queue<kFill>(I, keys, r, ai, bi, diag, q, 32, lane, below, pos, end, cnt, col,
                             val);
          const uint32_t rest = (lane + 32 < (uint32_t)qn) ? q[lane + 32] : 0u;
          __syncwarp();
          if (lane + 32 < (uint32_t)qn) q[lane] = rest;
          qn -= 32;
          __syncwarp();
        }
      }
    }
    if (qn > 0)
      flush_queue<kFill>(I, keys, r, ai, bi, diag, q, qn, lane, below, pos, end, cnt, col, val);
    __syncwarp();
    if (!kFill && lane == 0) rp[r] = cnt;
  }
}

__global__ void k_row_ptr(const uint64_t *off, uint32_t n, uint32_t nchunks, int64_t *row_ptr) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    row_ptr[i] = (int64_t)off[(size_t)i * nchunks];
}

// Remapping a key-ordered CSR to the caller's order: perm[r] is the caller's
// index of key-ordered row r.
__global__ void k_user_counts(const int64_t *rp, const uint32_t *perm, uint32_t n,
                              int64_t *cnt_user) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    cnt_user[perm[r]] = rp[r + 1] - rp[r];
}

__global__ void k_user_entries(const int64_t *rp, const int32_t *col, const uint32_t *perm,
                               uint32_t n, uint64_t *ekey) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const uint64_t u = (uint64_t)perm[r] << 32;
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      const uint32_t c = (uint32_t)col[k];
      ekey[k] = u | (c < n ? perm[c] : 0xffffffffu);
    }
  }
}

__global__ void k_low_cols(const uint64_t *ekey, size_t nnz, int32_t *col) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (size_t)gridDim.x * blockDim.x)
    col[k] = (int32_t)(uint32_t)ekey[k];
}

__global__ void k_iota(uint32_t *v, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = i;
}

__global__ void k_not_identity(const uint32_t *perm, uint32_t n, unsigned *flag) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (perm[i] != i) *flag = 1u;
}

struct HamGeom {
  uint32_t gx, gy, chunk;
};

// Rows in CTAs of 256; columns split so that the grid holds about 8 CTAs per
// SM (a slice never narrower than one shared-memory stage).
HamGeom ham_geom(uint32_t n) {
  HamGeom g;
  g.gx = (n + kRowThreads - 1) / kRowThreads;
  uint32_t want = (152u * 8u + g.gx - 1) / g.gx;
  const uint32_t most = (n + kColStage - 1) / kColStage;
  want = std::max(1u, std::min(want, most));
  g.chunk = (n + want - 1) / want;
  g.gy = (n + g.chunk - 1) / g.chunk;
  return g;
}

// ------------------------------ products -----------------------------------

__global__ void k_spmv(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const double *__restrict__ val, uint32_t n, const double *__restrict__ x,
                       double *__restrict__ y) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int64_t b = rp[r], e = rp[r + 1];
    double s = 0.0;
#pragma unroll 4
    for (int64_t k = b + lane; k < e; k += 32) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] = s;
  }
}

// out[k * s1] (and out2[k * s2] when given) = V_k . b for k = blockIdx.y
// (V_k = V + k * ld).  Each block writes the partial sum of its slice; the
// last block of a vector to finish (a ticket counter, reset by that block)
// adds the partials in block order, so the result does not depend on which
// block finishes last.
__global__ void __launch_bounds__(kDotThreads) k_dots(const double *V, size_t ld,
                                                      const double *b, size_t n, double *part,
                                                      unsigned *ticket, double *out, int s1,
                                                      double *out2, int s2) {
  __shared__ double red[kDotThreads / 32];
  __shared__ bool last;
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = (size_t)blockIdx.x * per, hi = min(n, lo + per);
  const int k = blockIdx.y;
  const double *v = V + (size_t)k * ld;
  double s = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += kDotThreads) s = fma(v[i], b[i], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += red[w];
    part[(size_t)k * gridDim.x + blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(ticket + k, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  const volatile double *pk = part + (size_t)k * gridDim.x;
  double t = 0.0;
  for (unsigned g = threadIdx.x; g < gridDim.x; g += 32) t += pk[g];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) {
    out[(size_t)k * s1] = t;
    if (out2) out2[(size_t)k * s2] = t;
    ticket[k] = 0u;
  }
}

// out = base * sb + sum_k coef[k] * sc * V_k (base nullable).
__global__ void k_combine(const double *V, size_t ld, int m, const double *coef, double sc,
                          const double *base, double sb, size_t n, double *out) {
  __shared__ double cf[kMaxSub];
  for (int k = threadIdx.x; k < m; k += blockDim.x) cf[k] = coef[k] * sc;
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double s = base ? base[i] * sb : 0.0;
    for (int k = 0; k < m; ++k) s = fma(cf[k], V[(size_t)k * ld + i], s);
    out[i] = s;
  }
}

// x = V c and wx = W c in one pass (c = the lowest Ritz vector's coefficients).
__global__ void k_ritz(const double *V, const double *W, size_t ld, int m, const double *coef,
                       size_t n, double *x, double *wx) {
  __shared__ double cf[kMaxSub];
  for (int k = threadIdx.x; k < m; k += blockDim.x) cf[k] = coef[k];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < m; ++k) {
      a = fma(cf[k], V[(size_t)k * ld + i], a);
      b = fma(cf[k], W[(size_t)k * ld + i], b);
    }
    x[i] = a;
    wx[i] = b;
  }
}

// r = wx - theta * x; t = r / (theta - H_ii) with the denominator kept at
// least 1e-8 in magnitude (or t = r when unpreconditioned).
__global__ void k_residual(const double *wx, const double *x, const double *theta,
                           const double *diag, size_t n, bool precondition, double *r,
                           double *t) {
  const double th = *theta;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double ri = fma(-th, x[i], wx[i]);
    r[i] = ri;
    if (precondition) {
      double d = th - diag[i];
      if (fabs(d) < 1e-8) d = d < 0.0 ? -1e-8 : 1e-8;
      t[i] = ri / d;
    } else {
      t[i] = ri;
    }
  }
}

// v *= 1 / sqrt(*norm2)
__global__ void k_normalize(double *v, size_t n, const double *norm2) {
  const double s = 1.0 / sqrt(*norm2);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

// All eigenpairs of the symmetric m x m matrix Hs (leading dimension ld) by
// Jacobi rotations in the parallel (round-robin) ordering (Brent and Luk,
// 1985; Golub and Van Loan, Sec. 8.5): a sweep is M - 1 rounds (M = m rounded
// up to even; the extra index, when there is one, has no couplings), each
// round pairs every index with one other, so its M / 2 rotations act on
// disjoint planes.  One thread per pair forms its rotation from the round's
// matrix, then the CTA applies all of them to the columns (and to the
// eigenvector matrix), then to the rows.
//
// GB300 executes about 1.7 FP64 operations per clock per SM, against some 126
// FP32 ones, so the sweeps run in two precisions: FP32 sweeps take the matrix
// to near-diagonal form (off-diagonal norm below 1e-6 of the diagonal's); the
// FP32 eigenvectors, promoted to FP64 and orthonormalised by two passes of
// classical Gram-Schmidt, transform Hs in FP64 (Q^T Hs Q, an exact similarity
// up to rounding); FP64 sweeps then finish (off-diagonal norm below 1e-13 of
// the diagonal's, one or two sweeps by quadratic convergence), accumulating
// into the same eigenvectors.  out: theta[r] in ascending order (ties by
// index), eigenvector r in Ct[r * kMaxSub + k].
constexpr int kEigThreads = 256;

// 1/sqrt(x) to FP64 accuracy from the FP32 estimate rsqrtf and two
// Newton-Raphson steps y <- y(3 - xy^2)/2 (2^-23 -> 2^-92), for x in
// [1e-30, 1e30]; with recip_fast it avoids the FP64 division and square-root
// sequences.
__device__ __forceinline__ double rsqrt_fast(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y * fma(-0.5 * x, y * y, 1.5);
}

// The Jacobi rotation (c, s) that zeroes a_pq: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c
// (Golub and Van Loan, Alg. 8.5.1), with the fast reciprocals when every
// operand is in their range and the exact operations otherwise.
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double *c,
                                         double *s) {
  const double d = aqq - app, a2 = 2.0 * apq;
  const bool fast = fabs(a2) > 1e-30 && fabs(a2) < 1e30 && fabs(d) < 1e15 * fabs(a2);
  double t;
  if (fast) {
    const double tau = d * recip_fast(a2);  // |tau| < 1e15
    const double y = fma(tau, tau, 1.0);
    const double den = fabs(tau) + y * rsqrt_fast(y);  // in [1, 2e15]
    t = (tau >= 0.0 ? 1.0 : -1.0) * recip_fast(den);
  } else {
    const double tau = d / a2;
    t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  }
  const double cs = rsqrt_fast(fma(t, t, 1.0));  // 1 + t^2 in [1, 2]
  *c = cs;
  *s = t * cs;
}

// The FP32 rotation of the same formulas (IEEE FP32 division and square root).
__device__ __forceinline__ void rotation_f(float app, float aqq, float apq, float *c, float *s) {
  const float tau = (aqq - app) / (2.0f * apq);
  const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
  const float cs = 1.0f / sqrtf(fmaf(t, t, 1.0f));
  *c = cs;
  *s = t * cs;
}

constexpr int kEigPer = (kMaxSub * kMaxSub + kEigThreads - 1) / kEigThreads;

struct EigScratch {
  int rp[kMaxSub / 2], rq[kMaxSub / 2];
  double rc[kMaxSub / 2], rs[kMaxSub / 2];
  double red[2][kEigThreads / 32];
  int done;
};

// Parallel-order Jacobi sweeps on A (symmetric, m x m) accumulating into Q,
// until the off-diagonal norm is at most sqrt(thr) of the diagonal's or after
// max_sweeps.  T is float or double; every thread of the CTA calls it.
template <typename T>
__device__ void jacobi_sweeps(T (*A)[kMaxSub + 1], T (*Q)[kMaxSub + 1], int m, int max_sweeps,
                              double thr, EigScratch &E) {
  const int tid = threadIdx.x;
  const int M = m + (m & 1);
  const int half = M / 2;
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int e = tid; e < m * m; e += kEigThreads) {
      const int i = e / m, k = e - (e / m) * m;
      const double a = (double)A[i][k];
      if (i == k) dg += a * a;
      else off += a * a;
    }
    for (int o = 16; o; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    if ((tid & 31) == 0) {
      E.red[0][tid >> 5] = off;
      E.red[1][tid >> 5] = dg;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, sd = 0.0;
      for (int w = 0; w < kEigThreads / 32; ++w) {
        so += E.red[0][w];
        sd += E.red[1][w];
      }
      E.done = so <= thr * sd;
    }
    __syncthreads();
    if (E.done) break;
    for (int r = 0; r < M - 1; ++r) {
      if (tid < half) {
        const int pa = tid == 0 ? 0 : 1 + (tid - 1 + r) % (M - 1);
        const int pb = 1 + (M - 2 - tid + r) % (M - 1);
        const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        double cs = 1.0, sn = 0.0;
        if (q < m) {
          if (sizeof(T) == sizeof(float)) {
            const float apq = (float)A[p][q];
            if (fabsf(apq) >= 1e-30f) {
              float c, s;
              rotation_f((float)A[p][p], (float)A[q][q], apq, &c, &s);
              cs = c;
              sn = s;
            }
          } else {
            const double apq = (double)A[p][q];
            if (fabs(apq) >= 1e-300) rotation((double)A[p][p], (double)A[q][q], apq, &cs, &sn);
          }
        }
        E.rc[tid] = cs;
        E.rs[tid] = sn;
        E.rp[tid] = p;
        E.rq[tid] = q;
      }
      __syncthreads();
      for (int e = tid; e < half * m; e += kEigThreads) {  // columns p, q of A and Q
        const int k = e / m, i = e - (e / m) * m;
        const int p = E.rp[k], q = E.rq[k];
        if (q >= m || E.rs[k] == 0.0) continue;
        const T cs = (T)E.rc[k], sn = (T)E.rs[k];
        const T aip = A[i][p], aiq = A[i][q];
        A[i][p] = cs * aip - sn * aiq;
        A[i][q] = sn * aip + cs * aiq;
        const T qip = Q[i][p], qiq = Q[i][q];
        Q[i][p] = cs * qip - sn * qiq;
        Q[i][q] = sn * qip + cs * qiq;
      }
      __syncthreads();
      for (int e = tid; e < half * m; e += kEigThreads) {  // rows p, q of A
        const int k = e / m, j = e - (e / m) * m;
        const int p = E.rp[k], q = E.rq[k];
        if (q >= m || E.rs[k] == 0.0) continue;
        const T cs = (T)E.rc[k], sn = (T)E.rs[k];
        const T apj = A[p][j], aqj = A[q][j];
        A[p][j] = cs * apj - sn * aqj;
        A[q][j] = sn * apj + cs * aqj;
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kEigThreads) k_small_eig(const double *Hs, int ld, int m,
                                                           double *theta, double *Ct) {
  __shared__ double A[kMaxSub][kMaxSub + 1];
  __shared__ double Q[kMaxSub][kMaxSub + 1];
  __shared__ float Af[kMaxSub][kMaxSub + 1];
  __shared__ float Qf[kMaxSub][kMaxSub + 1];
  __shared__ double gsr[kMaxSub];
  __shared__ double nrm;
  __shared__ EigScratch E;
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += kEigThreads) {
    const int i = e / m, k = e - (e / m) * m;
    Af[i][k] = (float)Hs[(size_t)i * ld + k];
    Qf[i][k] = (i == k) ? 1.0f : 0.0f;
  }
  __syncthreads();
  jacobi_sweeps<float>(Af, Qf, m, 16, 1e-12, E);
  for (int e = tid; e < m * m; e += kEigThreads) {
    const int i = e / m, k = e - (e / m) * m;
    Q[i][k] = (double)Qf[i][k];
  }
  __syncthreads();
  // orthonormal columns in FP64: two passes of classical Gram-Schmidt each
  for (int k = 0; k < m; ++k) {
    for (int pass = 0; pass < 2; ++pass) {
      if (tid < k) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t = fma(Q[i][tid], Q[i][k], t);
        gsr[tid] = t;
      }
      __syncthreads();
      if (tid < m) {
        double t = Q[tid][k];
        for (int j = 0; j < k; ++j) t = fma(-gsr[j], Q[tid][j], t);
        Q[tid][k] = t;
      }
      __syncthreads();
    }
    if (tid < 32) {
      double v = tid < m ? Q[tid][k] * Q[tid][k] : 0.0;
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (tid == 0) nrm = v;
    }
    __syncthreads();
    if (tid < m) Q[tid][k] *= rsqrt_fast(nrm);
    __syncthreads();
  }
  // A = Q^T Hs Q, through A = Hs Q and registers
  for (int e = tid; e < m * m; e += kEigThreads) {
    const int i = e / m, j = e - (e / m) * m;
    double t = 0.0;
    for (int l = 0; l < m; ++l) t = fma(Hs[(size_t)i * ld + l], Q[l][j], t);
    A[i][j] = t;
  }
  __syncthreads();
  double keep[kEigPer];
  for (int u = 0; u < kEigPer; ++u) {
    const int e = tid + u * kEigThreads;
    double t = 0.0;
    if (e < m * m) {
      const int i = e / m, j = e - (e / m) * m;
      for (int k = 0; k < m; ++k) t = fma(Q[k][i], A[k][j], t);
    }
    keep[u] = t;
  }
  __syncthreads();
  for (int u = 0; u < kEigPer; ++u) {
    const int e = tid + u * kEigThreads;
    if (e < m * m) A[e / m][e - (e / m) * m] = keep[u];
  }
  __syncthreads();
  jacobi_sweeps<double>(A, Q, m, 8, 1e-26, E);
  for (int i = tid; i < m; i += kEigThreads) {
    const double d = A[i][i];
    int rk = 0;
    for (int j = 0; j < m; ++j) rk += (A[j][j] < d) || (A[j][j] == d && j < i);
    theta[rk] = d;
    for (int k = 0; k < m; ++k) Ct[(size_t)rk * kMaxSub + k] = Q[k][i];
  }
}

// Hs = diag(theta[0..K)) after a restart.
__global__ void k_restart_hs(double *Hs, const double *theta, int K) {
  for (int e = threadIdx.x; e < kMaxSub * kMaxSub; e += blockDim.x) {
    const int i = e / kMaxSub, k = e - (e / kMaxSub) * kMaxSub;
    Hs[e] = (i == k && i < K) ? theta[i] : 0.0;
  }
}

// Largest |v_i| (lowest index among equal magnitudes): per-block candidates,
// then one block reduces them and flips the vector's sign if that entry is
// negative.
__global__ void k_absmax_part(const double *v, size_t n, double *bval, unsigned long long *bidx) {
  __shared__ double sv[256];
  __shared__ unsigned long long si[256];
  double best = -1.0;
  unsigned long long bi = ~0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double a = fabs(v[i]);
    if (a > best) {  // strided ascending: first index wins among equals
      best = a;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = 128; s; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const unsigned long long oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bval[blockIdx.x] = sv[0];
    bidx[blockIdx.x] = si[0];
  }
}

__global__ void k_absmax_sign(const double *bval, const unsigned long long *bidx, int nb,
                              const double *v, double *sign) {
  if (threadIdx.x != 0) return;
  double best = -1.0;
  unsigned long long bi = ~0ull;
  for (int b = 0; b < nb; ++b)
    if (bval[b] > best || (bval[b] == best && bidx[b] < bi)) {
      best = bval[b];
      bi = bidx[b];
    }
  *sign = (bi != ~0ull && v[bi] < 0.0) ? -1.0 : 1.0;
}

__global__ void k_scale_by(double *v, size_t n, const double *s) {
  const double f = *s;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] *= f;
}

__global__ void k_unit(double *v, size_t n, const double *diag) {
  // e_{argmin H_ii}, lowest index among equal values (one block scans)
  __shared__ double sv[256];
  __shared__ unsigned long long si[256];
  double best = INFINITY;
  unsigned long long bi = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x)
    if (diag[i] < best) {
      best = diag[i];
      bi = i;
    }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = 128; s; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const unsigned long long oi = si[threadIdx.x + s];
      if (o < sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = (i == si[0]) ? 1.0 : 0.0;
}

__global__ void k_csr_diag(const int64_t *rp, const int32_t *col, const double *val, uint32_t n,
                           double *diag) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
      if (col[k] == (int32_t)r) {
        d = val[k];
        break;
      }
    diag[r] = d;
  }
}

// Number of keys of a[n] absent from the sorted list b[m] (binary search).
__global__ void k_count_missing(const uint64_t *a, size_t n, const uint64_t *b, size_t m,
                                unsigned long long *cnt) {
  unsigned long long c = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t k = a[i];
    size_t lo = 0, hi = m;
    while (lo < hi) {
      const size_t mid = (lo + hi) >> 1;
      if (b[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    c += (lo == m || b[lo] != k);
  }
  if (c) atomicAdd(cnt, c);
}

__global__ void k_pack_dets(const asci_det *d, size_t n, uint64_t *keys) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    keys[i] = pack_key((uint32_t)d[i].alpha, (uint32_t)d[i].beta);
}

}  // namespace

// ------------------------------ host side ----------------------------------

struct Csr {
  const int64_t *row_ptr;
  const int32_t *col;
  const double *val;
  size_t n;
};

// Beta groups of key-ordered determinants and their neighbour graph.
struct BetaGraph {
  uint32_t G = 0;
  uint32_t *of_row = nullptr, *gstart = nullptr, *gbeta = nullptr, *nbr = nullptr;
  int64_t *nbr_ptr = nullptr;
};

static int beta_graph(const uint64_t *keys, uint32_t n, BetaGraph *bg, Arena &arena) {
  cudaStream_t s = arena.stream();
  uint32_t *head, *gid;
  ASCI_TRY(arena.alloc(&head, n));
  ASCI_TRY(arena.alloc(&gid, n));
  k_beta_heads<<<blocks_for(n, 256), 256, 0, s>>>(keys, n, head);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u32(head, gid, n, arena));
  uint32_t last[2];
  ASCI_TRY_CUDA(cudaMemcpyAsync(&last[0], gid + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(&last[1], head + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  const uint32_t G = last[0] + last[1];
  ASCI_TRY(arena.alloc(&bg->of_row, n));
  ASCI_TRY(arena.alloc(&bg->gstart, (size_t)G + 1));
  ASCI_TRY(arena.alloc(&bg->gbeta, G));
  k_beta_groups<<<blocks_for(n, 256), 256, 0, s>>>(keys, n, head, gid, bg->of_row, bg->gstart,
                                                    bg->gbeta);
  ASCI_CHECK_LAUNCH();
  // the group graph: count, scan, list
  const HamGeom g = ham_geom(G);
  const size_t slots = (size_t)G * g.gy;
  uint64_t *off;
  ASCI_TRY(arena.alloc(&off, slots + 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(off + slots, 0, sizeof(uint64_t), s));
  k_beta_pairs<false><<<dim3(g.gx, g.gy), kRowThreads, 0, s>>>(bg->gbeta, G, g.chunk, g.gy, off,
                                                                nullptr);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u64(off, off, slots + 1, arena));
  ASCI_TRY(arena.alloc(&bg->nbr_ptr, (size_t)G + 1));
  k_row_ptr<<<blocks_for((size_t)G + 1, 256), 256, 0, s>>>(off, G, g.gy, bg->nbr_ptr);
  ASCI_CHECK_LAUNCH();
  uint64_t total = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&total, off + slots, sizeof(total), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  ASCI_TRY(arena.alloc(&bg->nbr, total));
  k_beta_pairs<true><<<dim3(g.gx, g.gy), kRowThreads, 0, s>>>(bg->gbeta, G, g.chunk, g.gy, off,
                                                               bg->nbr);
  ASCI_CHECK_LAUNCH();
  bg->G = G;
  return ASCI_OK;
}

static unsigned row_blocks(uint32_t n) {
  return blocks_for((size_t)n * 32, kRowWarps * 32, 152 * 16);
}

// Counting pass and row pointers (rp[n + 1], device) of key-ordered keys.
static int ham_count(const DevInts &I, const uint64_t *keys, uint32_t n, const double *diag,
                     const BetaGraph &bg, int64_t *rp, size_t *nnz, Arena &arena) {
  cudaStream_t s = arena.stream();
  ASCI_TRY_CUDA(cudaMemsetAsync(rp + n, 0, sizeof(int64_t), s));
  k_ham_rows<false><<<row_blocks(n), kRowWarps * 32, 0, s>>>(I, keys, n, bg.of_row, bg.gstart, bg.gbeta,
                                                   bg.nbr_ptr, bg.nbr, diag, rp, nullptr,
                                                   nullptr);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(scan_exclusive_u64(reinterpret_cast<uint64_t *>(rp), reinterpret_cast<uint64_t *>(rp),
                              (size_t)n + 1, arena));
  int64_t total = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&total, rp + n, sizeof(total), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *nnz = (size_t)total;
  return ASCI_OK;
}

static int ham_fill(const DevInts &I, const uint64_t *keys, uint32_t n, const double *diag,
                    const BetaGraph &bg, int64_t *rp, int32_t *col, double *val, Arena &arena) {
  k_ham_rows<true><<<row_blocks(n), kRowWarps * 32, 0, arena.stream()>>>(I, keys, n, bg.of_row, bg.gstart,
                                                              bg.gbeta, bg.nbr_ptr, bg.nbr, diag,
                                                              rp, col, val);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

static int spmv(const Csr &H, const double *x, double *y, cudaStream_t s) {
  if (!H.n) return ASCI_OK;
  k_spmv<<<blocks_for(H.n * 32, 256, 152 * 32), 256, 0, s>>>(H.row_ptr, H.col, H.val,
                                                             (uint32_t)H.n, x, y);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// out[k * s1] (and out2[k * s2]) = V_k . b for k < m
// Scratch of the dot products: partial sums and the per-vector tickets (zero
// between calls).
struct DotScratch {
  double *part;
  unsigned *ticket;
};

static int dot_scratch(DotScratch *d, Arena &arena) {
  ASCI_TRY(arena.alloc(&d->part, (size_t)kMaxSub * kDotBlocks));
  ASCI_TRY(arena.alloc(&d->ticket, kMaxSub));
  ASCI_TRY_CUDA(cudaMemsetAsync(d->ticket, 0, kMaxSub * sizeof(unsigned), arena.stream()));
  return ASCI_OK;
}

static int dots(const double *V, size_t ld, int m, const double *b, size_t n,
                const DotScratch &d, double *out, int s1, double *out2, int s2, cudaStream_t s) {
  const int nblk = (int)std::min<size_t>(kDotBlocks, std::max<size_t>(1, (n + 1023) / 1024));
  k_dots<<<dim3(nblk, m), kDotThreads, 0, s>>>(V, ld, b, n, d.part, d.ticket, out, s1, out2, s2);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

struct DavidsonResult {
  double energy = 0.0, residual = 0.0;
  int iterations = 0;
  bool converged = false;
};

// Algorithm 5 on one device (see the file comment); vec receives the unit Ritz
// vector with its largest component positive.
static int davidson(const Csr &H, const double *diag, const double *guess,
                    const asci_davidson_opts &o, double *vec, DavidsonResult *res, Arena &arena) {
  cudaStream_t s = arena.stream();
  const size_t n = H.n;
  const int mmax = (int)std::min<size_t>((size_t)o.max_subspace, n);
  const unsigned gb = blocks_for(n, 256);
  const int keep = std::min(kKeep, mmax - 1);  // Ritz vectors kept at a restart
  double *V, *W, *Hs, *Ct, *th, *h, *sc, *x, *wx, *r, *t, *TV = nullptr, *TW = nullptr;
  DotScratch part;
  ASCI_TRY(arena.alloc(&V, (size_t)std::max(mmax, 1) * n));
  ASCI_TRY(arena.alloc(&W, (size_t)std::max(mmax, 1) * n));
  if (keep > 0) {
    ASCI_TRY(arena.alloc(&TV, (size_t)keep * n));
    ASCI_TRY(arena.alloc(&TW, (size_t)keep * n));
  }
  ASCI_TRY(arena.alloc(&Hs, (size_t)kMaxSub * kMaxSub));
  ASCI_TRY(arena.alloc(&Ct, (size_t)kMaxSub * kMaxSub));
  ASCI_TRY(arena.alloc(&th, kMaxSub));
  ASCI_TRY(arena.alloc(&h, kMaxSub));
  ASCI_TRY(dot_scratch(&part, arena));
  ASCI_TRY(arena.alloc(&sc, 8));  // scratch, |r|^2, |t|^2, sign
  ASCI_TRY(arena.alloc(&x, n));
  ASCI_TRY(arena.alloc(&wx, n));
  ASCI_TRY(arena.alloc(&r, n));
  ASCI_TRY(arena.alloc(&t, n));
  ASCI_TRY_CUDA(cudaMemsetAsync(Hs, 0, sizeof(double) * kMaxSub * kMaxSub, s));
  // v0: the guess, or the unit vector of the smallest H_ii; normalised
  if (guess) {
    ASCI_TRY_CUDA(cudaMemcpyAsync(V, guess, n * sizeof(double), cudaMemcpyDefault, s));
  } else {
    k_unit<<<1, 256, 0, s>>>(V, n, diag);
    ASCI_CHECK_LAUNCH();
  }
  ASCI_TRY(dots(V, n, 1, V, n, part, sc + 2, 1, nullptr, 0, s));
  double g2 = 0.0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&g2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (!(g2 > 0.0) || !std::isfinite(g2)) {
    record_error("Davidson guess is zero or not finite", __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  k_normalize<<<gb, 256, 0, s>>>(V, n, sc + 2);
  ASCI_CHECK_LAUNCH();
  int m = 1;         // basis vectors in V
  int have_w = 0;    // products already in W
  bool first = true;
  double theta = 0.0, rn = 0.0;
  for (;;) {
    // products of the new basis vectors and their column of V^T H V
    for (; have_w < m; ++have_w) {
      ASCI_TRY(spmv(H, V + (size_t)have_w * n, W + (size_t)have_w * n, s));
      ++res->iterations;
      ASCI_TRY(dots(V, n, have_w + 1, W + (size_t)have_w * n, n, part, Hs + have_w, kMaxSub,
                    Hs + (size_t)have_w * kMaxSub, 1, s));
    }
    k_small_eig<<<1, kEigThreads, 0, s>>>(Hs, kMaxSub, m, th, Ct);
    ASCI_CHECK_LAUNCH();
    k_ritz<<<gb, 256, 0, s>>>(V, W, n, m, Ct, n, x, wx);
    ASCI_CHECK_LAUNCH();
    k_residual<<<gb, 256, 0, s>>>(wx, x, th, diag, n, !first, r, t);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY(dots(r, n, 1, r, n, part, sc + 1, 1, nullptr, 0, s));
    // the next expansion vector is prepared before the convergence test is
    // read back, so that one host round trip serves both; when the test
    // stops the iteration, that work is simply dropped
    const bool restart = m == mmax && (size_t)m < n;
    if (restart) {  // thick restart: the `keep` lowest Ritz vectors and their products
      for (int k = 0; k < keep; ++k) {
        k_ritz<<<gb, 256, 0, s>>>(V, W, n, m, Ct + (size_t)k * kMaxSub, n, TV + (size_t)k * n,
                                  TW + (size_t)k * n);
        ASCI_CHECK_LAUNCH();
      }
      ASCI_TRY_CUDA(cudaMemcpyAsync(V, TV, (size_t)keep * n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
      ASCI_TRY_CUDA(cudaMemcpyAsync(W, TW, (size_t)keep * n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
      k_restart_hs<<<1, 256, 0, s>>>(Hs, th, keep);
      ASCI_CHECK_LAUNCH();
    }
    const int mb = restart ? keep : m;  // basis the correction is orthogonalised against
    for (int pass = 0; pass < 2; ++pass) {  // two passes of classical Gram-Schmidt
      ASCI_TRY(dots(V, n, mb, t, n, part, h, 1, nullptr, 0, s));
      k_combine<<<gb, 256, 0, s>>>(V, n, mb, h, -1.0, t, 1.0, n, t);
      ASCI_CHECK_LAUNCH();
    }
    ASCI_TRY(dots(t, n, 1, t, n, part, sc + 2, 1, nullptr, 0, s));
    double hs[3];
    ASCI_TRY_CUDA(cudaMemcpyAsync(&hs[0], th, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASCI_TRY_CUDA(cudaMemcpyAsync(&hs[1], sc + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    theta = hs[0];
    rn = std::sqrt(std::max(hs[1], 0.0));
    if (!std::isfinite(theta) || !std::isfinite(rn)) {
      record_error("Davidson produced a non-finite value", __FILE__, __LINE__);
      return ASCI_ECUDA;
    }
    if (rn <= o.tol || res->iterations >= o.max_iter || (size_t)m >= n) {
      res->converged = rn <= o.tol || (size_t)m >= n;
      break;
    }
    first = false;
    if (restart) {
      m = keep;
      have_w = keep;
    }
    if (!(hs[2] > 1e-28)) {  // the correction lies in the basis: nothing left to add
      res->converged = rn <= o.tol;
      break;
    }
    k_normalize<<<gb, 256, 0, s>>>(t, n, sc + 2);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY_CUDA(cudaMemcpyAsync(V + (size_t)m * n, t, n * sizeof(double),
                                  cudaMemcpyDeviceToDevice, s));
    ++m;
  }
  // unit Ritz vector, largest component positive
  {
    const int nb = (int)std::min<size_t>(296, std::max<size_t>(1, (n + 255) / 256));
    double *bval;
    unsigned long long *bidx;
    ASCI_TRY(arena.alloc(&bval, nb));
    ASCI_TRY(arena.alloc(&bidx, nb));
    ASCI_TRY(dots(x, n, 1, x, n, part, sc + 2, 1, nullptr, 0, s));
    k_normalize<<<gb, 256, 0, s>>>(x, n, sc + 2);
    ASCI_CHECK_LAUNCH();
    k_absmax_part<<<nb, 256, 0, s>>>(x, n, bval, bidx);
    ASCI_CHECK_LAUNCH();
    k_absmax_sign<<<1, 32, 0, s>>>(bval, bidx, nb, x, sc + 3);
    ASCI_CHECK_LAUNCH();
    k_scale_by<<<gb, 256, 0, s>>>(x, n, sc + 3);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY_CUDA(cudaMemcpyAsync(vec, x, n * sizeof(double), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  }
  res->energy = theta;
  res->residual = rn;
  return ASCI_OK;
}

static int check_davidson_opts(const asci_davidson_opts &o) {
  if (o.max_subspace < 2 || o.max_subspace > kMaxSub || o.max_iter < 1 || !(o.tol >= 0.0) ||
      !std::isfinite(o.tol))
    return ASCI_EINVAL;
  return ASCI_OK;
}

// Packed keys of a determinant list, validated (range, counts, duplicates);
// na / nb from the first determinant.
static int det_keys(const asci_det *dets, size_t n, int norb, uint64_t *keys, int *na, int *nb,
                    Arena &arena) {
  cudaStream_t s = arena.stream();
  asci_det d0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&d0, dets, sizeof(d0), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *na = __builtin_popcountll(d0.alpha);
  *nb = __builtin_popcountll(d0.beta);
  unsigned *err;
  uint64_t *sk, *sk_alt;
  ASCI_TRY(arena.alloc(&err, 1));
  ASCI_TRY(arena.alloc(&sk, n));
  ASCI_TRY(arena.alloc(&sk_alt, n));
  ASCI_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  k_det_keys<<<blocks_for(n, 256), 256, 0, s>>>(dets, n, norb, *na, *nb, keys, err);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(sk, keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  ASCI_TRY(radix_sort_u64(&sk, &sk_alt, n, 0, 64, arena));
  k_adjacent_equal<<<blocks_for(n, 256), 256, 0, s>>>(sk, n, err);
  ASCI_CHECK_LAUNCH();
  unsigned herr = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    record_error(herr & kDuplicate  ? "duplicate determinants"
                 : herr & kBadCount ? "determinants with different electron counts"
                                    : "determinant bits at or above norb",
                 __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  return ASCI_OK;
}

static int stage_tables(const asci_ints *ints, int na, int nb, Arena &arena, DevInts *I) {
  const size_t n = (size_t)ints->norb;
  const double *h1, *eri;
  ASCI_TRY(to_device(ints->h1, n * n, &h1, arena));
  ASCI_TRY(to_device(ints->eri, n * n * n * n, &eri, arena));
  unsigned *err;
  ASCI_TRY(arena.alloc(&err, 1));
  cudaStream_t s = arena.stream();
  ASCI_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  k_finite<<<blocks_for(n * n, 256), 256, 0, s>>>(h1, n * n, err);
  ASCI_CHECK_LAUNCH();
  k_finite<<<blocks_for(n * n * n * n, 256), 256, 0, s>>>(eri, n * n * n * n, err);
  ASCI_CHECK_LAUNCH();
  unsigned herr = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (herr || !std::isfinite(ints->ecore)) {
    record_error("non-finite integral", __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  return build_tables(h1, eri, (int)n, na, nb, ints->ecore, false, arena, I);
}

// H over key-ordered packed keys, allocated in the arena.
static int ham_build(const DevInts &I, const uint64_t *keys, size_t n, Arena &arena, Csr *H,
                     double **diag_out) {
  double *diag;
  int64_t *rp;
  ASCI_TRY(arena.alloc(&diag, n));
  ASCI_TRY(arena.alloc(&rp, n + 1));
  ASCI_TRY(diagonal_packed(I, keys, n, diag, arena));
  BetaGraph bg;
  ASCI_TRY(beta_graph(keys, (uint32_t)n, &bg, arena));
  size_t nnz = 0;
  ASCI_TRY(ham_count(I, keys, (uint32_t)n, diag, bg, rp, &nnz, arena));
  int32_t *col;
  double *val;
  ASCI_TRY(arena.alloc(&col, nnz));
  ASCI_TRY(arena.alloc(&val, nnz));
  ASCI_TRY(ham_fill(I, keys, (uint32_t)n, diag, bg, rp, col, val, arena));
  H->row_ptr = rp;
  H->col = col;
  H->val = val;
  H->n = n;
  *diag_out = diag;
  return ASCI_OK;
}

static size_t csr_nnz(const Csr &H, cudaStream_t s) {
  int64_t e = 0;
  if (cudaMemcpyAsync(&e, H.row_ptr + H.n, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 0;
  return (size_t)e;
}

// The ASCI loop (Algorithm 1); see asci_loop in the public header.
static int loop_impl(const asci_det *dets_in, const double *coeffs_in, size_t nd,
                     const asci_ints *ints, const asci_loop_opts &o, asci_det *out_dets,
                     double *out_coeffs, size_t *out_n, double *energy, asci_loop_stats *st,
                     cudaStream_t s) {
  Arena arena(s);
  const int norb = ints->norb;
  const asci_det *dets;
  const double *coeffs;
  ASCI_TRY(to_device(dets_in, nd, &dets, arena));
  ASCI_TRY(to_device(coeffs_in, nd, &coeffs, arena));
  uint64_t *keys, *keys_alt;
  double *c, *c_alt;
  int na = 0, nb = 0;
  ASCI_TRY(arena.alloc(&keys, nd));
  ASCI_TRY(arena.alloc(&keys_alt, nd));
  ASCI_TRY(det_keys(dets, nd, norb, keys, &na, &nb, arena));
  DevInts I;
  ASCI_TRY(stage_tables(ints, na, nb, arena, &I));
  const double *h1d, *erid;
  ASCI_TRY(to_device(ints->h1, (size_t)norb * norb, &h1d, arena));
  ASCI_TRY(to_device(ints->eri, (size_t)norb * norb * norb * norb, &erid, arena));
  asci_ints dints = *ints;
  dints.h1 = h1d;
  dints.eri = erid;
  // the start in key order
  ASCI_TRY(arena.alloc(&c, nd));
  ASCI_TRY(arena.alloc(&c_alt, nd));
  ASCI_TRY_CUDA(cudaMemcpyAsync(c, coeffs, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ASCI_TRY(radix_sort_u64_f64(&keys, &keys_alt, &c, &c_alt, nd, 0, 64, arena));
  double *sc;
  DotScratch part;
  ASCI_TRY(dot_scratch(&part, arena));
  ASCI_TRY(arena.alloc(&sc, 2));
  // E_0 = c.Hc / c.c on the start
  double E = 0.0;
  {
    Arena a2(s);
    Csr H;
    double *diag, *y;
    ASCI_TRY(ham_build(I, keys, nd, a2, &H, &diag));
    ASCI_TRY(a2.alloc(&y, nd));
    ASCI_TRY(spmv(H, c, y, s));
    ASCI_TRY(dots(c, nd, 1, y, nd, part, sc, 1, nullptr, 0, s));
    ASCI_TRY(dots(c, nd, 1, c, nd, part, sc + 1, 1, nullptr, 0, s));
    double hs[2];
    ASCI_TRY_CUDA(cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    if (!(hs[1] > 0.0)) {
      record_error("start coefficients are all zero", __FILE__, __LINE__);
      return ASCI_EINVAL;
    }
    E = hs[0] / hs[1];
  }
  if (st) st->start_energy = E;
  size_t m = nd;
  // per-step buffers live in their own arena; the current wavefunction is
  // carried between steps in buffers of the loop's arena
  uint64_t *cur_k = keys;
  double *cur_c = c;
  const size_t cap = std::max(nd, (size_t)o.ntdets);
  uint64_t *buf_k[2];
  double *buf_c[2];
  for (int b = 0; b < 2; ++b) {
    ASCI_TRY(arena.alloc(&buf_k[b], cap));
    ASCI_TRY(arena.alloc(&buf_c[b], cap));
  }
  int which = 0;
  for (int step = 0; step < o.max_steps; ++step) {
    Arena sa(s);
    StageTimer tm(s);
    double t_search = 0.0, t_build = 0.0, t_dav = 0.0;
    // 1. search from (psi_k, c_k, E_k)
    tm.start();
    asci_det *pd, *cand;
    double *cs;
    ASCI_TRY(sa.alloc(&pd, m));
    ASCI_TRY(sa.alloc(&cand, o.ntdets));
    ASCI_TRY(sa.alloc(&cs, o.ntdets));
    k_keys_to_dets<<<blocks_for(m, 256), 256, 0, s>>>(cur_k, m, pd);
    ASCI_CHECK_LAUNCH();
    size_t U = 0;
    asci_opts so = o.search;
    ASCI_TRY(asci_search(pd, cur_c, m, E, &dints, std::min<size_t>(o.ncdets, m), o.ntdets, &so,
                         cand, cs, &U, nullptr, s));
    if (U) {  // E_k equal to a candidate's H_ii leaves its score undefined
      unsigned *ferr;
      ASCI_TRY(sa.alloc(&ferr, 1));
      ASCI_TRY_CUDA(cudaMemsetAsync(ferr, 0, sizeof(unsigned), s));
      k_finite<<<blocks_for(U, 256), 256, 0, s>>>(cs, U, ferr);
      ASCI_CHECK_LAUNCH();
      unsigned hf = 0;
      ASCI_TRY_CUDA(cudaMemcpyAsync(&hf, ferr, sizeof(hf), cudaMemcpyDeviceToHost, s));
      ASCI_TRY_CUDA(cudaStreamSynchronize(s));
      if (hf) {
        record_error("a candidate's score is not finite (E equals its H_ii)", __FILE__, __LINE__);
        return ASCI_EINVAL;
      }
    }
    // 2. merge: psi_k valued by c, candidates by S; top ntdets, key order
    const size_t tot = m + U;
    uint64_t *uk, *sel_k, *sel_k_alt;
    double *uv, *sel_v, *sel_v_alt;
    ASCI_TRY(sa.alloc(&uk, tot));
    ASCI_TRY(sa.alloc(&uv, tot));
    ASCI_TRY_CUDA(cudaMemcpyAsync(uk, cur_k, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    ASCI_TRY_CUDA(cudaMemcpyAsync(uv, cur_c, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (U) {
      k_pack_dets<<<blocks_for(U, 256), 256, 0, s>>>(cand, U, uk + m);
      ASCI_CHECK_LAUNCH();
      ASCI_TRY_CUDA(cudaMemcpyAsync(uv + m, cs, U * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    const size_t keep = std::min<size_t>(tot, o.ntdets);
    ASCI_TRY(sa.alloc(&sel_k, keep));
    ASCI_TRY(sa.alloc(&sel_v, keep));
    ASCI_TRY(sa.alloc(&sel_k_alt, keep));
    ASCI_TRY(sa.alloc(&sel_v_alt, keep));
    size_t nsel = 0;
    ASCI_TRY(select_topn_packed(uk, uv, tot, o.ntdets, sel_k, sel_v, &nsel, sa));
    ASCI_TRY(radix_sort_u64_f64(&sel_k, &sel_k_alt, &sel_v, &sel_v_alt, nsel, 0, 64, sa));
    // determinants that entered (selected keys absent from psi_k)
    unsigned long long entered = 0;
    {
      unsigned long long *dc;
      ASCI_TRY(sa.alloc(&dc, 1));
      ASCI_TRY_CUDA(cudaMemsetAsync(dc, 0, sizeof(*dc), s));
      k_count_missing<<<blocks_for(nsel, 256), 256, 0, s>>>(sel_k, nsel, cur_k, m, dc);
      ASCI_CHECK_LAUNCH();
      ASCI_TRY_CUDA(cudaMemcpyAsync(&entered, dc, sizeof(entered), cudaMemcpyDeviceToHost, s));
      ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    }
    const bool changed = nsel != m || entered != 0;
    tm.stop(&t_search);
    // 3. H on the new space and its lowest eigenpair
    tm.start();
    Csr H;
    double *diag;
    ASCI_TRY(ham_build(I, sel_k, nsel, sa, &H, &diag));
    tm.stop(&t_build);
    tm.start();
    DavidsonResult dr;
    double *nc = buf_c[which];
    ASCI_TRY(davidson(H, diag, sel_v, o.davidson, nc, &dr, sa));
    tm.stop(&t_dav);
    if (!dr.converged) {
      record_error("Davidson did not converge within max_iter", __FILE__, __LINE__);
      return ASCI_ETIMEOUT;
    }
    ASCI_TRY_CUDA(cudaMemcpyAsync(buf_k[which], sel_k, nsel * sizeof(uint64_t),
                                  cudaMemcpyDeviceToDevice, s));
    if (st) {
      st->energy[step] = dr.energy;
      st->ndets[step] = nsel;
      st->nnz[step] = csr_nnz(H, s);
      st->davidson_iters[step] = dr.iterations;
      st->t_search[step] = t_search;
      st->t_hamiltonian[step] = t_build;
      st->t_davidson[step] = t_dav;
      st->new_dets[step] = entered;
      st->steps = step + 1;
    }
    const double Eold = E;
    E = dr.energy;
    cur_k = buf_k[which];
    cur_c = buf_c[which];
    m = nsel;
    which ^= 1;
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
    if (std::fabs(E - Eold) <= o.etol || !changed) break;
  }
  // outputs: the final space in key order and its vector
  asci_det *od;
  double *oc;
  ASCI_TRY(out_buffer(out_dets, m, &od, arena));
  ASCI_TRY(out_buffer(out_coeffs, m, &oc, arena));
  k_keys_to_dets<<<blocks_for(m, 256), 256, 0, s>>>(cur_k, m, od);
  ASCI_CHECK_LAUNCH();
  if (oc != cur_c)
    ASCI_TRY_CUDA(cudaMemcpyAsync(oc, cur_c, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ASCI_TRY(finish_out(out_dets, od, m, s));
  ASCI_TRY(finish_out(out_coeffs, oc, m, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = m;
  *energy = E;
  return ASCI_OK;
}

}  // namespace asci

using namespace asci;

extern "C" {

void asci_default_davidson_opts(asci_davidson_opts *o) {
  if (!o) return;
  o->max_subspace = 16;
  o->max_iter = 300;
  o->tol = 1e-8;
}

void asci_default_loop_opts(asci_loop_opts *o) {
  if (!o) return;
  o->ncdets = 10000;
  o->ntdets = 100000;
  o->max_steps = 8;
  o->etol = 1e-6;
  asci_default_opts(&o->search);
  asci_default_davidson_opts(&o->davidson);
}

int asci_hamiltonian(const asci_det *dets, size_t n, const asci_ints *ints, int64_t *row_ptr,
                     int32_t *col, double *val, size_t capacity, size_t *nnz,
                     void *cuda_stream) {
  if (nnz) *nnz = 0;
  if (!dets || !ints || !ints->h1 || !ints->eri || !row_ptr || !nnz) return ASCI_EINVAL;
  if (capacity && (!col || !val)) return ASCI_EINVAL;
  if (ints->norb < 1 || ints->norb > 32 || n == 0 || n >= (1ull << 31)) return ASCI_EINVAL;
  clear_last_error();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Arena arena(s);
  const asci_det *dd;
  ASCI_TRY(to_device(dets, n, &dd, arena));
  uint64_t *keys, *keys_alt;
  uint32_t *perm, *perm_alt;
  int na, nb;
  ASCI_TRY(arena.alloc(&keys, n));
  ASCI_TRY(arena.alloc(&keys_alt, n));
  ASCI_TRY(arena.alloc(&perm, n));
  ASCI_TRY(arena.alloc(&perm_alt, n));
  ASCI_TRY(det_keys(dd, n, ints->norb, keys, &na, &nb, arena));
  DevInts I;
  ASCI_TRY(stage_tables(ints, na, nb, arena, &I));
  // key order, and whether the caller's order already is key order
  k_iota<<<blocks_for(n, 256), 256, 0, s>>>(perm, (uint32_t)n);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY(radix_sort_u64_u32(&keys, &keys_alt, &perm, &perm_alt, n, 0, 64, arena));
  unsigned *flag, hflag = 0;
  ASCI_TRY(arena.alloc(&flag, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
  k_not_identity<<<blocks_for(n, 256), 256, 0, s>>>(perm, (uint32_t)n, flag);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  double *diag;
  ASCI_TRY(arena.alloc(&diag, n));
  ASCI_TRY(diagonal_packed(I, keys, n, diag, arena));
  BetaGraph bg;
  ASCI_TRY(beta_graph(keys, (uint32_t)n, &bg, arena));
  const bool same_order = hflag == 0;
  int64_t *rp, *urp;
  ASCI_TRY(out_buffer(row_ptr, n + 1, &urp, arena));
  if (same_order) rp = urp;
  else ASCI_TRY(arena.alloc(&rp, n + 1));
  size_t total = 0;
  ASCI_TRY(ham_count(I, keys, (uint32_t)n, diag, bg, rp, &total, arena));
  if (!same_order) {  // row pointers in the caller's order
    ASCI_TRY_CUDA(cudaMemsetAsync(urp + n, 0, sizeof(int64_t), s));
    k_user_counts<<<blocks_for(n, 256), 256, 0, s>>>(rp, perm, (uint32_t)n, urp);
    ASCI_CHECK_LAUNCH();
    ASCI_TRY(scan_exclusive_u64(reinterpret_cast<uint64_t *>(urp),
                                reinterpret_cast<uint64_t *>(urp), n + 1, arena));
  }
  if (total <= capacity) {
    int32_t *dc;
    double *dv;
    ASCI_TRY(out_buffer(col, total, &dc, arena));
    ASCI_TRY(out_buffer(val, total, &dv, arena));
    if (same_order) {
      ASCI_TRY(ham_fill(I, keys, (uint32_t)n, diag, bg, rp, dc, dv, arena));
    } else {
      // build in key order, then sort the entries on (caller row, caller column)
      if (total >= (1ull << 32)) {
        record_error("too many elements to reorder; pass the determinants in key order",
                     __FILE__, __LINE__);
        return ASCI_ENOMEM;
      }
      int32_t *kc;
      double *kv, *kv_alt;
      uint64_t *ek, *ek_alt;
      ASCI_TRY(arena.alloc(&kc, total));
      ASCI_TRY(arena.alloc(&kv, total));
      ASCI_TRY(arena.alloc(&kv_alt, total));
      ASCI_TRY(arena.alloc(&ek, total));
      ASCI_TRY(arena.alloc(&ek_alt, total));
      ASCI_TRY(ham_fill(I, keys, (uint32_t)n, diag, bg, rp, kc, kv, arena));
      k_user_entries<<<row_blocks((uint32_t)n), 256, 0, s>>>(rp, kc, perm, (uint32_t)n, ek);
      ASCI_CHECK_LAUNCH();
      ASCI_TRY(radix_sort_u64_f64(&ek, &ek_alt, &kv, &kv_alt, total, 0, 64, arena));
      k_low_cols<<<blocks_for(total, 256), 256, 0, s>>>(ek, total, dc);
      ASCI_CHECK_LAUNCH();
      ASCI_TRY_CUDA(cudaMemcpyAsync(dv, kv, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    ASCI_TRY(finish_out(col, dc, total, s));
    ASCI_TRY(finish_out(val, dv, total, s));
  }
  ASCI_TRY(finish_out(row_ptr, urp, n + 1, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *nnz = total;
  return ASCI_OK;
}

int asci_spmv(const int64_t *row_ptr, const int32_t *col, const double *val, size_t n,
              const double *x, double *y, void *cuda_stream) {
  if (!row_ptr || !col || !val || !x || !y || n >= (1ull << 31)) return ASCI_EINVAL;
  if (n == 0) return ASCI_OK;
  clear_last_error();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Arena arena(s);
  const int64_t *rp;
  ASCI_TRY(to_device(row_ptr, n + 1, &rp, arena));
  int64_t nnz = 0;  // needed only to stage host arrays
  if (!is_device_ptr(col) || !is_device_ptr(val)) {
    ASCI_TRY_CUDA(cudaMemcpyAsync(&nnz, rp + n, sizeof(nnz), cudaMemcpyDefault, s));
    ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  }
  const int32_t *dc;
  const double *dv, *dx;
  double *dy;
  ASCI_TRY(to_device(col, (size_t)nnz, &dc, arena));
  ASCI_TRY(to_device(val, (size_t)nnz, &dv, arena));
  ASCI_TRY(to_device(x, n, &dx, arena));
  ASCI_TRY(out_buffer(y, n, &dy, arena));
  Csr H = {rp, dc, dv, n};
  ASCI_TRY(spmv(H, dx, dy, s));
  ASCI_TRY(finish_out(y, dy, n, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  return ASCI_OK;
}

int asci_davidson(const int64_t *row_ptr, const int32_t *col, const double *val, size_t n,
                  const double *guess, const asci_davidson_opts *opts, double *energy,
                  double *vec, int32_t *iterations, double *residual, void *cuda_stream) {
  if (!row_ptr || !col || !val || !energy || !vec || n == 0 || n >= (1ull << 31))
    return ASCI_EINVAL;
  asci_davidson_opts o;
  asci_default_davidson_opts(&o);
  if (opts) o = *opts;
  ASCI_TRY(check_davidson_opts(o));
  clear_last_error();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Arena arena(s);
  const int64_t *rp;
  ASCI_TRY(to_device(row_ptr, n + 1, &rp, arena));
  int64_t nnz = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&nnz, rp + n, sizeof(nnz), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  const int32_t *dc;
  const double *dv, *dg = nullptr;
  ASCI_TRY(to_device(col, (size_t)nnz, &dc, arena));
  ASCI_TRY(to_device(val, (size_t)nnz, &dv, arena));
  if (guess) ASCI_TRY(to_device(guess, n, &dg, arena));
  Csr H = {rp, dc, dv, n};
  double *diag;
  ASCI_TRY(arena.alloc(&diag, n));
  k_csr_diag<<<blocks_for(n, 256), 256, 0, s>>>(rp, dc, dv, (uint32_t)n, diag);
  ASCI_CHECK_LAUNCH();
  DavidsonResult r;
  ASCI_TRY(davidson(H, diag, dg, o, vec, &r, arena));
  *energy = r.energy;
  if (iterations) *iterations = r.iterations;
  if (residual) *residual = r.residual;
  if (!r.converged) {
    record_error("Davidson did not converge within max_iter", __FILE__, __LINE__);
    return ASCI_ETIMEOUT;
  }
  return ASCI_OK;
}

int asci_loop(const asci_det *dets, const double *coeffs, size_t ndets, const asci_ints *ints,
              const asci_loop_opts *opts, asci_det *out_dets, double *out_coeffs,
              size_t capacity, size_t *out_n, double *energy, asci_loop_stats *stats,
              void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!dets || !coeffs || !ints || !ints->h1 || !ints->eri || !opts || !out_dets ||
      !out_coeffs || !out_n || !energy)
    return ASCI_EINVAL;
  const asci_loop_opts &o = *opts;
  if (ints->norb < 1 || ints->norb > 32 || ndets == 0 || ndets >= (1ull << 31) || o.ncdets == 0 ||
      o.ntdets == 0 || o.ntdets >= (1ull << 31) || capacity < o.ntdets || o.max_steps < 1 ||
      o.max_steps > ASCI_LOOP_MAX_STEPS || !(o.etol >= 0.0))
    return ASCI_EINVAL;
  ASCI_TRY(check_davidson_opts(o.davidson));
  clear_last_error();
  int r = loop_impl(dets, coeffs, ndets, ints, o, out_dets, out_coeffs, out_n, energy, stats,
                    (cudaStream_t)cuda_stream);
  if (r != ASCI_OK) *out_n = 0;
  return r;
}

}  // extern "C"
