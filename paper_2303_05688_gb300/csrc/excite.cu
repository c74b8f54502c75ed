// Excitation generation (Algorithm 2's inner loops) and the derived integral
// tables it reads.
//
// Every single and double excitation of a core determinant D_j is addressed by
// an index, decoded with popcount arithmetic (k-th set bit, colex pair
// unranking), and evaluated by the Slater-Condon rules with fermionic phases:
//   single i->a (spin s, other spin o):
//       sign * [h_ia + sum_{k in s} ((ia|kk) - (ik|ka)) + sum_{k in o} (ia|kk)]
//   same-spin double i<j -> a<b:  sign * [(ia|jb) - (ib|ja)], sign = i->a then j->b
//   opposite-spin double:         sign_alpha * sign_beta * (ia|jb)
// The partial quantity written per pair is v = H_ij * c_j (Alg. 2 with Eq. 1's
// numerator).
#include "asci_internal.cuh"

namespace asci {

ExcCounts exc_counts(int n, int na, int nb) {
  ExcCounts x;
  x.na = na;
  x.nb = nb;
  x.va = n - na;
  x.vb = n - nb;
  x.sa = x.na * x.va;
  x.sb = x.nb * x.vb;
  x.pa_h = x.na * (x.na - (x.na ? 1 : 0)) / 2;
  x.pa_p = x.va * (x.va - (x.va ? 1 : 0)) / 2;
  x.pb_h = x.nb * (x.nb - (x.nb ? 1 : 0)) / 2;
  x.pb_p = x.vb * (x.vb - (x.vb ? 1 : 0)) / 2;
  x.daa = (uint64_t)x.pa_h * x.pa_p;
  x.dbb = (uint64_t)x.pb_h * x.pb_p;
  x.dab = (uint64_t)x.sa * x.sb;
  x.total = (uint64_t)x.sa + x.sb + x.daa + x.dbb + x.dab;
  return x;
}

namespace {

// ------------------------------ tables -------------------------------------

__global__ void k_tables_n4(const double *eri, int n, double *asym, float *eri32, float *asym32,
                            double *asymT, float *asymT32) {
  size_t n4 = (size_t)n * n * n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4;
       t += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(t % n), j = (int)((t / n) % n), a = (int)((t / n / n) % n), i = (int)(t / n / n / n);
    double v = eri[t] - eri[(((size_t)i * n + b) * n + j) * n + a];
    const size_t tt = (((size_t)j * n + b) * n + i) * n + a;
    asym[t] = v;
    asymT[tt] = v;
    if (eri32) eri32[t] = (float)eri[t];
    if (asym32) {
      asym32[t] = (float)v;
      asymT32[tt] = (float)v;
    }
  }
}

__global__ void k_tables_n3(const double *eri, int n, double *s_same, double *s_opp) {
  size_t n3 = (size_t)n * n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3;
       t += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(t % n), a = (int)((t / n) % n), i = (int)(t / n / n);
    double iakk = eri[(((size_t)i * n + a) * n + k) * n + k];
    double ikka = eri[(((size_t)i * n + k) * n + k) * n + a];
    s_same[t] = iakk - ikka;
    s_opp[t] = iakk;
  }
}

__global__ void k_tables_n2(const double *eri, int n, double *jk, double *jj) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int p = t / n, q = t % n;
  double J = eri[(((size_t)p * n + p) * n + q) * n + q];
  double K = eri[(((size_t)p * n + q) * n + q) * n + p];
  jj[t] = J;
  jk[t] = J - K;
}

// ------------------------------ evaluation ---------------------------------

__device__ __forceinline__ void decode_single(uint32_t s, uint32_t virt, uint32_t idx, uint32_t nv,
                                              int *i, int *a) {
  *i = nth_set_bit(s, (int)(idx / nv));
  *a = nth_set_bit(virt, (int)(idx % nv));
}

__device__ __forceinline__ void decode_double(uint32_t s, uint32_t virt, uint32_t idx,
                                              uint32_t npp, int *i, int *j, int *a, int *b) {
  int h1, h2, p1, p2;
  unrank_pair(idx / npp, &h1, &h2);
  unrank_pair(idx % npp, &p1, &p2);
  *i = nth_set_bit(s, h1);
  *j = nth_set_bit(s, h2);
  *a = nth_set_bit(virt, p1);
  *b = nth_set_bit(virt, p2);
}

// Excitation e (fixed order) of determinant (A, B): target and H_ij.
__device__ void fixed_order_pair(const DevInts &I, const ExcCounts &X, uint32_t A, uint32_t B,
                                 uint64_t e, uint32_t *ta, uint32_t *tb, double *h) {
  const uint32_t full = full_mask(I.n);
  const uint32_t va = ~A & full, vb = ~B & full;
  int i, j, a, b;
  if (e < X.sa) {
    decode_single(A, va, (uint32_t)e, X.va, &i, &a);
    *ta = A ^ (1u << i) ^ (1u << a);
    *tb = B;
    double v = single_value(I, A, B, i, a);
    *h = single_parity(A, i, a) ? -v : v;
    return;
  }
  e -= X.sa;
  if (e < X.sb) {
    decode_single(B, vb, (uint32_t)e, X.vb, &i, &a);
    *ta = A;
    *tb = B ^ (1u << i) ^ (1u << a);
    double v = single_value(I, B, A, i, a);
    *h = single_parity(B, i, a) ? -v : v;
    return;
  }
  e -= X.sb;
  if (e < X.daa) {
    decode_double(A, va, (uint32_t)e, X.pa_p, &i, &j, &a, &b);
    *ta = A ^ (1u << i) ^ (1u << j) ^ (1u << a) ^ (1u << b);
    *tb = B;
    double v = eri4(I.asym, I.n, i, a, j, b);
    *h = double_parity(A, i, j, a, b) ? -v : v;
    return;
  }
  e -= X.daa;
  if (e < X.dbb) {
    decode_double(B, vb, (uint32_t)e, X.pb_p, &i, &j, &a, &b);
    *ta = A;
    *tb = B ^ (1u << i) ^ (1u << j) ^ (1u << a) ^ (1u << b);
    double v = eri4(I.asym, I.n, i, a, j, b);
    *h = double_parity(B, i, j, a, b) ? -v : v;
    return;
  }
  e -= X.dbb;
  {
    decode_single(A, va, (uint32_t)(e / X.sb), X.va, &i, &a);
    decode_single(B, vb, (uint32_t)(e % X.sb), X.vb, &j, &b);
    *ta = A ^ (1u << i) ^ (1u << a);
    *tb = B ^ (1u << j) ^ (1u << b);
    double v = eri4(I.eri, I.n, i, a, j, b);
    *h = (single_parity(A, i, a) ^ single_parity(B, j, b)) ? -v : v;
  }
}

__global__ void k_emit_fixed(DevInts I, ExcCounts X, const uint64_t *core_keys,
                             const double *core_c, size_t ncore, uint64_t *out_keys,
                             double *out_vals) {
  const uint64_t total = (uint64_t)ncore * X.total;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t m = p / X.total, e = p - m * X.total;
    uint64_t k = core_keys[m];
    uint32_t ta, tb;
    double h;
    fixed_order_pair(I, X, key_alpha(k), key_beta(k), e, &ta, &tb, &h);
    out_keys[p] = pack_key(ta, tb);
    out_vals[p] = h * core_c[m];
  }
}

}  // namespace

int build_tables(const double *h1_dev, const double *eri_dev, int n, int na, int nb, double ecore,
                 bool want_fp32, Arena &arena, DevInts *out) {
  DevInts I;
  I.n = n;
  I.na = na;
  I.nb = nb;
  I.ecore = ecore;
  I.h1 = h1_dev;
  I.eri = eri_dev;
  size_t n2 = (size_t)n * n, n3 = n2 * n, n4 = n3 * n;
  double *asym, *asymT, *s_same, *s_opp, *jk, *jj;
  float *eri32 = nullptr, *asym32 = nullptr, *asymT32 = nullptr;
  ASCI_TRY(arena.alloc(&asym, n4));
  ASCI_TRY(arena.alloc(&asymT, n4));
  ASCI_TRY(arena.alloc(&s_same, n3));
  ASCI_TRY(arena.alloc(&s_opp, n3));
  ASCI_TRY(arena.alloc(&jk, n2));
  ASCI_TRY(arena.alloc(&jj, n2));
  if (want_fp32) {
    ASCI_TRY(arena.alloc(&eri32, n4));
    ASCI_TRY(arena.alloc(&asym32, n4));
    ASCI_TRY(arena.alloc(&asymT32, n4));
  }
  cudaStream_t s = arena.stream();
  k_tables_n4<<<(unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096), 256, 0, s>>>(
      eri_dev, n, asym, eri32, asym32, asymT, asymT32);
  ASCI_CHECK_LAUNCH();
  k_tables_n3<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(eri_dev, n, s_same, s_opp);
  ASCI_CHECK_LAUNCH();
  k_tables_n2<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(eri_dev, n, jk, jj);
  ASCI_CHECK_LAUNCH();
  I.asym = asym;
  I.s_same = s_same;
  I.s_opp = s_opp;
  I.jk = jk;
  I.jj = jj;
  I.eri32 = eri32;
  I.asym32 = asym32;
  I.asymT = asymT;
  I.asymT32 = asymT32;
  *out = I;
  return ASCI_OK;
}

int emit_fixed_order(const DevInts &I, const uint64_t *core_keys, const double *core_c,
                     size_t ncore, uint64_t *out_keys, double *out_vals, Arena &arena) {
  ExcCounts X = exc_counts(I.n, I.na, I.nb);
  uint64_t total = (uint64_t)ncore * X.total;
  if (total == 0) return ASCI_OK;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_emit_fixed<<<(unsigned)blocks, 256, 0, arena.stream()>>>(I, X, core_keys, core_c, ncore,
                                                             out_keys, out_vals);
  ASCI_CHECK_LAUNCH();
  return ASCI_OK;
}

// ---------------------------------------------------------------------------
// constraint-batched generation
// ---------------------------------------------------------------------------
//
// The core determinants are grouped by alpha string (group k holds the core
// dets with alpha string A_k).  An "item" is (group k, alpha operation o): no
// alpha change (o = 0), an alpha single (1 <= o <= sa) or an alpha-alpha double.
// It fixes the target's alpha string A' and therefore its constraint class:
// the class of a determinant at level L is the set of its L highest occupied
// alpha orbitals (Sec. 2.2, triplet constraints and their refinements), and
// classes are contiguous ranges once items are sorted by A'.  Each item emits
// its pairs for every core det of its group:
//   o = 0:      beta singles and beta-beta doubles      (sb + dbb per det)
//   single:     the alpha single itself and the alpha-beta doubles (1 + sb)
//   double:     the alpha-alpha double                  (1)

namespace {

// One CTA per group (persistent over groups): the group's occupied and
// virtual orbitals and the unranked orbital-index pairs sit in shared memory,
// so an operation's target costs two table reads per orbital pair and the
// items of a group are written contiguously.  The operation numbering is the
// one of decode_single / decode_double.
__global__ void __launch_bounds__(256)
    k_make_items(ExcCounts X, int n, const uint32_t *grp_alpha, uint32_t ngroups,
                 uint32_t o_begin, uint32_t nops, int opbits, FastDiv by_nv, FastDiv by_npp,
                 uint64_t *items, unsigned *t_or, unsigned *t_and) {
  __shared__ uint8_t occ[32], vir[32];
  __shared__ uint8_t pr_x[496], pr_y[496];  // pair r -> (x, y), x < y < 32
  const uint32_t per = nops - o_begin;
  const uint32_t full = full_mask(n);
  uint32_t any_or = 0u, all_and = 0xffffffffu;
  for (int r = threadIdx.x; r < 496; r += blockDim.x) {
    int x, y;
    unrank_pair((uint32_t)r, &x, &y);
    pr_x[r] = (uint8_t)x;
    pr_y[r] = (uint8_t)y;
  }
  for (uint32_t k = blockIdx.x; k < ngroups; k += gridDim.x) {
    const uint32_t A = grp_alpha[k], va = ~A & full;
    __syncthreads();  // previous group's lists no longer read
    if (threadIdx.x < 32) {
      const uint32_t bit = 1u << threadIdx.x;
      if (A & bit) occ[__popc(A & (bit - 1u))] = (uint8_t)threadIdx.x;
      if (va & bit) vir[__popc(va & (bit - 1u))] = (uint8_t)threadIdx.x;
    }
    __syncthreads();
    uint64_t *out = items + (uint64_t)k * per;
    const uint64_t lo_k = (uint64_t)k << opbits;
    for (uint32_t t = threadIdx.x; t < per; t += blockDim.x) {
      const uint32_t o = o_begin + t;
      uint32_t At = A;
      if (o != 0 && o <= X.sa) {
        const uint32_t idx = o - 1, h = by_nv.div(idx);
        At ^= (1u << occ[h]) ^ (1u << vir[idx - h * X.va]);
      } else if (o != 0) {
        const uint32_t idx = o - 1 - X.sa, hp = by_npp.div(idx), pp = idx - hp * X.pa_p;
        At ^= (1u << occ[pr_x[hp]]) ^ (1u << occ[pr_y[hp]]) ^ (1u << vir[pr_x[pp]]) ^
              (1u << vir[pr_y[pp]]);
      }
      out[t] = ((uint64_t)At << 32) | lo_k | o;
      any_or |= At;
      all_and &= At;
    }
  }
  // the bits in which the target strings differ (for the sort), one atomic
  // pair per warp
  any_or = __reduce_or_sync(0xffffffffu, any_or);
  all_and = __reduce_and_sync(0xffffffffu, all_and);
  if ((threadIdx.x & 31u) == 0) {
    atomicOr(t_or, any_or);
    atomicAnd(t_and, all_and);
  }
}

}  // namespace

int make_items(const ExcCounts &X, int n, const uint32_t *grp_alpha, uint32_t ngroups,
               uint32_t o_begin, uint32_t nops, int opbits, uint64_t *items,
               uint64_t *varying, Arena &arena) {
  *varying = 0;
  uint64_t total = (uint64_t)ngroups * (nops - o_begin);
  if (!total) return ASCI_OK;
  cudaStream_t s = arena.stream();
  unsigned *bits;
  ASCI_TRY(arena.alloc(&bits, 2));
  const unsigned init[2] = {0u, 0xffffffffu};
  ASCI_TRY_CUDA(cudaMemcpyAsync(bits, init, sizeof(init), cudaMemcpyHostToDevice, s));
  const unsigned blocks = (unsigned)std::min<uint64_t>(ngroups, 152 * 8);
  k_make_items<<<blocks, 256, 0, s>>>(X, n, grp_alpha, ngroups, o_begin, nops, opbits,
                                      FastDiv(X.va ? X.va : 1), FastDiv(X.pa_p ? X.pa_p : 1),
                                      items, bits, bits + 1);
  ASCI_CHECK_LAUNCH();
  unsigned h[2] = {0u, 0u};
  ASCI_TRY_CUDA(cudaMemcpyAsync(h, bits, sizeof(h), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *varying = (uint64_t)(h[0] ^ h[1]) << 32;
  return ASCI_OK;
}

}  // namespace asci
