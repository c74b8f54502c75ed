// Shared declarations of the constraint-tile search (fused.cu) and its host
// orchestration (search.cu).
#pragma once

#include "asci_internal.cuh"

namespace asci {

// Integral terms of the diagonal in 64-bit fixed point (multiples of 2^-s).
struct FxInts {
  int n;
  int s;              // values are multiples of 2^-s
  int64_t ecore_x;
  const int64_t *hh;  // n      h_pp
  const int64_t *jk;  // n*n    (pp|qq) - (pq|qp), zero diagonal
  const int64_t *jj;  // n*n    (pp|qq)
  // single excitations i -> a in fixed point, multiples of 2^-s1:
  // h1x = h_ia, ssx[(i*n+a)*n+k] = (ia|kk) - (ik|ka), sox[(i*n+a)*n+k] = (ia|kk)
  int s1;
  const int64_t *h1x, *ssx, *sox;
};

// One staged pair (16 bytes, written with one vector store): the value
// H_ij c_j, the target's beta string and the denominator E0 - H_ii as a float,
// which serves the threshold screen only; the exact diagonal is recomputed for
// targets that pass it.
struct __align__(16) StageRec {
  double v;
  uint32_t beta;
  float den;
};
static_assert(sizeof(StageRec) == 16, "staged pair layout");

// The staging buffer of a batch: records, and the target alpha string of the
// records of classes packed several to a tile (other tiles know theirs).
struct Stage {
  StageRec *rec;
  uint32_t *alpha;
  uint64_t cap;  // records the buffer holds
};

// Records that found their hash-bucket cell full (kCap records), and their
// order by tile: keys[j] = tile << 32 | index into rec.
struct Spill {
  const StageRec *rec;
  const uint64_t *keys;
  uint32_t n;
};

// Everything the batch kernels read that stays fixed during one search.
struct FusedCore {
  DevInts I;
  FxInts X;
  ExcCounts E;
  const uint64_t *items, *Wexcl;
  const uint32_t *item_group;
  int opbits;
  const uint32_t *grp_alpha, *grp_start, *grp_count, *core_beta;
  const double *core_c;
  const int64_t *Dx, *Fa, *Fb;
  const uint32_t *g_alpha;
  const uint64_t *g_P0;
  int64_t E0_x;
  const uint64_t *psi_ht;
  uint64_t psi_mask;
  const uint64_t *psi_keys;  // psi keys, sorted
  size_t npsi;
  uint32_t ncore;
  int prec;  // pair-value precision: 0 FP64, 1 FP32 integrals, 2 FP32 integrals and product
  int screened;  // Alg. 2's eps screen is on: staged records may be marked dropped
  int ctas_per_sm;  // cap on the persistent kernels' CTAs per SM (0: as many as fit)
};

}  // namespace asci
