/*
 * Plain FP64 CPU oracle for the ASCI determinant search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the GPU path.  It is deliberately slow and direct: nested loops,
 * a general Slater-Condon evaluator called per pair, qsort, and compensated sums.
 *
 * What it computes (arXiv:2303.05688):
 *  - Eq. 1, the ASCI score of a determinant D_i outside psi:
 *        S_i = sum_j H_ij C_j / (H_ii - E_k).
 *    Following the search definition the numerator sum runs over the core
 *    determinants, and the returned score uses the sign num / (E0 - H_ii);
 *    ranking is by |S|, which is the same under either sign.
 *  - Algorithm 2, the ASCI search: take the N_cdets core determinants of
 *    largest |C_j|; enumerate every single and double excitation of each;
 *    form the partial quantity per (target, core) pair; screen by
 *    |S_i^(j)| > eps; sort the pairs on the target; accumulate per unique
 *    target; score; keep the top N_tdets (Sec. 2.2, "sort-and-accumulate").
 *  - The selection follows the duplicate-aware definition of Sec. 2.2 (the
 *    k-th largest element a_k with |{a > a_k}| < k <= |{a >= a_k}|); among
 *    equal |S| the oracle breaks ties by the 128-bit key ascending (beta word
 *    high, alpha word low) so that its answer is a single set.
 *
 * Readings where the paper is silent (each is pinned by tests/ against a
 * brute-force second-quantised Hamiltonian, not by the paper):
 *  - H = ecore + sum_{pq,s} h_pq a+_ps a_qs
 *          + 1/2 sum_{pqrs,st} (pq|rs) a+_ps a+_rt a_st a_qs,
 *    real integrals with 8-fold symmetry, chemists' layout
 *    eri[((p*n+q)*n+r)*n+s] = (pq|rs).
 *  - |D> = prod_{p in alpha, ascending} a+_{p,alpha}
 *          prod_{q in beta, ascending} a+_{q,beta} |0>.
 *  - A single p -> q on one spin carries (-1)^(number of occupied orbitals of
 *    that spin strictly between p and q).  A same-spin double i<j -> a<b is the
 *    single i -> a followed by the single j -> b on the updated string.
 *    An opposite-spin double is the product of its two singles.
 *  - eps == 0 keeps every generated pair (even H_ij == 0), so that the set of
 *    candidate keys is purely structural.
 *
 * Every function below states the passage it follows.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* integrals                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;
  double ecore;
  const double *h1;  /* n*n */
  const double *eri; /* n^4 */
} oints;

static double H1(const oints *I, int p, int q) { return I->h1[(size_t)p * I->n + q]; }

static double ERI(const oints *I, int p, int q, int r, int s) {
  size_t n = (size_t)I->n;
  return I->eri[((p * n + q) * n + r) * n + s];
}

static int occupied(uint64_t s, int p) { return (int)((s >> p) & 1u); }

static int count_bits(uint64_t s) {
  int c = 0;
  while (s) {
    c += (int)(s & 1u);
    s >>= 1;
  }
  return c;
}

/* Neumaier-compensated running sum. */
typedef struct {
  double s, c;
} nsum;

static void nsum_add(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* (-1)^(number of occupied orbitals of string s strictly between p and q). */
static int single_sign(uint64_t s, int p, int q) {
  int lo = p < q ? p : q, hi = p < q ? q : p, k, cnt = 0;
  for (k = lo + 1; k < hi; k++) cnt += occupied(s, k);
  return (cnt & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------------ */
/* Slater-Condon rules (textbook; reading of the Hamiltonian above)          */
/* ------------------------------------------------------------------------ */

/* One term of the diagonal sum: added to the value and, by magnitude, to the
 * sum of |terms| that bounds the rounding error of any evaluation order. */
static void diag_term(nsum *acc, nsum *mag, double t) {
  nsum_add(acc, t);
  nsum_add(mag, fabs(t));
}

/* Diagonal element <D|H|D>; *abs_out (nullable) receives the sum of the
 * magnitudes of its terms. */
static double diag_with_abs(const oints *I, uint64_t a, uint64_t b, double *abs_out) {
  int n = I->n, p, q;
  nsum acc = {0.0, 0.0}, mag = {0.0, 0.0};
  diag_term(&acc, &mag, I->ecore);
  for (p = 0; p < n; p++) {
    if (occupied(a, p)) diag_term(&acc, &mag, H1(I, p, p));
    if (occupied(b, p)) diag_term(&acc, &mag, H1(I, p, p));
  }
  for (p = 0; p < n; p++)
    for (q = 0; q < n; q++) {
      /* same-spin pairs, 1/2 sum over ordered pairs */
      if (occupied(a, p) && occupied(a, q))
        diag_term(&acc, &mag, 0.5 * (ERI(I, p, p, q, q) - ERI(I, p, q, q, p)));
      if (occupied(b, p) && occupied(b, q))
        diag_term(&acc, &mag, 0.5 * (ERI(I, p, p, q, q) - ERI(I, p, q, q, p)));
      /* opposite-spin Coulomb */
      if (occupied(a, p) && occupied(b, q)) diag_term(&acc, &mag, ERI(I, p, p, q, q));
    }
  if (abs_out) *abs_out = nsum_get(&mag);
  return nsum_get(&acc);
}

double oracle_diag_impl(const oints *I, uint64_t a, uint64_t b) {
  return diag_with_abs(I, a, b, NULL);
}

/* Single excitation i -> a on spin string s (the other spin string is o),
 * evaluated on the ket's occupations; returns the value without the sign. */
static double single_value(const oints *I, uint64_t s, uint64_t o, int i, int a) {
  int n = I->n, k;
  nsum acc = {0.0, 0.0};
  nsum_add(&acc, H1(I, i, a));
  for (k = 0; k < n; k++) {
    if (occupied(s, k)) nsum_add(&acc, ERI(I, i, a, k, k) - ERI(I, i, k, k, a));
    if (occupied(o, k)) nsum_add(&acc, ERI(I, i, a, k, k));
  }
  return nsum_get(&acc);
}

/* Orbitals set in x, lowest first; returns how many were written (<= 2 used). */
static int list_bits(uint64_t x, int n, int *out, int cap) {
  int p, c = 0;
  for (p = 0; p < n; p++)
    if (occupied(x, p)) {
      if (c < cap) out[c] = p;
      c++;
    }
  return c;
}

/* <bra|H|ket> for two determinants of the same electron counts. */
double oracle_hij_impl(const oints *I, uint64_t bra_a, uint64_t bra_b, uint64_t ket_a,
                       uint64_t ket_b) {
  int n = I->n;
  uint64_t xa = bra_a ^ ket_a, xb = bra_b ^ ket_b;
  int ea = count_bits(xa) / 2, eb = count_bits(xb) / 2;
  int ha[2], pa[2], hb[2], pb[2];
  if (ea + eb == 0) return oracle_diag_impl(I, ket_a, ket_b);
  if (ea + eb > 2) return 0.0;
  /* holes: occupied in ket only; particles: occupied in bra only */
  list_bits(xa & ket_a, n, ha, 2);
  list_bits(xa & bra_a, n, pa, 2);
  list_bits(xb & ket_b, n, hb, 2);
  list_bits(xb & bra_b, n, pb, 2);
  if (ea == 1 && eb == 0)
    return single_sign(ket_a, ha[0], pa[0]) * single_value(I, ket_a, ket_b, ha[0], pa[0]);
  if (ea == 0 && eb == 1)
    return single_sign(ket_b, hb[0], pb[0]) * single_value(I, ket_b, ket_a, hb[0], pb[0]);
  if (ea == 1 && eb == 1) {
    int s = single_sign(ket_a, ha[0], pa[0]) * single_sign(ket_b, hb[0], pb[0]);
    return s * ERI(I, ha[0], pa[0], hb[0], pb[0]);
  }
  {
    /* same-spin double: holes i<j, particles a<b; i -> a then j -> b */
    uint64_t s0 = (ea == 2) ? ket_a : ket_b;
    int *h = (ea == 2) ? ha : hb, *p = (ea == 2) ? pa : pb;
    int i = h[0], j = h[1], a = p[0], b = p[1];
    uint64_t s1 = s0 ^ (1ull << i) ^ (1ull << a);
    int sg = single_sign(s0, i, a) * single_sign(s1, j, b);
    return sg * (ERI(I, i, a, j, b) - ERI(I, i, b, j, a));
  }
}

/* ------------------------------------------------------------------------ */
/* the search (Algorithm 2)                                                 */
/* ------------------------------------------------------------------------ */

/* 128-bit key order: beta word high, alpha word low. */
static int key_cmp(uint64_t a1, uint64_t b1, uint64_t a2, uint64_t b2) {
  if (b1 != b2) return b1 < b2 ? -1 : 1;
  if (a1 != a2) return a1 < a2 ? -1 : 1;
  return 0;
}

/* splitmix64 finaliser; used only to split the target space into buckets. */
static uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

uint64_t oracle_bucket_of(uint64_t a, uint64_t b, uint64_t nbuckets) {
  return mix64(a ^ mix64(b)) % nbuckets;
}

typedef struct {
  uint64_t a, b;
  double v;
  size_t order; /* generation order: makes the sort deterministic */
} opair;

static int opair_cmp(const void *x, const void *y) {
  const opair *p = (const opair *)x, *q = (const opair *)y;
  int c = key_cmp(p->a, p->b, q->a, q->b);
  if (c) return c;
  return (p->order > q->order) - (p->order < q->order);
}

/* core selection order: |c| descending, then key ascending (Alg. 2, first step) */
typedef struct {
  uint64_t a, b;
  double absc;
  size_t idx;
} ocore;

static int ocore_cmp(const void *x, const void *y) {
  const ocore *p = (const ocore *)x, *q = (const ocore *)y;
  if (p->absc != q->absc) return p->absc > q->absc ? -1 : 1;
  return key_cmp(p->a, p->b, q->a, q->b);
}

typedef struct {
  uint64_t a, b;
} okey;

static int okey_cmp(const void *x, const void *y) {
  const okey *p = (const okey *)x, *q = (const okey *)y;
  return key_cmp(p->a, p->b, q->a, q->b);
}

typedef struct {
  size_t n, cap;
  opair *v;
  size_t order;
} opairs;

static int opairs_push(opairs *P, uint64_t a, uint64_t b, double v) {
  if (P->n == P->cap) {
    size_t nc = P->cap ? 2 * P->cap : 1024;
    opair *nv = (opair *)realloc(P->v, nc * sizeof(opair));
    if (!nv) return -1;
    P->v = nv;
    P->cap = nc;
  }
  P->v[P->n].a = a;
  P->v[P->n].b = b;
  P->v[P->n].v = v;
  P->v[P->n].order = P->order++;
  P->n++;
  return 0;
}

typedef struct {
  const oints *I;
  double E0, eps;
  uint64_t nbuckets, bucket;
  size_t generated, surviving;
  opairs P;
  int err;
} ogen;

/* One (target, core) pair: Alg. 2 inner body (partial score, screen, append). */
static void visit(ogen *g, uint64_t ta, uint64_t tb, uint64_t ka, uint64_t kb, double cj) {
  double hij, v;
  g->generated++;
  if (g->nbuckets > 1 && oracle_bucket_of(ta, tb, g->nbuckets) != g->bucket) return;
  hij = oracle_hij_impl(g->I, ta, tb, ka, kb);
  v = hij * cj;
  if (g->eps > 0.0) {
    double hii = oracle_diag_impl(g->I, ta, tb);
    if (!(fabs(v / (g->E0 - hii)) > g->eps)) return;
  }
  g->surviving++;
  if (opairs_push(&g->P, ta, tb, v)) g->err = 1;
}

/* Every single and double excitation of (ka, kb), by nested loops in a fixed
 * order: alpha singles, beta singles, alpha-alpha doubles, beta-beta doubles,
 * alpha-beta doubles (the set {D_j^sd} of Alg. 2; Sec. 2.1 explains why only
 * singles and doubles connect through a two-body H). */
static void enumerate(ogen *g, int n, uint64_t ka, uint64_t kb, double cj) {
  int i, j, a, b;
  for (i = 0; i < n; i++)
    for (a = 0; a < n; a++)
      if (occupied(ka, i) && !occupied(ka, a))
        visit(g, ka ^ (1ull << i) ^ (1ull << a), kb, ka, kb, cj);
  for (i = 0; i < n; i++)
    for (a = 0; a < n; a++)
      if (occupied(kb, i) && !occupied(kb, a))
        visit(g, ka, kb ^ (1ull << i) ^ (1ull << a), ka, kb, cj);
  for (i = 0; i < n; i++)
    for (j = i + 1; j < n; j++)
      for (a = 0; a < n; a++)
        for (b = a + 1; b < n; b++)
          if (occupied(ka, i) && occupied(ka, j) && !occupied(ka, a) && !occupied(ka, b))
            visit(g, ka ^ (1ull << i) ^ (1ull << j) ^ (1ull << a) ^ (1ull << b), kb, ka, kb, cj);
  for (i = 0; i < n; i++)
    for (j = i + 1; j < n; j++)
      for (a = 0; a < n; a++)
        for (b = a + 1; b < n; b++)
          if (occupied(kb, i) && occupied(kb, j) && !occupied(kb, a) && !occupied(kb, b))
            visit(g, ka, kb ^ (1ull << i) ^ (1ull << j) ^ (1ull << a) ^ (1ull << b), ka, kb, cj);
  for (i = 0; i < n; i++)
    for (a = 0; a < n; a++)
      if (occupied(ka, i) && !occupied(ka, a))
        for (j = 0; j < n; j++)
          for (b = 0; b < n; b++)
            if (occupied(kb, j) && !occupied(kb, b))
              visit(g, ka ^ (1ull << i) ^ (1ull << a), kb ^ (1ull << j) ^ (1ull << b), ka, kb, cj);
}

typedef struct {
  size_t ncand;
  uint64_t *a, *b;
  double *num, *abssum, *haa, *haa_abs, *score;
  size_t generated, surviving, unique, excluded, ncore;
} oresult;

void oracle_free(oresult *r) {
  if (!r) return;
  free(r->a);
  free(r->b);
  free(r->num);
  free(r->abssum);
  free(r->haa);
  free(r->haa_abs);
  free(r->score);
  free(r);
}

/* Core selection (Alg. 2, first step): indices of the C determinants with the
 * largest |c|, ties by key ascending, written in that order.  Returns count. */
size_t oracle_core_select(const uint64_t *da, const uint64_t *db, const double *c, size_t nd,
                          size_t C, size_t *out_idx) {
  size_t i, m = C < nd ? C : nd;
  ocore *v = (ocore *)malloc((nd ? nd : 1) * sizeof(ocore));
  if (!v) return 0;
  for (i = 0; i < nd; i++) {
    v[i].a = da[i];
    v[i].b = db[i];
    v[i].absc = fabs(c[i]);
    v[i].idx = i;
  }
  qsort(v, nd, sizeof(ocore), ocore_cmp);
  for (i = 0; i < m; i++) out_idx[i] = v[i].idx;
  free(v);
  return m;
}

/*
 * Algorithm 2 with Eq. 1 (unbatched).  When nbuckets > 1 only targets whose
 * bucket_of() equals `bucket` are kept: the candidate space is split into
 * disjoint hash classes so that large cases run in bounded memory, pass by pass.
 * Returns every unique candidate outside psi with its numerator, the sum of
 * |H_ij c_j| over its contributions, H_ii and the signed score.
 */
oresult *oracle_search(int n, const double *h1, const double *eri, double ecore,
                       const uint64_t *da, const uint64_t *db, const double *c, size_t nd,
                       double E0, size_t C, double eps, uint64_t nbuckets, uint64_t bucket) {
  oints I = {n, ecore, h1, eri};
  ogen g;
  size_t i, m, u, k;
  size_t *core;
  okey *psi;
  oresult *r = (oresult *)calloc(1, sizeof(oresult));
  if (!r) return NULL;
  memset(&g, 0, sizeof(g));
  g.I = &I;
  g.E0 = E0;
  g.eps = eps;
  g.nbuckets = nbuckets ? nbuckets : 1;
  g.bucket = bucket;

  core = (size_t *)malloc((nd ? nd : 1) * sizeof(size_t));
  m = oracle_core_select(da, db, c, nd, C, core);
  r->ncore = m;
  for (i = 0; i < m; i++) enumerate(&g, n, da[core[i]], db[core[i]], c[core[i]]);
  free(core);
  r->generated = g.generated;
  r->surviving = g.surviving;
  if (g.err) {
    free(g.P.v);
    oracle_free(r);
    return NULL;
  }

  /* sort-and-accumulate (Sec. 2.2) */
  qsort(g.P.v, g.P.n, sizeof(opair), opair_cmp);
  psi = (okey *)malloc((nd ? nd : 1) * sizeof(okey));
  for (i = 0; i < nd; i++) {
    psi[i].a = da[i];
    psi[i].b = db[i];
  }
  qsort(psi, nd, sizeof(okey), okey_cmp);

  u = 0;
  for (i = 0; i < g.P.n; i++)
    if (i == 0 || key_cmp(g.P.v[i].a, g.P.v[i].b, g.P.v[i - 1].a, g.P.v[i - 1].b)) u++;
  r->unique = u;
  r->a = (uint64_t *)malloc((u ? u : 1) * sizeof(uint64_t));
  r->b = (uint64_t *)malloc((u ? u : 1) * sizeof(uint64_t));
  r->num = (double *)malloc((u ? u : 1) * sizeof(double));
  r->abssum = (double *)malloc((u ? u : 1) * sizeof(double));
  r->haa = (double *)malloc((u ? u : 1) * sizeof(double));
  r->haa_abs = (double *)malloc((u ? u : 1) * sizeof(double));
  r->score = (double *)malloc((u ? u : 1) * sizeof(double));
  k = 0;
  for (i = 0; i < g.P.n;) {
    size_t j = i;
    nsum num = {0.0, 0.0}, abssum = {0.0, 0.0};
    okey key;
    while (j < g.P.n && !key_cmp(g.P.v[j].a, g.P.v[j].b, g.P.v[i].a, g.P.v[i].b)) {
      nsum_add(&num, g.P.v[j].v);
      nsum_add(&abssum, fabs(g.P.v[j].v));
      j++;
    }
    key.a = g.P.v[i].a;
    key.b = g.P.v[i].b;
    /* Eq. 1's free index runs over determinants outside psi */
    if (nd && bsearch(&key, psi, nd, sizeof(okey), okey_cmp)) {
      r->excluded++;
    } else {
      double habs = 0.0, hii = diag_with_abs(&I, key.a, key.b, &habs);
      r->a[k] = key.a;
      r->b[k] = key.b;
      r->num[k] = nsum_get(&num);
      r->abssum[k] = nsum_get(&abssum);
      r->haa[k] = hii;
      r->haa_abs[k] = habs;
      r->score[k] = r->num[k] / (E0 - hii);
      k++;
    }
    i = j;
  }
  r->ncand = k;
  free(psi);
  free(g.P.v);
  return r;
}

/*
 * All-core form of oracle_search (eps, no bucket filter), for the CPU baseline
 * and for parity runs at sizes the single-core form takes minutes on.  It
 * computes the same result bit for bit: the same core, the same pairs and
 * values, and each target's contributions summed in the same order.
 *  1. The core determinants are enumerated in parallel, each into its
 *     thread's list; a pair's order field is (core rank, position in that
 *     determinant's enumeration), which sorts like the single-core counter.
 *  2. Pairs are scattered into `parts` lists by oracle_bucket_of(target), so
 *     every target's contributions land in one list.
 *  3. The lists are sorted and accumulated in parallel (the loop of
 *     oracle_search), then the candidates of all lists are put in key order.
 */
typedef struct {
  uint64_t a, b;
  double num, abssum, haa, haa_abs, score;
} ocand;

static int ocand_cmp(const void *x, const void *y) {
  const ocand *p = (const ocand *)x, *q = (const ocand *)y;
  return key_cmp(p->a, p->b, q->a, q->b);
}

oresult *oracle_search_parallel(int n, const double *h1, const double *eri, double ecore,
                                const uint64_t *da, const uint64_t *db, const double *c,
                                size_t nd, double E0, size_t C, double eps, int threads) {
  oints I = {n, ecore, h1, eri};
  size_t i, m, t, nparts, total = 0;
  size_t *core, *fill, *cnt, *off;
  ogen *gens;
  opair **part;
  ocand **cand;
  size_t *ncand, *nuniq, *nexcl;
  okey *psi;
  int nt, bad = 0;
  oresult *r = (oresult *)calloc(1, sizeof(oresult));
  if (!r) return NULL;
  nt = threads > 0 ? threads : 1;
  nparts = (size_t)nt * 8;
  core = (size_t *)malloc((nd ? nd : 1) * sizeof(size_t));
  m = oracle_core_select(da, db, c, nd, C, core);
  r->ncore = m;
  gens = (ogen *)calloc((size_t)nt, sizeof(ogen));
  cnt = (size_t *)calloc((size_t)nt * nparts, sizeof(size_t));
  off = (size_t *)calloc((size_t)nt * nparts, sizeof(size_t));
  fill = (size_t *)calloc(nparts + 1, sizeof(size_t));
  part = (opair **)calloc(nparts, sizeof(opair *));
  cand = (ocand **)calloc(nparts, sizeof(ocand *));
  ncand = (size_t *)calloc(nparts, sizeof(size_t));
  nuniq = (size_t *)calloc(nparts, sizeof(size_t));
  nexcl = (size_t *)calloc(nparts, sizeof(size_t));
  psi = (okey *)malloc((nd ? nd : 1) * sizeof(okey));
  if (!core || !gens || !cnt || !off || !fill || !part || !cand || !ncand || !nuniq || !nexcl ||
      !psi) {
    bad = 1;
    goto done;
  }
  for (i = 0; i < nd; i++) {
    psi[i].a = da[i];
    psi[i].b = db[i];
  }
  qsort(psi, nd, sizeof(okey), okey_cmp);

  /* 1. enumeration, one list per thread */
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int me = omp_get_thread_num();
#else
    int me = 0;
#endif
    ogen *g = &gens[me];
    long long k;
    g->I = &I;
    g->E0 = E0;
    g->eps = eps;
    g->nbuckets = 1;
#pragma omp for schedule(dynamic, 4)
    for (k = 0; k < (long long)m; k++) {
      g->P.order = (size_t)k << 32;
      enumerate(g, n, da[core[k]], db[core[k]], c[core[k]]);
    }
  }
  for (t = 0; t < (size_t)nt; t++) {
    if (gens[t].err) bad = 1;
    r->generated += gens[t].generated;
    r->surviving += gens[t].surviving;
  }
  if (bad) goto done;

  /* 2. scatter by target bucket (counts per thread and bucket, then offsets) */
#pragma omp parallel for num_threads(nt) schedule(static, 1)
  for (t = 0; t < (size_t)nt; t++) {
    size_t q;
    for (q = 0; q < gens[t].P.n; q++)
      cnt[t * nparts + oracle_bucket_of(gens[t].P.v[q].a, gens[t].P.v[q].b, nparts)]++;
  }
  for (i = 0; i < nparts; i++) {
    size_t run = 0;
    for (t = 0; t < (size_t)nt; t++) {
      off[t * nparts + i] = run;
      run += cnt[t * nparts + i];
    }
    fill[i] = run;
    total += run;
    part[i] = (opair *)malloc((run ? run : 1) * sizeof(opair));
    if (!part[i]) bad = 1;
  }
  if (bad) goto done;
#pragma omp parallel for num_threads(nt) schedule(static, 1)
  for (t = 0; t < (size_t)nt; t++) {
    size_t q;
    for (q = 0; q < gens[t].P.n; q++) {
      const opair *p = &gens[t].P.v[q];
      size_t bkt = oracle_bucket_of(p->a, p->b, nparts);
      part[bkt][off[t * nparts + bkt]++] = *p;
    }
    free(gens[t].P.v);
    gens[t].P.v = NULL;
  }

  /* 3. sort and accumulate each list */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (i = 0; i < nparts; i++) {
    size_t q, u = 0, k = 0, np = fill[i];
    opair *v = part[i];
    qsort(v, np, sizeof(opair), opair_cmp);
    for (q = 0; q < np; q++)
      if (q == 0 || key_cmp(v[q].a, v[q].b, v[q - 1].a, v[q - 1].b)) u++;
    nuniq[i] = u;
    cand[i] = (ocand *)malloc((u ? u : 1) * sizeof(ocand));
    if (!cand[i]) continue;
    for (q = 0; q < np;) {
      size_t j = q;
      nsum num = {0.0, 0.0}, abssum = {0.0, 0.0};
      okey key;
      while (j < np && !key_cmp(v[j].a, v[j].b, v[q].a, v[q].b)) {
        nsum_add(&num, v[j].v);
        nsum_add(&abssum, fabs(v[j].v));
        j++;
      }
      key.a = v[q].a;
      key.b = v[q].b;
      if (nd && bsearch(&key, psi, nd, sizeof(okey), okey_cmp)) {
        nexcl[i]++;
      } else {
        ocand *o = &cand[i][k++];
        o->a = key.a;
        o->b = key.b;
        o->haa = diag_with_abs(&I, key.a, key.b, &o->haa_abs);
        o->num = nsum_get(&num);
        o->abssum = nsum_get(&abssum);
        o->score = o->num / (E0 - o->haa);
      }
      q = j;
    }
    ncand[i] = k;
    free(part[i]);
    part[i] = NULL;
  }

  /* 4. every list's candidates, in key order */
  {
    size_t u = 0, k = 0, e = 0;
    ocand *all;
    for (i = 0; i < nparts; i++) {
      if (!cand[i]) bad = 1;
      u += ncand[i];
      r->unique += nuniq[i];
      e += nexcl[i];
    }
    r->excluded = e;
    if (bad) goto done;
    all = (ocand *)malloc((u ? u : 1) * sizeof(ocand));
    r->a = (uint64_t *)malloc((u ? u : 1) * sizeof(uint64_t));
    r->b = (uint64_t *)malloc((u ? u : 1) * sizeof(uint64_t));
    r->num = (double *)malloc((u ? u : 1) * sizeof(double));
    r->abssum = (double *)malloc((u ? u : 1) * sizeof(double));
    r->haa = (double *)malloc((u ? u : 1) * sizeof(double));
    r->haa_abs = (double *)malloc((u ? u : 1) * sizeof(double));
    r->score = (double *)malloc((u ? u : 1) * sizeof(double));
    if (!all || !r->a || !r->b || !r->num || !r->abssum || !r->haa || !r->haa_abs || !r->score) {
      free(all);
      bad = 1;
      goto done;
    }
    for (i = 0; i < nparts; i++) {
      memcpy(all + k, cand[i], ncand[i] * sizeof(ocand));
      k += ncand[i];
    }
    qsort(all, u, sizeof(ocand), ocand_cmp);
    for (k = 0; k < u; k++) {
      r->a[k] = all[k].a;
      r->b[k] = all[k].b;
      r->num[k] = all[k].num;
      r->abssum[k] = all[k].abssum;
      r->haa[k] = all[k].haa;
      r->haa_abs[k] = all[k].haa_abs;
      r->score[k] = all[k].score;
    }
    r->ncand = u;
    free(all);
  }

done:
  if (gens)
    for (t = 0; t < (size_t)nt; t++) free(gens[t].P.v);
  if (part)
    for (i = 0; i < nparts; i++) free(part[i]);
  if (cand)
    for (i = 0; i < nparts; i++) free(cand[i]);
  free(gens);
  free(cnt);
  free(off);
  free(fill);
  free(part);
  free(cand);
  free(ncand);
  free(nuniq);
  free(nexcl);
  free(psi);
  free(core);
  if (bad) {
    oracle_free(r);
    return NULL;
  }
  return r;
}

size_t oracle_result_count(const oresult *r) { return r ? r->ncand : 0; }

void oracle_result_stats(const oresult *r, size_t *out5) {
  out5[0] = r->generated;
  out5[1] = r->surviving;
  out5[2] = r->unique;
  out5[3] = r->excluded;
  out5[4] = r->ncore;
}

void oracle_result_copy(const oresult *r, uint64_t *a, uint64_t *b, double *num, double *abssum,
                        double *haa, double *haa_abs, double *score) {
  size_t k = r->ncand;
  memcpy(a, r->a, k * sizeof(uint64_t));
  memcpy(b, r->b, k * sizeof(uint64_t));
  memcpy(num, r->num, k * sizeof(double));
  memcpy(abssum, r->abssum, k * sizeof(double));
  memcpy(haa, r->haa, k * sizeof(double));
  memcpy(haa_abs, r->haa_abs, k * sizeof(double));
  memcpy(score, r->score, k * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* selection (Sec. 2.2, "selection problem")                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t a, b;
  double abss;
  size_t idx;
} osel;

static int osel_cmp(const void *x, const void *y) {
  const osel *p = (const osel *)x, *q = (const osel *)y;
  if (p->abss != q->abss) return p->abss > q->abss ? -1 : 1;
  return key_cmp(p->a, p->b, q->a, q->b);
}

/* Indices of the top-N candidates by |score|, ties by key ascending.
 * Writes min(N, n) indices in rank order and returns that count. */
size_t oracle_topn(const uint64_t *a, const uint64_t *b, const double *score, size_t n, size_t N,
                   size_t *out_idx) {
  size_t i, m = N < n ? N : n;
  osel *v = (osel *)malloc((n ? n : 1) * sizeof(osel));
  if (!v) return 0;
  for (i = 0; i < n; i++) {
    v[i].a = a[i];
    v[i].b = b[i];
    v[i].abss = fabs(score[i]);
    v[i].idx = i;
  }
  qsort(v, n, sizeof(osel), osel_cmp);
  for (i = 0; i < m; i++) out_idx[i] = v[i].idx;
  free(v);
  return m;
}

/* ------------------------------------------------------------------------ */
/* per-stage views used by the tests                                        */
/* ------------------------------------------------------------------------ */

double oracle_hij(int n, const double *h1, const double *eri, double ecore, uint64_t bra_a,
                  uint64_t bra_b, uint64_t ket_a, uint64_t ket_b) {
  oints I = {n, ecore, h1, eri};
  return oracle_hij_impl(&I, bra_a, bra_b, ket_a, ket_b);
}

double oracle_diag(int n, const double *h1, const double *eri, double ecore, uint64_t a,
                   uint64_t b) {
  oints I = {n, ecore, h1, eri};
  return oracle_diag_impl(&I, a, b);
}

/* Sum of the magnitudes of the terms of <D|H|D> (the scale of its rounding
 * error). */
double oracle_diag_abs(int n, const double *h1, const double *eri, double ecore, uint64_t a,
                       uint64_t b) {
  oints I = {n, ecore, h1, eri};
  double m = 0.0;
  diag_with_abs(&I, a, b, &m);
  return m;
}

/* Dense matrix H[i][j] = <D_i|H|D_j> over a list of determinants (row-major). */
void oracle_dense_h(int n, const double *h1, const double *eri, double ecore, const uint64_t *da,
                    const uint64_t *db, size_t nd, double *out) {
  oints I = {n, ecore, h1, eri};
  size_t i, j;
  for (i = 0; i < nd; i++)
    for (j = 0; j < nd; j++) out[i * nd + j] = oracle_hij_impl(&I, da[i], db[i], da[j], db[j]);
}

/* Selected dense rows of the same matrix: out[r][j] = <D_rows[r]|H|D_j>. */
void oracle_h_rows(int n, const double *h1, const double *eri, double ecore, const uint64_t *da,
                   const uint64_t *db, size_t nd, const size_t *rows, size_t nrows, double *out) {
  oints I = {n, ecore, h1, eri};
  size_t r, j;
  for (r = 0; r < nrows; r++) {
    size_t i = rows[r];
    for (j = 0; j < nd; j++) out[r * nd + j] = oracle_hij_impl(&I, da[i], db[i], da[j], db[j]);
  }
}

/* The pre-sort pair list of Alg. 2 for the given core determinants, in
 * generation order (eps = 0).  Returns the number of pairs written; call with
 * cap == 0 to get the count only. */
size_t oracle_pairs(int n, const double *h1, const double *eri, double ecore, const uint64_t *ca,
                    const uint64_t *cb, const double *cc, size_t ncore, size_t cap,
                    uint64_t *out_a, uint64_t *out_b, double *out_v) {
  oints I = {n, ecore, h1, eri};
  ogen g;
  size_t i, k;
  memset(&g, 0, sizeof(g));
  g.I = &I;
  g.nbuckets = 1;
  for (i = 0; i < ncore; i++) enumerate(&g, n, ca[i], cb[i], cc[i]);
  if (g.err) {
    free(g.P.v);
    return 0;
  }
  for (k = 0; k < g.P.n && k < cap; k++) {
    out_a[k] = g.P.v[k].a;
    out_b[k] = g.P.v[k].b;
    out_v[k] = g.P.v[k].v;
  }
  k = g.P.n;
  free(g.P.v);
  return k;
}

/* Numerator of Eq. 1 for one target, by brute force over the core list:
 * sum_j <target|H|D_j> c_j over every core determinant (no enumeration). */
double oracle_numerator(int n, const double *h1, const double *eri, double ecore, uint64_t ta,
                        uint64_t tb, const uint64_t *ca, const uint64_t *cb, const double *cc,
                        size_t ncore, double *abssum_out) {
  oints I = {n, ecore, h1, eri};
  nsum num = {0.0, 0.0}, abssum = {0.0, 0.0};
  size_t j;
  for (j = 0; j < ncore; j++) {
    uint64_t xa = ta ^ ca[j], xb = tb ^ cb[j];
    if (count_bits(xa) + count_bits(xb) > 4 || (xa == 0 && xb == 0)) continue;
    {
      double v = oracle_hij_impl(&I, ta, tb, ca[j], cb[j]) * cc[j];
      nsum_add(&num, v);
      nsum_add(&abssum, fabs(v));
    }
  }
  if (abssum_out) *abssum_out = nsum_get(&abssum);
  return nsum_get(&num);
}
