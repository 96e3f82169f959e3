/*
 * Plain FP64 CPU oracle for the screened periodic LRI exchange matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference the CUDA
 * library is checked against; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the library.
 *
 * What it computes (Sec. II of the paper):
 *   Eq. HFX_ERIs   Sigma_{Ii,Jj} = sum_{K,L} sum_{k,l} (Ii Kk | Jj Ll) D_{Kk,Ll}
 *   Eq. LRI        phi_Ii phi_Kk ~ sum_{A in {I,K}} sum_alpha C^{A alpha}_{Ii,Kk} P_{A alpha}
 *                  with {I,K} a SET of sites: one term when K is I.
 *   Eq. HFX_LRI /  the four pieces, one per placement of the two ABF centres
 *   Eq. HFX_split  (A in {I,K}, B in {J,L}), each a partial ERI (Eq. partial_
 *                  integrals) contracted with D_{K,L}.
 * in the loop order of Algorithm 1 (pairs <I,J> outermost, K in N[I] and
 * L in N[J] inside, four partial-ERI terms per (K,L)), each term evaluated in
 * the C((VC)D) multiplication order the paper adopts (Appendix A, Table 1):
 *   Y[alpha][j][l] = sum_beta V_AB[alpha][beta] cB[beta][j][l]
 *   T[alpha][j][k] = sum_l    Y[alpha][j][l] D_KL[k][l]
 *   Ht[i][j]       = sum_{alpha,k} cA[alpha][i][k] T[alpha][j][k]
 * Y for A = I does not depend on K and is computed once per (J, L, B) entry
 * (loop-invariant, same values).
 *
 * Readings where the paper is silent:
 *  - sign: Sigma carries an overall minus sign and E_X = 1/2 sum D.Sigma;
 *  - screening: a term survives iff S > theta with
 *      S = (maxabs(C_A-side) * maxabs(C_B-side)) * (maxabs(V_AB) * maxabs(D_KL)),
 *    multiplied in exactly that association in round-to-nearest FP64 (block
 *    upper limits, Sec. III.B; strict ">" as in Algorithm 4);
 *  - optional Cauchy-Schwarz ERI screen (Sec. III.C, Eq. CS-ERI; orc_set_eri):
 *    a term also needs sqrt(Q_AF) * sqrt(Q_BG) > eps_eri, Q the largest
 *    diagonal ERI of the AO-pair sites {A, F} and {B, G} under Eq. LRI;
 *  - a block exists iff it was supplied; missing blocks are zero.
 *
 * Coefficient roles: cA[alpha][i][k] = C(I,K)[alpha][i][k] when A = I and
 * C(K,I)[alpha][k][i] when A = K (K not I); cB likewise for (J, L).
 *
 * Accumulation of the terms into each Sigma element is Neumaier-compensated.
 *
 * Keys are (i, j, n1, n2, n3): the block between site (i, 0) and site (j, n).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { int32_t a, n[3]; } site_t;

/* ---------------- key hash (open addressing) ---------------- */
static uint64_t pack_key(int32_t i, int32_t j, int32_t n1, int32_t n2, int32_t n3) {
  return ((uint64_t)(uint32_t)i << 44) | ((uint64_t)(uint32_t)j << 24) |
         ((uint64_t)((n1 + 128) & 0xFF) << 16) | ((uint64_t)((n2 + 128) & 0xFF) << 8) |
         (uint64_t)((n3 + 128) & 0xFF);
}
static uint64_t mix64(uint64_t x) {
  x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ULL;
  x ^= x >> 27; x *= 0x94d049bb133111ebULL;
  x ^= x >> 31; return x;
}
typedef struct { uint64_t *keys; int64_t *vals; uint64_t mask; int64_t count; } hmap_t;
#define EMPTY_KEY (~0ULL)

static void hm_init(hmap_t *h, int64_t expected) {
  uint64_t cap = 16;
  while (cap < (uint64_t)(expected * 2 + 16)) cap <<= 1;
  h->keys = (uint64_t *)malloc(cap * sizeof(uint64_t));
  h->vals = (int64_t *)malloc(cap * sizeof(int64_t));
  for (uint64_t s = 0; s < cap; ++s) h->keys[s] = EMPTY_KEY;
  h->mask = cap - 1;
  h->count = 0;
}
static void hm_free(hmap_t *h) { free(h->keys); free(h->vals); }
static void hm_grow(hmap_t *h);
/* insert if absent; returns the value stored for the key */
static int64_t hm_put(hmap_t *h, uint64_t k, int64_t v) {
  if ((uint64_t)(h->count + 1) * 2 > h->mask + 1) hm_grow(h);
  uint64_t s = mix64(k) & h->mask;
  while (h->keys[s] != EMPTY_KEY) {
    if (h->keys[s] == k) return h->vals[s];
    s = (s + 1) & h->mask;
  }
  h->keys[s] = k; h->vals[s] = v; h->count++;
  return v;
}
static void hm_grow(hmap_t *h) {
  hmap_t n;
  hm_init(&n, (int64_t)(h->mask + 1));
  for (uint64_t s = 0; s <= h->mask; ++s)
    if (h->keys[s] != EMPTY_KEY) hm_put(&n, h->keys[s], h->vals[s]);
  hm_free(h);
  *h = n;
}
static int64_t hm_get(const hmap_t *h, uint64_t k) {
  uint64_t s = mix64(k) & h->mask;
  while (h->keys[s] != EMPTY_KEY) {
    if (h->keys[s] == k) return h->vals[s];
    s = (s + 1) & h->mask;
  }
  return -1;
}

/* ---------------- block sets ---------------- */
typedef struct {
  int64_t n;
  const int32_t *keys;   /* n x 5 */
  const double *data;
  const int64_t *offs;   /* n + 1 */
  double *maxabs;        /* per block upper limit (Sec. III.B) */
  hmap_t map;
} bset_t;

typedef struct { int32_t other, n[3]; int64_t blk; } nbr_t;

typedef struct orc {
  int32_t natoms;
  int32_t *nao, *nabf;
  bset_t C, V, D;
  /* per atom x: C(x, y, n) blocks ("out") and C(y, x, m) blocks ("in") */
  int64_t *cout_start, *cin_start;
  nbr_t *cout, *cin;
  /* per atom a: V(a, b, n) blocks */
  int64_t *vout_start;
  nbr_t *vout;
  /* Cauchy-Schwarz ERI screen: per C block sqrt(max(Q, 0)); off when !eri_on */
  int eri_on;
  double eps_eri;
  double *eri_sq;
} orc;

static void bset_init(bset_t *b, int64_t n, const int32_t *keys, const double *data,
                      const int64_t *offs) {
  b->n = n; b->keys = keys; b->data = data; b->offs = offs;
  b->maxabs = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  hm_init(&b->map, n);
  for (int64_t e = 0; e < n; ++e) {
    const int32_t *k = keys + 5 * e;
    hm_put(&b->map, pack_key(k[0], k[1], k[2], k[3], k[4]), e);
    double m = 0.0;
    for (int64_t t = offs[e]; t < offs[e + 1]; ++t) {
      double a = fabs(data[t]);
      if (a > m) m = a;
    }
    b->maxabs[e] = m;
  }
}

static int64_t bset_find(const bset_t *b, int32_t i, int32_t j, const int32_t n[3]) {
  return hm_get(&b->map, pack_key(i, j, n[0], n[1], n[2]));
}

orc *orc_create(int32_t natoms, const int32_t *nao, const int32_t *nabf,
                int64_t nC, const int32_t *kC, const double *dC, const int64_t *oC,
                int64_t nV, const int32_t *kV, const double *dV, const int64_t *oV,
                int64_t nD, const int32_t *kD, const double *dD, const int64_t *oD) {
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->natoms = natoms;
  o->nao = (int32_t *)malloc(sizeof(int32_t) * natoms);
  o->nabf = (int32_t *)malloc(sizeof(int32_t) * natoms);
  memcpy(o->nao, nao, sizeof(int32_t) * natoms);
  memcpy(o->nabf, nabf, sizeof(int32_t) * natoms);
  bset_init(&o->C, nC, kC, dC, oC);
  bset_init(&o->V, nV, kV, dV, oV);
  bset_init(&o->D, nD, kD, dD, oD);
  /* neighbour lists from the C key set */
  o->cout_start = (int64_t *)calloc(natoms + 1, sizeof(int64_t));
  o->cin_start = (int64_t *)calloc(natoms + 1, sizeof(int64_t));
  for (int64_t e = 0; e < nC; ++e) {
    o->cout_start[kC[5 * e] + 1]++;
    o->cin_start[kC[5 * e + 1] + 1]++;
  }
  for (int32_t a = 0; a < natoms; ++a) {
    o->cout_start[a + 1] += o->cout_start[a];
    o->cin_start[a + 1] += o->cin_start[a];
  }
  o->cout = (nbr_t *)malloc(sizeof(nbr_t) * (nC > 0 ? nC : 1));
  o->cin = (nbr_t *)malloc(sizeof(nbr_t) * (nC > 0 ? nC : 1));
  int64_t *fo = (int64_t *)malloc(sizeof(int64_t) * (natoms + 1));
  int64_t *fi = (int64_t *)malloc(sizeof(int64_t) * (natoms + 1));
  memcpy(fo, o->cout_start, sizeof(int64_t) * (natoms + 1));
  memcpy(fi, o->cin_start, sizeof(int64_t) * (natoms + 1));
  for (int64_t e = 0; e < nC; ++e) {
    const int32_t *k = kC + 5 * e;
    nbr_t *p = &o->cout[fo[k[0]]++];
    p->other = k[1]; p->n[0] = k[2]; p->n[1] = k[3]; p->n[2] = k[4]; p->blk = e;
    /* C(y, x, m): seen from x at cell 0, y sits at cell -m */
    nbr_t *q = &o->cin[fi[k[1]]++];
    q->other = k[0]; q->n[0] = -k[2]; q->n[1] = -k[3]; q->n[2] = -k[4]; q->blk = e;
  }
  free(fo); free(fi);
  o->vout_start = (int64_t *)calloc(natoms + 1, sizeof(int64_t));
  for (int64_t e = 0; e < nV; ++e) o->vout_start[kV[5 * e] + 1]++;
  for (int32_t a = 0; a < natoms; ++a) o->vout_start[a + 1] += o->vout_start[a];
  o->vout = (nbr_t *)malloc(sizeof(nbr_t) * (nV > 0 ? nV : 1));
  int64_t *fv = (int64_t *)malloc(sizeof(int64_t) * (natoms + 1));
  memcpy(fv, o->vout_start, sizeof(int64_t) * (natoms + 1));
  for (int64_t e = 0; e < nV; ++e) {
    const int32_t *k = kV + 5 * e;
    nbr_t *p = &o->vout[fv[k[0]]++];
    p->other = k[1]; p->n[0] = k[2]; p->n[1] = k[3]; p->n[2] = k[4]; p->blk = e;
  }
  free(fv);
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  hm_free(&o->C.map); hm_free(&o->V.map); hm_free(&o->D.map);
  free(o->C.maxabs); free(o->V.maxabs); free(o->D.maxabs);
  free(o->cout_start); free(o->cin_start); free(o->cout); free(o->cin);
  free(o->vout_start); free(o->vout);
  free(o->eri_sq);
  free(o->nao); free(o->nabf); free(o);
}

/* x^T V y over the V block between two sites (row-major [nx][ny]); a missing
 * block (v < 0) contributes zero. */
static double vform(const orc *o, int64_t v, const double *x, int nx, const double *y, int ny) {
  if (v < 0) return 0.0;
  const double *V = o->V.data + o->V.offs[v];
  double q = 0.0;
  for (int al = 0; al < nx; ++al) {
    double t = 0.0;
    for (int be = 0; be < ny; ++be) t += V[(int64_t)al * ny + be] * y[be];
    q += x[al] * t;
  }
  return q;
}

/*
 * Cauchy-Schwarz ERI screen (Sec. III.C, Eq. CS-ERI).  For every C block
 * (x, y, n) -- the AO-pair sites X = (x, 0), Y = (y, n) -- the largest diagonal
 * ERI Q = max over a in x, f in y of (phi_Xa phi_Yf | phi_Xa phi_Yf).  By
 * Eq. LRI the pair is sum_alpha C(x,y,n)[alpha][a][f] P_{X alpha} plus, when Y
 * is another site, sum_beta C(y,x,-n)[beta][f][a] P_{Y beta}; the diagonal ERI
 * is the V-norm of that expansion, with the V blocks V_XX, V_XY, V_YX, V_YY
 * (missing blocks and missing C(y,x,-n) are zero).  Q is the same for both C
 * blocks of one site pair.  A term with AO pairs {A,F} and {B,G} (C blocks
 * eK and eL) is then kept only if sqrt(max(Q_eK, 0)) * sqrt(max(Q_eL, 0)) >
 * eps; eps < 0 turns the screen off.
 */
void orc_set_eri(orc *o, double eps) {
  free(o->eri_sq);
  o->eri_sq = NULL;
  o->eri_on = eps >= 0.0;
  o->eps_eri = eps;
  if (!o->eri_on) return;
  o->eri_sq = (double *)malloc(sizeof(double) * (size_t)(o->C.n > 0 ? o->C.n : 1));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t e = 0; e < o->C.n; ++e) {
    const int32_t *k = o->C.keys + 5 * e;
    const int32_t x = k[0], y = k[1];
    const int32_t zero[3] = {0, 0, 0}, n[3] = {k[2], k[3], k[4]}, m[3] = {-k[2], -k[3], -k[4]};
    const int px = o->nabf[x], py = o->nabf[y], nx = o->nao[x], ny = o->nao[y];
    const int same = x == y && n[0] == 0 && n[1] == 0 && n[2] == 0;
    const double *cX = o->C.data + o->C.offs[e];
    const int64_t eY = same ? -1 : bset_find(&o->C, y, x, m);
    const double *cY = eY >= 0 ? o->C.data + o->C.offs[eY] : NULL;
    const int64_t vXX = bset_find(&o->V, x, x, zero);
    const int64_t vXY = same ? -1 : bset_find(&o->V, x, y, n);
    const int64_t vYX = same ? -1 : bset_find(&o->V, y, x, m);
    const int64_t vYY = same ? -1 : bset_find(&o->V, y, y, zero);
    double *u = (double *)malloc(sizeof(double) * (size_t)(px + py));
    double *w = u + px;
    double qmax = -INFINITY;
    for (int a = 0; a < nx; ++a)
      for (int f = 0; f < ny; ++f) {
        for (int al = 0; al < px; ++al) u[al] = cX[((int64_t)al * nx + a) * ny + f];
        double q = vform(o, vXX, u, px, u, px);
        if (!same) {
          for (int be = 0; be < py; ++be) w[be] = cY ? cY[((int64_t)be * ny + f) * nx + a] : 0.0;
          q += vform(o, vXY, u, px, w, py) + vform(o, vYX, w, py, u, px) +
               vform(o, vYY, w, py, w, py);
        }
        if (q > qmax) qmax = q;
      }
    free(u);
    o->eri_sq[e] = sqrt(qmax > 0.0 ? qmax : 0.0);
  }
}

/* sqrt(max(Q, 0)) per C block of the last orc_set_eri (zeros when off). */
void orc_eri_sq(const orc *o, double *out) {
  for (int64_t e = 0; e < o->C.n; ++e) out[e] = o->eri_on ? o->eri_sq[e] : 0.0;
}

/* One way an ABF centre is placed for an AO pair (X, Y), X the Sigma-side site:
 * the partner site Y, the ABF site (X itself or Y), the C block and whether it
 * is read transposed (ABFs on Y: C(Y,X)[alpha][y][x]). */
typedef struct { site_t partner, abf; int64_t cblk; int transposed; } role_t;

/* All (partner, ABF centre) entries for the Sigma-side site X = (x, nx):
 * partner Y with C(X,Y) present -> ABF on X; Y != X with C(Y,X) present -> ABF on Y. */
static int64_t roles_of(const orc *o, int32_t x, const int32_t nx[3], role_t **out) {
  int64_t n_out = o->cout_start[x + 1] - o->cout_start[x];
  int64_t n_in = o->cin_start[x + 1] - o->cin_start[x];
  role_t *r = (role_t *)malloc(sizeof(role_t) * (size_t)(n_out + n_in + 1));
  int64_t c = 0;
  for (int64_t t = o->cout_start[x]; t < o->cout_start[x + 1]; ++t) {
    const nbr_t *p = &o->cout[t];
    role_t *e = &r[c++];
    e->partner.a = p->other;
    for (int d = 0; d < 3; ++d) e->partner.n[d] = nx[d] + p->n[d];
    e->abf.a = x;
    for (int d = 0; d < 3; ++d) e->abf.n[d] = nx[d];
    e->cblk = p->blk; e->transposed = 0;
  }
  for (int64_t t = o->cin_start[x]; t < o->cin_start[x + 1]; ++t) {
    const nbr_t *p = &o->cin[t];
    int same = (p->other == x) && p->n[0] == 0 && p->n[1] == 0 && p->n[2] == 0;
    if (same) continue; /* {X, Y} is one site: the single term is the ABF-on-X one */
    role_t *e = &r[c++];
    e->partner.a = p->other;
    for (int d = 0; d < 3; ++d) e->partner.n[d] = nx[d] + p->n[d];
    e->abf = e->partner;
    e->cblk = p->blk; e->transposed = 1;
  }
  *out = r;
  return c;
}

static int same_site(const site_t *a, const site_t *b) {
  return a->a == b->a && a->n[0] == b->n[0] && a->n[1] == b->n[1] && a->n[2] == b->n[2];
}

/* Block between two sites: key (x, y, ny - nx). */
static int64_t find_between(const bset_t *b, const site_t *x, const site_t *y) {
  int32_t n[3] = {y->n[0] - x->n[0], y->n[1] - x->n[1], y->n[2] - x->n[2]};
  return bset_find(b, x->a, y->a, n);
}

/* Screening quantity of one term, in the fixed association. */
static double screen_S(const orc *o, const role_t *eK, const role_t *eL, int64_t v, int64_t d) {
  double cc = o->C.maxabs[eK->cblk] * o->C.maxabs[eL->cblk];
  double vd = o->V.maxabs[v] * o->D.maxabs[d];
  return cc * vd;
}

/* Does a term survive: the block screen S > theta and, when on, the
 * Cauchy-Schwarz ERI screen of its two AO pairs. */
static int survives(const orc *o, const role_t *eK, const role_t *eL, int64_t v, int64_t d,
                    double theta) {
  if (!(screen_S(o, eK, eL, v, d) > theta)) return 0;
  if (o->eri_on && !(o->eri_sq[eK->cblk] * o->eri_sq[eL->cblk] > o->eps_eri)) return 0;
  return 1;
}

/* variant index: 0 = ABFs on (I,J), 1 = (I,L), 2 = (K,J), 3 = (K,L) */
static int variant_of(const role_t *eK, const role_t *eL) {
  return (eK->transposed ? 2 : 0) + (eL->transposed ? 1 : 0);
}

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return (a > b) - (a < b);
}
void orc_sort_u64(uint64_t *v, int64_t n) { qsort(v, (size_t)n, sizeof(uint64_t), cmp_u64); }

/*
 * Enumerate the Sigma key set at theta for central atoms i in [a0, a1): every
 * (i, j, n) receiving at least one surviving term, and the number of
 * surviving terms per variant.  Returns the number of keys; writes at most
 * cap keys (sorted) when keys_out is non-null.  extra (nullable) receives
 * [0] the number of distinct (A, B, G) triples with a surviving term and
 * [1] the Algorithm 3 multiply-add count of the build: per surviving term the
 * T and Ht contractions, per active (A, B, G) the product Y = V C_BG.
 */
int64_t orc_keys(orc *o, double theta, int32_t a0, int32_t a1, int32_t *keys_out, int64_t cap,
                 int64_t counts[4], int64_t extra[2]) {
  if (a0 < 0) a0 = 0;
  if (a1 > o->natoms || a1 <= 0) a1 = o->natoms;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  hmap_t *keysets = (hmap_t *)malloc(sizeof(hmap_t) * nth);
  hmap_t *triples = (hmap_t *)malloc(sizeof(hmap_t) * nth);
  int64_t *cnt = (int64_t *)calloc((size_t)nth * 5, sizeof(int64_t));
  for (int t = 0; t < nth; ++t) { hm_init(&keysets[t], 1024); hm_init(&triples[t], 1024); }
#pragma omp parallel num_threads(nth)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    hmap_t *ks = &keysets[tid], *tr = &triples[tid];
    int64_t *c = cnt + 5 * tid;
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = a0; i < a1; ++i) {
      int32_t zero[3] = {0, 0, 0};
      site_t I = {i, {0, 0, 0}};
      role_t *KI;
      int64_t nK = roles_of(o, i, zero, &KI);
      for (int64_t a = 0; a < nK; ++a) {
        const role_t *eK = &KI[a];
        const site_t *A = &eK->abf, *K = &eK->partner;
        const site_t *F = same_site(A, &I) ? K : &I;   /* the AO site without the ABFs */
        const int64_t pA = o->nabf[A->a], na = o->nao[A->a], nf = o->nao[F->a];
        /* B: every site with V(A, B) */
        for (int64_t tv = o->vout_start[A->a]; tv < o->vout_start[A->a + 1]; ++tv) {
          const nbr_t *pv = &o->vout[tv];
          const int64_t vb = pv->blk;
          site_t B = {pv->other, {A->n[0] + pv->n[0], A->n[1] + pv->n[1], A->n[2] + pv->n[2]}};
          const int64_t pB = o->nabf[B.a], nb = o->nao[B.a];
          const int64_t dKB = find_between(&o->D, K, &B);
          /* every C(B, Y) block: either J = B with L = Y (ABFs on J), or L = B with
           * J = Y != B (ABFs on L); in both cases Y is the site G without ABFs */
          for (int64_t t = o->cout_start[B.a]; t < o->cout_start[B.a + 1]; ++t) {
            const nbr_t *p = &o->cout[t];
            site_t Y = {p->other, {B.n[0] + p->n[0], B.n[1] + p->n[1], B.n[2] + p->n[2]}};
            const int64_t ng = o->nao[Y.a];
            int alive = 0;
            role_t eL;
            /* J = B, L = Y */
            int64_t d = find_between(&o->D, K, &Y);
            if (d >= 0) {
              eL.partner = Y; eL.abf = B; eL.cblk = p->blk; eL.transposed = 0;
              if (survives(o, eK, &eL, vb, d, theta)) {
                const int v = variant_of(eK, &eL);
                c[v]++;
                alive = 1;
                /* v1: T[al,b,f] over g, Ht over (al,f);  v3: T[al,a,b] over g, Ht over (al,a) */
                c[4] += v == 0 ? pA * nb * nf * (ng + na) : pA * na * nb * (ng + nf);
                hm_put(ks, pack_key(i, B.a, B.n[0], B.n[1], B.n[2]), 0);
              }
            }
            /* L = B, J = Y */
            if (dKB >= 0 && !same_site(&Y, &B)) {
              eL.partner = B; eL.abf = B; eL.cblk = p->blk; eL.transposed = 1;
              if (survives(o, eK, &eL, vb, dKB, theta)) {
                const int v = variant_of(eK, &eL);
                c[v]++;
                alive = 1;
                /* v2: T[al,f,g] over b, Ht over (al,f);  v4: T[al,a,g] over b, Ht over (al,a) */
                c[4] += v == 1 ? pA * nf * ng * (nb + na) : pA * na * ng * (nb + nf);
                hm_put(ks, pack_key(i, Y.a, Y.n[0], Y.n[1], Y.n[2]), 0);
              }
            }
            /* (A, B, G) with A moved to the home cell: (V block, C(B,G) block) */
            if (alive) hm_put(tr, ((uint64_t)vb << 32) | (uint64_t)p->blk, pA * pB * nb * ng);
          }
        }
      }
      free(KI);
    }
  }
  /* merge: keys are disjoint per central atom, triples are not */
  int64_t nk = 0;
  for (int t = 0; t < nth; ++t) nk += keysets[t].count;
  uint64_t *kall = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk > 0 ? nk : 1));
  int64_t c = 0;
  for (int t = 0; t < nth; ++t)
    for (uint64_t sl = 0; sl <= keysets[t].mask; ++sl)
      if (keysets[t].keys[sl] != EMPTY_KEY) kall[c++] = keysets[t].keys[sl];
  orc_sort_u64(kall, nk);
  hmap_t tall;
  hm_init(&tall, 1024);
  for (int t = 0; t < nth; ++t)
    for (uint64_t sl = 0; sl <= triples[t].mask; ++sl)
      if (triples[t].keys[sl] != EMPTY_KEY) hm_put(&tall, triples[t].keys[sl], triples[t].vals[sl]);
  int64_t ymacs = 0;
  for (uint64_t sl = 0; sl <= tall.mask; ++sl)
    if (tall.keys[sl] != EMPTY_KEY) ymacs += tall.vals[sl];
  if (keys_out) {
    for (int64_t e = 0; e < nk && e < cap; ++e) {
      uint64_t k = kall[e];
      keys_out[5 * e + 0] = (int32_t)(k >> 44);
      keys_out[5 * e + 1] = (int32_t)((k >> 24) & 0xFFFFF);
      keys_out[5 * e + 2] = (int32_t)((k >> 16) & 0xFF) - 128;
      keys_out[5 * e + 3] = (int32_t)((k >> 8) & 0xFF) - 128;
      keys_out[5 * e + 4] = (int32_t)(k & 0xFF) - 128;
    }
  }
  int64_t tot[5] = {0, 0, 0, 0, 0};
  for (int t = 0; t < nth; ++t)
    for (int v = 0; v < 5; ++v) tot[v] += cnt[5 * t + v];
  if (counts) for (int v = 0; v < 4; ++v) counts[v] = tot[v];
  if (extra) { extra[0] = tall.count; extra[1] = tot[4] + ymacs; }
  for (int t = 0; t < nth; ++t) { hm_free(&keysets[t]); hm_free(&triples[t]); }
  free(keysets); free(triples); free(cnt); free(kall);
  hm_free(&tall);
  return nk;
}

/* Neumaier-compensated accumulation. */
static void kahan_add(double *s, double *c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

/* Copy an entry's coefficients into cbuf[alpha][x][y] (x on the Sigma-side
 * site, y on its partner): the C block straight, or transposed in its AO pair. */
static void load_coef(const orc *o, const role_t *e, int nx, int ny, int np, double *cbuf) {
  const double *b = o->C.data + o->C.offs[e->cblk];
  if (!e->transposed) {
    memcpy(cbuf, b, sizeof(double) * (size_t)np * nx * ny);
    return;
  }
  for (int al = 0; al < np; ++al)
    for (int x = 0; x < nx; ++x)
      for (int y = 0; y < ny; ++y)
        cbuf[((int64_t)al * nx + x) * ny + y] = b[((int64_t)al * ny + y) * nx + x];
}

enum { MAXAO = 64, MAXABF = 128, SLAB = MAXABF * MAXAO * MAXAO };

/*
 * Sigma block (I, J) for I = (i, 0), J = (j, n): Algorithm 1 for one pair.
 * out has nao(i) * nao(j) doubles (row-major [i][j]).
 */
static int64_t sigma_block(const orc *o, double theta, int32_t i, int32_t j, const int32_t nJ[3],
                           double *out, double *work) {
  int64_t nterms = 0;
  const int ni = o->nao[i], nj = o->nao[j];
  int32_t zero[3] = {0, 0, 0};
  role_t *KI, *LJ;
  int64_t nK = roles_of(o, i, zero, &KI);
  int64_t nL = roles_of(o, j, nJ, &LJ);
  double *acc = work;                 /* [i][j] running sum */
  double *cmp = acc + MAXAO * MAXAO;  /* compensation */
  double *cB = cmp + MAXAO * MAXAO;   /* [beta][j][l] */
  double *cA = cB + SLAB;             /* [alpha][i][k] */
  double *Y = cA + SLAB;              /* [alpha][j][l] */
  double *YI = Y + SLAB;              /* Y for A = I */
  double *T = YI + SLAB;              /* [alpha][j][k] */
  for (int t = 0; t < ni * nj; ++t) { acc[t] = 0.0; cmp[t] = 0.0; }
  site_t I = {i, {0, 0, 0}};
  for (int64_t b = 0; b < nL; ++b) {
    const role_t *eL = &LJ[b];
    const site_t *L = &eL->partner, *B = &eL->abf;
    const int nl = o->nao[L->a];
    const int pB = o->nabf[B->a];
    int yi_ready = 0, cb_ready = 0;
    for (int64_t a = 0; a < nK; ++a) {
      const role_t *eK = &KI[a];
      const site_t *K = &eK->partner, *A = &eK->abf;
      const int64_t d = find_between(&o->D, K, L);
      if (d < 0) continue;
      const int64_t v = find_between(&o->V, A, B);
      if (v < 0) continue;
      if (!survives(o, eK, eL, v, d, theta)) continue;
      ++nterms;
      const int nk = o->nao[K->a];
      const int pA = o->nabf[A->a];
      const double *Vb = o->V.data + o->V.offs[v];
      const double *Db = o->D.data + o->D.offs[d];
      if (!cb_ready) { load_coef(o, eL, nj, nl, pB, cB); cb_ready = 1; }
      /* Y[alpha][j][l] = sum_beta V_AB[alpha][beta] cB[beta][j][l] */
      double *Yuse;
      const int a_is_I = same_site(A, &I);
      if (a_is_I && yi_ready) {
        Yuse = YI;
      } else {
        Yuse = a_is_I ? YI : Y;
        const int njl = nj * nl;
        for (int al = 0; al < pA; ++al) {
          double *y = Yuse + (int64_t)al * njl;
          for (int t = 0; t < njl; ++t) y[t] = 0.0;
          for (int be = 0; be < pB; ++be) {
            const double w = Vb[(int64_t)al * pB + be];
            const double *c = cB + (int64_t)be * njl;
            for (int t = 0; t < njl; ++t) y[t] += w * c[t];
          }
        }
        if (a_is_I) yi_ready = 1;
      }
      /* T[alpha][j][k] = sum_l Y[alpha][j][l] D_KL[k][l] */
      for (int al = 0; al < pA; ++al)
        for (int jj = 0; jj < nj; ++jj) {
          const double *y = Yuse + ((int64_t)al * nj + jj) * nl;
          for (int kk = 0; kk < nk; ++kk) {
            const double *dk = Db + (int64_t)kk * nl;
            double s = 0.0;
            for (int ll = 0; ll < nl; ++ll) s += y[ll] * dk[ll];
            T[((int64_t)al * nj + jj) * nk + kk] = s;
          }
        }
      /* Ht[i][j] = sum_{alpha,k} cA[alpha][i][k] T[alpha][j][k];  Sigma -= Ht */
      load_coef(o, eK, ni, nk, pA, cA);
      for (int ii = 0; ii < ni; ++ii)
        for (int jj = 0; jj < nj; ++jj) {
          double s = 0.0;
          for (int al = 0; al < pA; ++al) {
            const double *ca = cA + ((int64_t)al * ni + ii) * nk;
            const double *tt = T + ((int64_t)al * nj + jj) * nk;
            for (int kk = 0; kk < nk; ++kk) s += ca[kk] * tt[kk];
          }
          kahan_add(&acc[ii * nj + jj], &cmp[ii * nj + jj], -s);
        }
    }
  }
  for (int t = 0; t < ni * nj; ++t) out[t] = acc[t] + cmp[t];
  free(KI);
  free(LJ);
  return nterms;
}

/* Work buffer size (doubles) per thread for sigma_block. */
static int64_t work_doubles(void) { return 2 * MAXAO * MAXAO + 5 * (int64_t)SLAB; }

/*
 * Compute the requested Sigma blocks.  req_keys: nreq x 5 (i, j, n1, n2, n3)
 * with arbitrary (i, j, n); out_offs: nreq + 1 offsets into out (filled here).
 * nthreads <= 0 uses the OpenMP default.  terms_out (nullable, nreq entries)
 * receives the number of surviving terms summed into each block.  Returns 0,
 * or -1 on a size the oracle's work buffers do not cover (nao > 64 or
 * nabf > 128).
 */
int orc_blocks(orc *o, double theta, int64_t nreq, const int32_t *req_keys, double *out,
               int64_t *out_offs, int nthreads, int64_t *terms_out) {
  for (int32_t a = 0; a < o->natoms; ++a)
    if (o->nao[a] > MAXAO || o->nabf[a] > MAXABF) return -1;
  out_offs[0] = 0;
  for (int64_t r = 0; r < nreq; ++r)
    out_offs[r + 1] = out_offs[r] + (int64_t)o->nao[req_keys[5 * r]] * o->nao[req_keys[5 * r + 1]];
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double *work = (double *)malloc(sizeof(double) * (size_t)work_doubles());
#pragma omp for schedule(dynamic, 1)
    for (int64_t r = 0; r < nreq; ++r) {
      const int32_t *k = req_keys + 5 * r;
      int32_t n[3] = {k[2], k[3], k[4]};
      const int64_t nt = sigma_block(o, theta, k[0], k[1], n, out + out_offs[r], work);
      if (terms_out) terms_out[r] = nt;
    }
    free(work);
  }
  return 0;
}

/*
 * E_X = 1/2 sum over Sigma keys that are also D keys of sum_ij D[i][j] Sigma[i][j]
 * (Algorithm 5, "Calculate E^X"), summed in key order, compensated.
 */
double orc_ex(orc *o, int64_t nkeys, const int32_t *keys, const double *sig, const int64_t *offs) {
  double s = 0.0, c = 0.0;
  for (int64_t e = 0; e < nkeys; ++e) {
    const int32_t *k = keys + 5 * e;
    int32_t n[3] = {k[2], k[3], k[4]};
    int64_t d = bset_find(&o->D, k[0], k[1], n);
    if (d < 0) continue;
    const double *Db = o->D.data + o->D.offs[d];
    int64_t len = offs[e + 1] - offs[e];
    for (int64_t t = 0; t < len; ++t) kahan_add(&s, &c, Db[t] * sig[offs[e] + t]);
  }
  return 0.5 * (s + c);
}

/* Replace the block upper limits used by the screen (e.g. to keep the set of
 * surviving terms of an unperturbed input fixed in a finite difference). */
void orc_set_maxabs(orc *o, char which, const double *vals) {
  bset_t *b = which == 'C' ? &o->C : which == 'V' ? &o->V : &o->D;
  memcpy(b->maxabs, vals, sizeof(double) * (size_t)b->n);
}

/* Block upper limits as computed here (exposed for tests). */
void orc_maxabs(orc *o, char which, double *out) {
  const bset_t *b = which == 'C' ? &o->C : which == 'V' ? &o->V : &o->D;
  memcpy(out, b->maxabs, sizeof(double) * (size_t)b->n);
}
