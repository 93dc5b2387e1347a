/*
 * FP64 CPU oracle for the RBSOG + RBL force evaluation of Born-Mayer-Huggins
 * (BMH) systems (arXiv 2512.24970, "Random Batch Sum-of-Gaussians Method for
 * Molecular Dynamics of Born-Mayer-Huggins Systems").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Every function follows the paper's statement of the method, in its order
 * and notation, without blocking or fusion:
 *   - BMH pair potential                      Eq. (BMH), Sec. 2.1
 *   - SOG (u-series) split, C^1 cutoff         Eqs. (1r),(far),(short), Sec. 2.1
 *   - short-range force                        Eq. (Fshort)
 *   - Fourier transform of the far part        Eq. (Fouriertransform)
 *   - structure factor, long-range force       Eq. (Long), Sec. 2.1
 *   - RBL core/shell split, shell estimator,
 *     momentum correction                      Sec. 2.2
 *   - importance density P(k), RBSOG estimator Eqs. (Pk),(long-rangeforce), Sec. 2.2
 * Where the paper is silent the conventions below are readings, all listed in
 * the design notes of the repository (fixed-point coordinates, the FP32 list
 * predicate, the canonical shell order, Floyd sampling without replacement,
 * the Philox counter layout, the exact mixture sampler for P(k)).
 *
 * Units: metal (Angstrom, eV, ps, amu, e).  Coulomb terms carry k_e.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction:
 * the list predicate is defined in IEEE binary32 with explicit fmaf only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KE 14.3996454784 /* eV * Angstrom / e^2 */

/* status codes (mirrors nothing: the oracle has its own) */
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOROOT (-2)
#define ORC_ECAP (-3)

/* ------------------------------------------------------------------------ */
/* System description passed from Python (ctypes mirror in oracle/__init__). */
typedef struct {
  int64_t n;              /* atoms */
  int32_t n_species;
  int32_t M;              /* Gaussians m = 0..M */
  const double *pos;      /* [n][3] FP64 positions */
  const int32_t *species; /* [n] */
  const double *charge;   /* [n_species] */
  const double *bmh;      /* [n_species][n_species][5] = A, sigma, rho, C, D */
  const double *w;        /* [M+1] SOG weights, w[0] already C^1-modified */
  double L[3];            /* box */
  double b, s;            /* SOG base and bandwidth */
  double r_core, r_shell; /* RBL radii; r_shell is also the SOG cutoff r_c */
  int32_t P_R, P_F;       /* batch sizes */
  uint64_t seed;
  int64_t step;
  double skin;            /* Verlet skin of the kept lists (orc_*_skin only) */
  const double *r_core_pair; /* [n_species][n_species] core radius of each species pair, or NULL */
} orc_sys;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Two 32x32->64 bit
 * multiplies per round with constants 0xD2511F53 and 0xCD9E8D57; the key is
 * bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 after every round.  */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout of every random draw of the method:
 *   ctr = (index, step_lo, step_hi, stream << 24 | block), key = (seed_lo, seed_hi)
 * streams: 0 = RBL shell batch (index = atom), 1 = k-batch (index = p),
 *          2 = Langevin noise (index = atom).                               */
static void draw(uint64_t seed, int64_t step, uint32_t index, uint32_t stream,
                 uint32_t block, uint32_t out[4]) {
  uint32_t ctr[4] = {index, (uint32_t)(uint64_t)step,
                     (uint32_t)((uint64_t)step >> 32), (stream << 24) | block};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, out);
}

void orc_philox(int64_t n, const uint32_t *ctr, const uint32_t *key,
                uint32_t *out) {
  for (int64_t i = 0; i < n; i++) philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

void orc_draw(uint64_t seed, int64_t step, int64_t n, const uint32_t *index,
              uint32_t stream, uint32_t block, uint32_t *out) {
  for (int64_t i = 0; i < n; i++) draw(seed, step, index[i], stream, block, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* SOG split, Sec. 2.1.
 * Nominal weights of Eq. (far): w_m = sqrt(2) ln b / (sqrt(pi) b^m s).
 * The narrowest weight w_0 is replaced so that N(r_c) = 0 (value continuity,
 * reading of the garbled w_0 formula: m = 0 in its exponent, F(r_c) summed
 * over m = 1..M), and s is chosen so that N'(r_c) = 0 (force continuity,
 * reading of the C^1 condition as -1/r_c^2 - F'(r_c) = 0).              */
static double sog_a(double b, double s, int m) { /* a_m = (b^m s)^2 */
  double bm = pow(b, (double)m) * s;
  return bm * bm;
}

static void sog_weights_for(double b, int M, double rc, double s, double *w) {
  const double lnb = log(b);
  for (int m = 0; m <= M; m++)
    w[m] = sqrt(2.0) * lnb / (sqrt(M_PI) * pow(b, (double)m) * s);
  double f1 = 0.0;
  for (int m = 1; m <= M; m++) f1 += w[m] * exp(-rc * rc / (2.0 * sog_a(b, s, m)));
  w[0] = exp(rc * rc / (2.0 * s * s)) * (1.0 / rc - f1);
}

static double sog_dN_at_rc(double b, int M, double rc, double s, double *w) {
  sog_weights_for(b, M, rc, s, w);
  double fp = 0.0; /* -F'(rc) = sum w_m rc/a_m exp(-rc^2/(2 a_m)) */
  for (int m = 0; m <= M; m++) {
    double a = sog_a(b, s, m);
    fp += w[m] * rc / a * exp(-rc * rc / (2.0 * a));
  }
  return -1.0 / (rc * rc) + fp;
}

/* Solve (s, w_0) for given (b, M, r_c): bisection for every sign change of
 * N'(r_c) on s in [r_c/6, r_c/2]; the root whose w_0 is closest to nominal. */
int orc_sog_solve(double b, int32_t M, double rc, double *s_out, double *w_out) {
  if (!(b > 1.0) || M < 1 || !(rc > 0.0)) return ORC_EINVAL;
  double *w = (double *)malloc(sizeof(double) * (size_t)(M + 1));
  const int NS = 4000;
  double lo = rc / 6.0, hi = rc / 2.0;
  double best_s = -1.0, best_dev = 1e300;
  double prev_s = lo, prev_v = sog_dN_at_rc(b, M, rc, lo, w);
  for (int k = 1; k <= NS; k++) {
    double sk = lo + (hi - lo) * (double)k / (double)NS;
    double vk = sog_dN_at_rc(b, M, rc, sk, w);
    if ((prev_v < 0.0 && vk > 0.0) || (prev_v > 0.0 && vk < 0.0) || vk == 0.0) {
      double a = prev_s, c = sk, va = prev_v;
      for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (a + c);
        if (mid <= a || mid >= c) break;
        double vm = sog_dN_at_rc(b, M, rc, mid, w);
        if ((va < 0.0) == (vm < 0.0) && vm != 0.0) { a = mid; va = vm; }
        else c = mid;
      }
      double sr = 0.5 * (a + c);
      sog_weights_for(b, M, rc, sr, w);
      double w0nom = sqrt(2.0) * log(b) / (sqrt(M_PI) * sr);
      double dev = fabs(w[0] / w0nom - 1.0);
      if (dev < best_dev) { best_dev = dev; best_s = sr; }
    }
    prev_s = sk; prev_v = vk;
  }
  if (best_s < 0.0) { free(w); return ORC_ENOROOT; }
  sog_weights_for(b, M, rc, best_s, w);
  *s_out = best_s;
  memcpy(w_out, w, sizeof(double) * (size_t)(M + 1));
  free(w);
  return ORC_OK;
}

/* F(r) of Eq. (far) and its radial derivative, using the given weights. */
void orc_sog_eval(int32_t M, double b, double s, const double *w, int64_t n,
                  const double *r, double *F, double *dF) {
  for (int64_t i = 0; i < n; i++) {
    double f = 0.0, df = 0.0;
    for (int m = 0; m <= M; m++) {
      double a = sog_a(b, s, m);
      double e = exp(-r[i] * r[i] / (2.0 * a));
      f += w[m] * e;
      df -= w[m] * r[i] / a * e;
    }
    F[i] = f;
    dF[i] = df;
  }
}

/* Eq. (Fouriertransform): Fhat(k) = (2 pi)^{3/2} sum_m w_m b^{3m} s^3 e^{-b^{2m} s^2 k^2 / 2} */
static double sog_fhat(const orc_sys *S, double k2) {
  double f = 0.0;
  for (int m = 0; m <= S->M; m++) {
    double a = sog_a(S->b, S->s, m);
    f += S->w[m] * pow(S->b, 3.0 * m) * S->s * S->s * S->s * exp(-a * k2 / 2.0);
  }
  return pow(2.0 * M_PI, 1.5) * f;
}

/* dFhat/d(k^2) = -(2 pi)^{3/2} sum_m w_m b^{3m} s^3 (b^{2m} s^2 / 2) e^{-b^{2m} s^2 k^2 / 2},
 * the derivative the far-field virial needs (strain changes k, not k . r). */
static double sog_fhat_dk2(const orc_sys *S, double k2) {
  double f = 0.0;
  for (int m = 0; m <= S->M; m++) {
    double a = sog_a(S->b, S->s, m);
    f -= S->w[m] * pow(S->b, 3.0 * m) * S->s * S->s * S->s * (a / 2.0) * exp(-a * k2 / 2.0);
  }
  return pow(2.0 * M_PI, 1.5) * f;
}

void orc_sog_fhat_dk2(const orc_sys *S, int64_t n, const double *k2, double *out) {
  for (int64_t i = 0; i < n; i++) out[i] = sog_fhat_dk2(S, k2[i]);
}

void orc_sog_fhat(const orc_sys *S, int64_t n, const double *k2, double *out) {
  for (int64_t i = 0; i < n; i++) out[i] = sog_fhat(S, k2[i]);
}

/* ------------------------------------------------------------------------ */
/* Pair terms of Eq. (Fshort) (force f_ij = phi * r_ij, r_ij = r_i - r_j) and
 * the matching pair energy q_i q_j N(r) + B_BMH(r) of Eqs. (short),(short2). */
static void pair_terms(const orc_sys *S, int si, int sj, double r2, double *phi,
                       double *e) {
  const double r = sqrt(r2);
  const double qq = ORC_KE * S->charge[si] * S->charge[sj];
  const double *p = S->bmh + 5 * (si * S->n_species + sj);
  const double A = p[0], sig = p[1], rho = p[2], C = p[3], D = p[4];
  double g = 0.0, f = 0.0;
  for (int m = 0; m <= S->M; m++) {
    double a = sog_a(S->b, S->s, m);
    double ex = exp(-r2 / (2.0 * a));
    g += S->w[m] / a * ex;
    f += S->w[m] * ex;
  }
  const double rep = A * exp((sig - r) / rho);
  const double r6 = r2 * r2 * r2, r8 = r6 * r2;
  *phi = qq * (1.0 / (r2 * r) - g) + rep / (rho * r) - 6.0 * C / r8 -
         8.0 * D / (r8 * r2);
  *e = qq * (1.0 / r - f) + rep - C / r6 - D / r8;
}

void orc_pair_terms(const orc_sys *S, int32_t si, int32_t sj, int64_t n,
                    const double *r2, double *phi, double *e) {
  for (int64_t i = 0; i < n; i++) pair_terms(S, si, sj, r2[i], phi + i, e + i);
}

/* ------------------------------------------------------------------------ */
/* Fixed-point fractional coordinates: u = floor(frac(x / L) * 2^32), with
 * x / L evaluated as x * (1 / L).  All phases and list decisions use u.     */
static uint32_t fixed_point(double x, double invL) {
  double t = x * invL;
  double y = floor(t * 4294967296.0);
  return (uint32_t)(uint64_t)(int64_t)y;
}

void orc_fixed_point(const orc_sys *S, uint32_t *u) {
  double inv[3] = {1.0 / S->L[0], 1.0 / S->L[1], 1.0 / S->L[2]};
  for (int64_t i = 0; i < S->n; i++)
    for (int a = 0; a < 3; a++) u[3 * i + a] = fixed_point(S->pos[3 * i + a], inv[a]);
}

/* Cell grid of the canonical order: n_c = max(1, floor(L / (r_out/2 * (1 + 2^-12)))),
 * cell = (u * n_c) >> 32, linear index x fastest.  r_out is the outer list
 * radius: r_shell for the per-step lists, r_shell + skin for kept lists.  */
static void cell_grid_r(const orc_sys *S, double r_out, int32_t nc[3]) {
  for (int a = 0; a < 3; a++) {
    double w = 0.5 * r_out * (1.0 + 1.0 / 4096.0);
    int32_t c = (int32_t)floor(S->L[a] / w);
    nc[a] = c < 1 ? 1 : c;
  }
}
void orc_cell_grid(const orc_sys *S, int32_t nc[3]) { cell_grid_r(S, S->r_shell, nc); }
void orc_cell_grid_skin(const orc_sys *S, int32_t nc[3]) { cell_grid_r(S, S->r_shell + S->skin, nc); }

static int64_t cell_linear(const uint32_t *u, const int32_t nc[3]) {
  int64_t c[3];
  for (int a = 0; a < 3; a++) c[a] = (int64_t)(((uint64_t)u[a] * (uint64_t)nc[a]) >> 32);
  return c[0] + (int64_t)nc[0] * (c[1] + (int64_t)nc[1] * c[2]);
}

/* List predicate in IEEE binary32: 23-bit coordinates v = u >> 9, the
 * minimum-image difference of v sign-extended from 23 bits, scaled by
 * h = fl32(L / 2^23); r^2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx)).           */
static float pred_r2(const uint32_t *ui, const uint32_t *uj, const float h[3]) {
  float d[3];
  for (int a = 0; a < 3; a++) {
    uint32_t dv = ((uj[a] >> 9) - (ui[a] >> 9)) << 9;
    int32_t sv = ((int32_t)dv) >> 9;
    d[a] = (float)sv * h[a];
  }
  float r2 = d[0] * d[0];
  r2 = fmaf(d[1], d[1], r2);
  r2 = fmaf(d[2], d[2], r2);
  return r2;
}

typedef struct { int64_t key; uint32_t ux; int32_t j; } cand_t;
static int cand_cmp(const void *a, const void *b) {
  const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->ux != y->ux) return x->ux < y->ux ? -1 : 1;
  return x->j < y->j ? -1 : (x->j > y->j);
}

typedef struct {
  float h[3], rc2, rs2;
  int32_t nc[3];
  uint32_t *u;     /* [n][3] */
  int64_t *cell;   /* [n] */
} orc_geo;

/* Geometry of the positions pos with outer list radius r_out. */
static void geo_init_at(const orc_sys *S, const double *pos, double r_out, orc_geo *G) {
  for (int a = 0; a < 3; a++) G->h[a] = (float)(S->L[a] * 0x1p-23);
  G->rc2 = (float)(S->r_core * S->r_core);
  G->rs2 = (float)(r_out * r_out);
  cell_grid_r(S, r_out, G->nc);
  G->u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)S->n);
  G->cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)S->n);
  double inv[3] = {1.0 / S->L[0], 1.0 / S->L[1], 1.0 / S->L[2]};
  for (int64_t i = 0; i < S->n; i++)
    for (int a = 0; a < 3; a++) G->u[3 * i + a] = fixed_point(pos[3 * i + a], inv[a]);
  for (int64_t i = 0; i < S->n; i++) G->cell[i] = cell_linear(G->u + 3 * i, G->nc);
}
static void geo_init(const orc_sys *S, orc_geo *G) { geo_init_at(S, S->pos, S->r_shell, G); }
static void geo_free(orc_geo *G) { free(G->u); free(G->cell); }

/* Core set {j != i : r^2 < fl32(r_core^2)} and shell set
 * {j != i : fl32(r_core^2) <= r^2 < fl32(r_shell^2)} of atom i, both in
 * canonical order: ascending (cell linear index of j, fixed-point x
 * coordinate u_x of j, j).  Brute force.  With species-dependent core radii
 * (the adaptive cutoff of Sec. 1, a reading: a symmetric table of r_core per
 * species pair, none above r_core) the core threshold of the pair (i, j) is
 * fl32(r_core(s_i, s_j)^2).                                                */
static int atom_lists(const orc_sys *S, const orc_geo *G, int64_t i, cand_t *core,
                      int32_t *ncore, int cap_core, cand_t *shell, int32_t *nshell,
                      int cap_shell) {
  int nc = 0, ns = 0, over = 0;
  const uint32_t *ui = G->u + 3 * i;
  for (int64_t j = 0; j < S->n; j++) {
    if (j == i) continue;
    float r2 = pred_r2(ui, G->u + 3 * j, G->h);
    float rc2 = G->rc2;
    if (S->r_core_pair) {
      const double rc = S->r_core_pair[S->species[i] * S->n_species + S->species[j]];
      rc2 = (float)(rc * rc);
    }
    if (r2 < rc2) {
      if (nc < cap_core) { core[nc].key = G->cell[j]; core[nc].ux = G->u[3 * j]; core[nc].j = (int32_t)j; }
      else over = 1;
      nc++;
    } else if (r2 < G->rs2) {
      if (ns < cap_shell) { shell[ns].key = G->cell[j]; shell[ns].ux = G->u[3 * j]; shell[ns].j = (int32_t)j; }
      else over = 1;
      ns++;
    }
  }
  if (!over) {
    qsort(core, (size_t)nc, sizeof(cand_t), cand_cmp);
    qsort(shell, (size_t)ns, sizeof(cand_t), cand_cmp);
  }
  *ncore = nc;
  *nshell = ns;
  return over ? ORC_ECAP : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* RBL shell batch, Sec. 2.2: P_R of the N_shell shell neighbours, without
 * replacement (the variance factor (N_shell - P_R)/P_R of the proof), by
 * Floyd's algorithm; draw r uses 64 bits of Philox block r/2 of stream 0;
 * uniform integer on [0, J] = high 64 bits of U * (J + 1).
 * Returns the chosen canonical positions t, ascending.                    */
static int floyd_batch(uint64_t seed, int64_t step, uint32_t atom, int32_t nshell,
                       int32_t PR, int32_t *t_out) {
  if (nshell <= PR) {
    for (int32_t t = 0; t < nshell; t++) t_out[t] = t;
    return nshell;
  }
  int cnt = 0;
  uint32_t wv[4];
  for (int32_t r = 0; r < PR; r++) {
    if ((r & 1) == 0) draw(seed, step, atom, 0u, (uint32_t)(r >> 1), wv);
    uint64_t U = ((uint64_t)wv[2 * (r & 1) + 1] << 32) | (uint64_t)wv[2 * (r & 1)];
    uint32_t J = (uint32_t)(nshell - PR + r);
    uint32_t t = (uint32_t)(((unsigned __int128)U * (unsigned __int128)((uint64_t)J + 1u)) >> 64);
    int present = 0;
    for (int k = 0; k < cnt; k++)
      if (t_out[k] == (int32_t)t) { present = 1; break; }
    t_out[cnt++] = present ? (int32_t)J : (int32_t)t;
  }
  for (int a = 1; a < cnt; a++) { /* insertion sort, ascending */
    int32_t v = t_out[a];
    int b = a - 1;
    while (b >= 0 && t_out[b] > v) { t_out[b + 1] = t_out[b]; b--; }
    t_out[b + 1] = v;
  }
  return cnt;
}

int32_t orc_floyd(uint64_t seed, int64_t step, uint32_t atom, int32_t nshell,
                  int32_t PR, int32_t *t_out) {
  return floyd_batch(seed, step, atom, nshell, PR, t_out);
}

/* Lists and shell batch of selected atoms (parity hook).  core/shell rows
 * hold atom indices in canonical order; batch rows hold the sampled atom
 * indices in canonical order and weight = N_shell / P_R (1 if all taken). */
int orc_lists(const orc_sys *S, const int64_t *sel, int64_t nsel, int32_t cap_core,
              int32_t cap_shell, int32_t *core, int32_t *ncore, int32_t *shell,
              int32_t *nshell, int32_t *batch, int32_t *nbatch, double *weight) {
  orc_geo G;
  geo_init(S, &G);
  int status = ORC_OK;
#pragma omp parallel
  {
    cand_t *cc = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap_core);
    cand_t *ss = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap_shell);
    int32_t *tt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->P_R > 0 ? S->P_R : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nsel; q++) {
      int64_t i = sel[q];
      int32_t nc, ns;
      if (atom_lists(S, &G, i, cc, &nc, cap_core, ss, &ns, cap_shell) != ORC_OK) {
#pragma omp atomic write
        status = ORC_ECAP;
        ncore[q] = nc; nshell[q] = ns;
        continue;
      }
      ncore[q] = nc;
      nshell[q] = ns;
      for (int k = 0; k < nc; k++) core[q * cap_core + k] = cc[k].j;
      for (int k = 0; k < ns; k++) shell[q * cap_shell + k] = ss[k].j;
      if (batch) {
        int nb = floyd_batch(S->seed, S->step, (uint32_t)i, ns, S->P_R, tt);
        nbatch[q] = nb;
        for (int k = 0; k < nb; k++) batch[q * S->P_R + k] = ss[tt[k]].j;
        weight[q] = ns <= S->P_R ? 1.0 : (double)ns / (double)S->P_R;
      }
    }
    free(cc); free(ss); free(tt);
  }
  geo_free(&G);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Near field of Sec. 2.2 for selected atoms: F_core + (N_shell/P_R) sum_B f_ij
 * (uncorrected), with pair displacements r_ij from the 32-bit fixed-point
 * minimum image, r_ij = (int32)(u_i - u_j) * (L / 2^32).  With all_shell != 0
 * the whole shell is taken with weight 1 (the deterministic r_shell-cutoff
 * force).  Per-atom energy: 1/2 of the same weighted pair sum; per-atom
 * virial W[q][6] (xx, yy, zz, xy, xz, yz): 1/2 of the same weighted sum of
 * r_ij (x) f_ij (the pair virial, whose sum over atoms is -dU_N/d strain).  */
#define ORC_CAP 4096
static void add_virial(double *w, const double *d, double phi) {
  w[0] += d[0] * phi * d[0]; w[1] += d[1] * phi * d[1]; w[2] += d[2] * phi * d[2];
  w[3] += d[0] * phi * d[1]; w[4] += d[0] * phi * d[2]; w[5] += d[1] * phi * d[2];
}
int orc_near(const orc_sys *S, const int64_t *sel, int64_t nsel, int32_t all_shell,
             double *F, double *E, double *W) {
  orc_geo G;
  geo_init(S, &G);
  int status = ORC_OK;
  const double sc[3] = {S->L[0] * 0x1p-32, S->L[1] * 0x1p-32, S->L[2] * 0x1p-32};
#pragma omp parallel
  {
    cand_t *cc = (cand_t *)malloc(sizeof(cand_t) * ORC_CAP);
    cand_t *ss = (cand_t *)malloc(sizeof(cand_t) * ORC_CAP);
    int32_t *tt = (int32_t *)malloc(sizeof(int32_t) * ORC_CAP);
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nsel; q++) {
      int64_t i = sel[q];
      int32_t nc, ns;
      if (atom_lists(S, &G, i, cc, &nc, ORC_CAP, ss, &ns, ORC_CAP) != ORC_OK) {
#pragma omp atomic write
        status = ORC_ECAP;
        continue;
      }
      const uint32_t *ui = G.u + 3 * i;
      const int si = S->species[i];
      double fc[3] = {0, 0, 0}, fs[3] = {0, 0, 0}, ec = 0.0, es = 0.0;
      double wc[6] = {0, 0, 0, 0, 0, 0}, ws[6] = {0, 0, 0, 0, 0, 0};
      for (int k = 0; k < nc; k++) {
        const int64_t j = cc[k].j;
        const uint32_t *uj = G.u + 3 * j;
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)(int32_t)(ui[a] - uj[a]) * sc[a];
        double phi, e;
        pair_terms(S, si, S->species[j], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], &phi, &e);
        for (int a = 0; a < 3; a++) fc[a] += phi * d[a];
        ec += e;
        add_virial(wc, d, phi);
      }
      int nb;
      double wgt;
      if (all_shell || ns <= S->P_R) {
        nb = ns;
        for (int k = 0; k < ns; k++) tt[k] = k;
        wgt = 1.0;
      } else {
        nb = floyd_batch(S->seed, S->step, (uint32_t)i, ns, S->P_R, tt);
        wgt = (double)ns / (double)S->P_R;
      }
      for (int k = 0; k < nb; k++) {
        const int64_t j = ss[tt[k]].j;
        const uint32_t *uj = G.u + 3 * j;
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)(int32_t)(ui[a] - uj[a]) * sc[a];
        double phi, e;
        pair_terms(S, si, S->species[j], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], &phi, &e);
        for (int a = 0; a < 3; a++) fs[a] += phi * d[a];
        es += e;
        add_virial(ws, d, phi);
      }
      for (int a = 0; a < 3; a++) F[3 * q + a] = fc[a] + wgt * fs[a];
      if (E) E[q] = 0.5 * (ec + wgt * es);
      if (W)
        for (int c = 0; c < 6; c++) W[6 * q + c] = 0.5 * (wc[c] + wgt * ws[c]);
    }
    free(cc); free(ss); free(tt);
  }
  geo_free(&G);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Kept (Verlet-skin) random batch lists: the RBL of Sec. 2.2 with neighbour
 * lists that live for several steps, as in the paper's LAMMPS implementation
 * (Sec. 3), whose per-step work is the core list plus P_R shell members
 * (Sec. 2.4).  The lists are built at the positions pos_b with the outer
 * radius r_list = r_shell + skin (cell grid of r_list / 2, canonical order of
 * pos_b):
 *   A_i = {j != i : pred_b < fl32(r_core^2)}
 *   B_i = {j != i : fl32(r_core^2) <= pred_b < fl32(r_list^2)}.
 * At the current positions every pair term carries the indicator
 * 1[pred < fl32(r_shell^2)]:
 *   F_i = sum_{j in A_i} f_ij 1[.] + (|B_i| / P_R) sum_{t in T_i} f_{i B_i[t]} 1[.]
 * with T_i Floyd's P_R of |B_i| (all of B_i with weight 1 when |B_i| <= P_R).
 * While no atom has moved by skin / 2 since pos_b, A_i and B_i hold every j
 * with r_ij < r_shell, so the mean over T_i is the r_shell-cutoff force.    */
int orc_lists_skin(const orc_sys *S, const double *pos_b, const int64_t *sel, int64_t nsel,
                   int32_t cap_a, int32_t cap_b, int32_t *A, int32_t *na, int32_t *B, int32_t *nb,
                   int32_t *batch, int32_t *nbatch, double *weight) {
  orc_geo G;
  geo_init_at(S, pos_b, S->r_shell + S->skin, &G);
  int status = ORC_OK;
#pragma omp parallel
  {
    cand_t *aa = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap_a);
    cand_t *bb = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap_b);
    int32_t *tt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->P_R > 0 ? S->P_R : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nsel; q++) {
      int64_t i = sel[q];
      int32_t n_a, n_b;
      if (atom_lists(S, &G, i, aa, &n_a, cap_a, bb, &n_b, cap_b) != ORC_OK) {
#pragma omp atomic write
        status = ORC_ECAP;
        na[q] = n_a; nb[q] = n_b;
        continue;
      }
      na[q] = n_a;
      nb[q] = n_b;
      for (int k = 0; k < n_a; k++) A[q * cap_a + k] = aa[k].j;
      for (int k = 0; k < n_b; k++) B[q * cap_b + k] = bb[k].j;
      if (batch) {
        int m = floyd_batch(S->seed, S->step, (uint32_t)i, n_b, S->P_R, tt);
        nbatch[q] = m;
        for (int k = 0; k < m; k++) batch[q * S->P_R + k] = bb[tt[k]].j;
        weight[q] = n_b <= S->P_R ? 1.0 : (double)n_b / (double)S->P_R;
      }
    }
    free(aa); free(bb); free(tt);
  }
  geo_free(&G);
  return status;
}

/* Uncorrected near field of selected atoms with the kept lists of pos_b (see
 * above); all_shell != 0 takes the whole of B_i with weight 1.  Per-atom
 * energy: 1/2 of the same weighted pair sum.                               */
int orc_near_skin(const orc_sys *S, const double *pos_b, const int64_t *sel, int64_t nsel,
                  int32_t all_shell, double *F, double *E, double *W) {
  orc_geo Gb, Gn;
  geo_init_at(S, pos_b, S->r_shell + S->skin, &Gb);
  geo_init_at(S, S->pos, S->r_shell, &Gn);
  int status = ORC_OK;
  const double sc[3] = {S->L[0] * 0x1p-32, S->L[1] * 0x1p-32, S->L[2] * 0x1p-32};
#pragma omp parallel
  {
    cand_t *aa = (cand_t *)malloc(sizeof(cand_t) * ORC_CAP);
    cand_t *bb = (cand_t *)malloc(sizeof(cand_t) * ORC_CAP);
    int32_t *tt = (int32_t *)malloc(sizeof(int32_t) * ORC_CAP);
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nsel; q++) {
      int64_t i = sel[q];
      int32_t n_a, n_b;
      if (atom_lists(S, &Gb, i, aa, &n_a, ORC_CAP, bb, &n_b, ORC_CAP) != ORC_OK) {
#pragma omp atomic write
        status = ORC_ECAP;
        continue;
      }
      const uint32_t *ui = Gn.u + 3 * i;
      const int si = S->species[i];
      double fa[3] = {0, 0, 0}, fb[3] = {0, 0, 0}, ea = 0.0, eb = 0.0;
      double wa[6] = {0, 0, 0, 0, 0, 0}, wb[6] = {0, 0, 0, 0, 0, 0};
      for (int k = 0; k < n_a; k++) {
        const int64_t j = aa[k].j;
        const uint32_t *uj = Gn.u + 3 * j;
        if (!(pred_r2(ui, uj, Gn.h) < Gn.rs2)) continue;
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)(int32_t)(ui[a] - uj[a]) * sc[a];
        double phi, e;
        pair_terms(S, si, S->species[j], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], &phi, &e);
        for (int a = 0; a < 3; a++) fa[a] += phi * d[a];
        ea += e;
        add_virial(wa, d, phi);
      }
      int m;
      double wgt;
      if (all_shell || n_b <= S->P_R) {
        m = n_b;
        for (int k = 0; k < n_b; k++) tt[k] = k;
        wgt = 1.0;
      } else {
        m = floyd_batch(S->seed, S->step, (uint32_t)i, n_b, S->P_R, tt);
        wgt = (double)n_b / (double)S->P_R;
      }
      for (int k = 0; k < m; k++) {
        const int64_t j = bb[tt[k]].j;
        const uint32_t *uj = Gn.u + 3 * j;
        if (!(pred_r2(ui, uj, Gn.h) < Gn.rs2)) continue;
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = (double)(int32_t)(ui[a] - uj[a]) * sc[a];
        double phi, e;
        pair_terms(S, si, S->species[j], d[0] * d[0] + d[1] * d[1] + d[2] * d[2], &phi, &e);
        for (int a = 0; a < 3; a++) fb[a] += phi * d[a];
        eb += e;
        add_virial(wb, d, phi);
      }
      for (int a = 0; a < 3; a++) F[3 * q + a] = fa[a] + wgt * fb[a];
      if (E) E[q] = 0.5 * (ea + wgt * eb);
      if (W)
        for (int c = 0; c < 6; c++) W[6 * q + c] = 0.5 * (wa[c] + wgt * wb[c]);
    }
    free(aa); free(bb); free(tt);
  }
  geo_free(&Gb);
  geo_free(&Gn);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Importance density of Eq. (Pk): P(k) = k^2 Fhat(k) / S over k != 0.
 * Exact i.i.d. sampler of that P (reading of the paper's MH sampler):
 * k^2 Fhat(k) = sum_g sum_d c_g k_d^2 e^{-a_g k_d^2/2} prod_{d' != d} e^{-a_g k_{d'}^2/2}
 * with a_g = (b^g s)^2, c_g = (2 pi)^{3/2} w_g b^{3g} s^3, so P is a mixture
 * over (g, d) with weight Z_{g,d} = c_g T2_{g,d} prod_{d'!=d} T0_{g,d'} of
 * separable lattice Gaussians; T0 = sum_n e^{-a k_n^2/2}, T2 = sum_n k_n^2 e^{..},
 * k_n = 2 pi n / L_d.  S = sum Z.  Decisions compare 64-bit uniforms with
 * 64-bit fixed-point CDFs: index = #{i < len-1 : C[i] <= U}.            */
#define ORC_KCUT 60.0
typedef struct {
  int G;            /* M + 1 */
  int *nmax;        /* [G][3] */
  uint64_t **cdf0;  /* [G*3] plain 1-D CDFs, length 2*nmax+1 */
  uint64_t **cdf2;  /* [G*3] k^2-weighted 1-D CDFs */
  uint64_t *cmix;   /* [G*3] mixture CDF */
  double S;
} orc_sampler;

static uint64_t fixed_cdf(double cum, double total) {
  double x = floor(cum / total * 18446744073709551616.0);
  if (x >= 18446744073709551616.0) return UINT64_MAX;
  if (x <= 0.0) return 0;
  return (uint64_t)x;
}

static int cdf_pick(const uint64_t *C, int len, uint64_t U) {
  int idx = 0;
  for (int i = 0; i < len - 1; i++) idx += (C[i] <= U);
  return idx;
}

static void sampler_build(const orc_sys *S, orc_sampler *T) {
  const int G = S->M + 1;
  T->G = G;
  T->nmax = (int *)malloc(sizeof(int) * 3 * (size_t)G);
  T->cdf0 = (uint64_t **)malloc(sizeof(uint64_t *) * 3 * (size_t)G);
  T->cdf2 = (uint64_t **)malloc(sizeof(uint64_t *) * 3 * (size_t)G);
  T->cmix = (uint64_t *)malloc(sizeof(uint64_t) * 3 * (size_t)G);
  double *Z = (double *)malloc(sizeof(double) * 3 * (size_t)G);
  for (int g = 0; g < G; g++) {
    const double a = sog_a(S->b, S->s, g);
    const double cg = pow(2.0 * M_PI, 1.5) * S->w[g] * pow(S->b, 3.0 * g) * S->s * S->s * S->s;
    double T0[3], T2[3];
    for (int d = 0; d < 3; d++) {
      const double kap = 2.0 * M_PI / S->L[d];
      int nm = (int)ceil(sqrt(2.0 * ORC_KCUT / a) / kap);
      if (nm < 1) nm = 1;
      T->nmax[3 * g + d] = nm;
      const int len = 2 * nm + 1;
      double *e0 = (double *)malloc(sizeof(double) * (size_t)len);
      double *e2 = (double *)malloc(sizeof(double) * (size_t)len);
      double s0 = 0.0, s2 = 0.0;
      for (int q = 0; q < len; q++) {
        const double k = kap * (double)(q - nm);
        e0[q] = exp(-a * k * k / 2.0);
        e2[q] = k * k * e0[q];
        s0 += e0[q];
        s2 += e2[q];
      }
      T0[d] = s0;
      T2[d] = s2;
      uint64_t *c0 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
      uint64_t *c2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
      double r0 = 0.0, r2 = 0.0;
      for (int q = 0; q < len; q++) {
        r0 += e0[q];
        r2 += e2[q];
        c0[q] = fixed_cdf(r0, s0);
        c2[q] = s2 > 0.0 ? fixed_cdf(r2, s2) : UINT64_MAX;
      }
      T->cdf0[3 * g + d] = c0;
      T->cdf2[3 * g + d] = c2;
      free(e0); free(e2);
    }
    for (int d = 0; d < 3; d++) {
      double z = cg * T2[d];
      for (int e = 0; e < 3; e++) if (e != d) z *= T0[e];
      Z[3 * g + d] = z;
    }
  }
  double tot = 0.0;
  for (int q = 0; q < 3 * G; q++) tot += Z[q];
  double run = 0.0;
  for (int q = 0; q < 3 * G; q++) {
    run += Z[q];
    T->cmix[q] = fixed_cdf(run, tot);
  }
  T->S = tot;
  free(Z);
}

static void sampler_free(orc_sampler *T) {
  for (int q = 0; q < 3 * T->G; q++) { free(T->cdf0[q]); free(T->cdf2[q]); }
  free(T->cdf0); free(T->cdf2); free(T->cmix); free(T->nmax);
}

/* S = sum_{k != 0} k^2 Fhat(k) (closed form of the mixture). */
double orc_sampler_S(const orc_sys *S) {
  orc_sampler T;
  sampler_build(S, &T);
  double v = T.S;
  sampler_free(&T);
  return v;
}

/* Mixture weights Z[g][d] (for tests). */
void orc_sampler_Z(const orc_sys *S, double *Z) {
  const int G = S->M + 1;
  for (int g = 0; g < G; g++) {
    const double a = sog_a(S->b, S->s, g);
    const double cg = pow(2.0 * M_PI, 1.5) * S->w[g] * pow(S->b, 3.0 * g) * S->s * S->s * S->s;
    double T0[3], T2[3];
    for (int d = 0; d < 3; d++) {
      const double kap = 2.0 * M_PI / S->L[d];
      int nm = (int)ceil(sqrt(2.0 * ORC_KCUT / a) / kap);
      if (nm < 1) nm = 1;
      double s0 = 0.0, s2 = 0.0;
      for (int q = -nm; q <= nm; q++) {
        const double k = kap * q;
        const double e = exp(-a * k * k / 2.0);
        s0 += e;
        s2 += k * k * e;
      }
      T0[d] = s0; T2[d] = s2;
    }
    for (int d = 0; d < 3; d++) {
      double z = cg * T2[d];
      for (int e = 0; e < 3; e++) if (e != d) z *= T0[e];
      Z[3 * g + d] = z;
    }
  }
}

/* k-batch of Sec. 2.2: P_F i.i.d. draws m_p != 0 from P(k) (Philox stream 1,
 * index p, blocks 0 and 1: U0 picks (g,d), U1 picks m_d from the
 * k^2-weighted CDF, U2 and U3 the other two axes in ascending axis order),
 * and c_p = S / (P_F |k_p|^2).  Returns S.                               */
double orc_kbatch(const orc_sys *S, int32_t *m, double *c) {
  orc_sampler T;
  sampler_build(S, &T);
  for (int p = 0; p < S->P_F; p++) {
    uint32_t w0[4], w1[4];
    draw(S->seed, S->step, (uint32_t)p, 1u, 0u, w0);
    draw(S->seed, S->step, (uint32_t)p, 1u, 1u, w1);
    const uint64_t U0 = ((uint64_t)w0[1] << 32) | w0[0];
    const uint64_t U1 = ((uint64_t)w0[3] << 32) | w0[2];
    const uint64_t U2 = ((uint64_t)w1[1] << 32) | w1[0];
    const uint64_t U3 = ((uint64_t)w1[3] << 32) | w1[2];
    const int q = cdf_pick(T.cmix, 3 * T.G, U0);
    const int g = q / 3, d = q % 3;
    int mm[3];
    {
      const int nm = T.nmax[3 * g + d];
      mm[d] = cdf_pick(T.cdf2[3 * g + d], 2 * nm + 1, U1) - nm;
    }
    const uint64_t Uo[2] = {U2, U3};
    int o = 0;
    for (int e = 0; e < 3; e++) {
      if (e == d) continue;
      const int nm = T.nmax[3 * g + e];
      mm[e] = cdf_pick(T.cdf0[3 * g + e], 2 * nm + 1, Uo[o++]) - nm;
    }
    double k2 = 0.0;
    for (int e = 0; e < 3; e++) {
      const double k = 2.0 * M_PI * mm[e] / S->L[e];
      k2 += k * k;
      m[3 * p + e] = mm[e];
    }
    c[p] = T.S / ((double)S->P_F * k2);
  }
  double Sv = T.S;
  sampler_free(&T);
  return Sv;
}

/* ------------------------------------------------------------------------ */
/* Phase of atom j for lattice vector m: k . r_j = 2 pi (m . u_j mod 2^32) / 2^32,
 * taken as pi * x with x = (int32)(m . u_j) * 2^-31 in [-1, 1).          */
static double phase_pi(const int32_t *m, const uint32_t *u) {
  uint32_t th = (uint32_t)m[0] * u[0] + (uint32_t)m[1] * u[1] + (uint32_t)m[2] * u[2];
  return (double)(int32_t)th * 0x1p-31;
}

/* rho(k_p) = sum_j q_j e^{i k_p . r_j}  (Sec. 2.1), FP64. */
void orc_rho(const orc_sys *S, int32_t P, const int32_t *m, double *rho) {
  uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)S->n);
  orc_fixed_point(S, u);
#pragma omp parallel for schedule(static)
  for (int p = 0; p < P; p++) {
    double re = 0.0, im = 0.0;
    for (int64_t j = 0; j < S->n; j++) {
      const double x = phase_pi(m + 3 * p, u + 3 * j);
      const double q = S->charge[S->species[j]];
      re += q * cos(M_PI * x);
      im += q * sin(M_PI * x);
    }
    rho[2 * p] = re;
    rho[2 * p + 1] = im;
  }
  free(u);
}

/* Far-field force of selected atoms for a list of modes with weights c_p:
 * F_i = -(k_e q_i / V) sum_p c_p k_p Im(e^{-i k_p . r_i} rho_p).
 * With c_p = Fhat(k_p) over all k != 0 this is Eq. (Long); with the sampled
 * batch and c_p = S/(P_F |k_p|^2) it is Eq. (long-rangeforce).
 * Energy U_F* = k_e/(2V) sum_p c_p |rho_p|^2 (Eq. of U_F^* with the same weights). */
void orc_far(const orc_sys *S, int32_t P, const int32_t *m, const double *c,
             const double *rho, const int64_t *sel, int64_t nsel, double *F,
             double *Ufar) {
  const double V = S->L[0] * S->L[1] * S->L[2];
  double *kv = (double *)malloc(sizeof(double) * 3 * (size_t)P);
  for (int p = 0; p < P; p++)
    for (int e = 0; e < 3; e++) kv[3 * p + e] = 2.0 * M_PI * m[3 * p + e] / S->L[e];
  const double inv[3] = {1.0 / S->L[0], 1.0 / S->L[1], 1.0 / S->L[2]};
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < nsel; q++) {
    const int64_t i = sel[q];
    uint32_t ui[3];
    for (int a = 0; a < 3; a++) ui[a] = fixed_point(S->pos[3 * i + a], inv[a]);
    double f[3] = {0, 0, 0};
    for (int p = 0; p < P; p++) {
      const double x = phase_pi(m + 3 * p, ui);
      const double cs = cos(M_PI * x), sn = sin(M_PI * x);
      const double imv = cs * rho[2 * p + 1] - sn * rho[2 * p];
      for (int e = 0; e < 3; e++) f[e] += c[p] * kv[3 * p + e] * imv;
    }
    const double qi = S->charge[S->species[i]];
    for (int e = 0; e < 3; e++) F[3 * q + e] = -ORC_KE * qi / V * f[e];
  }
  if (Ufar) {
    double u = 0.0;
    for (int p = 0; p < P; p++) u += c[p] * (rho[2 * p] * rho[2 * p] + rho[2 * p + 1] * rho[2 * p + 1]);
    *Ufar = ORC_KE / (2.0 * V) * u;
  }
  free(kv);
}

/* Self term U_F^self = (k_e / 2) sum_i q_i^2 F(0), F(0) = sum_m w_m. */
double orc_self_energy(const orc_sys *S) {
  double f0 = 0.0;
  for (int m = 0; m <= S->M; m++) f0 += S->w[m];
  double q2 = 0.0;
  for (int64_t i = 0; i < S->n; i++) {
    double q = S->charge[S->species[i]];
    q2 += q * q;
  }
  return 0.5 * ORC_KE * q2 * f0;
}

int32_t orc_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (the CPU baseline times one core
 * and all cores). */
void orc_set_num_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
