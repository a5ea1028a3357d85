/*
 * Order-exact weighted pivoted Cholesky with pivot fusion -- oracle.
 *
 * TEST INFRASTRUCTURE: plain C, FP64, built with -ffp-contract=off so that
 * every product and sum below is rounded exactly as written (fma() is an
 * explicit, correctly rounded fused multiply-add).  Loops over grid points may
 * be split across OpenMP threads; each point's sums keep the stated order, so
 * the results do not depend on the thread count.
 *
 * Follows Alg. 1 (scalar branch) and the gradient branch of Sec. II.D:
 *   t1(g,h) = sum_p phi_p(g) phi_p(h)                         (p ascending)
 *   t2(g,h) = sum_c sum_p dphi_{c,p}(g) dphi_{c,p}(h)         (c outer, p inner)
 *   scalar   S(g,h) = (w_g w_h) (t1 t1),   d_g = S(g,g)
 *   gradient S(g,h) = (w_g w_h) (t1 t2),   d_g = S(g,g)
 *   step: g* = argmax_g d_g (lowest index on ties);
 *         L_mu(g) = (S(g,g*) - sum_{l<mu} L_l(g) L_l(g*)) / sqrt(d_g*);
 *         d_g = max(d_g - L_mu(g)^2, 0);  then d_g* = 0.
 * Every sum is accumulated with acc = fma(a, b, acc) in the stated order and
 * every subtraction of a product with acc = fma(-a, b, acc).
 *
 * Readings (the paper is silent on these):
 *   - a channel stops when d_g* <= 64 eps max_g d_g(initial) (a zero pivot
 *     would divide by zero; the paper has no tolerance criterion);
 *   - fusion to exactly n_mu points: alternate one scalar and one gradient
 *     step (scalar first), append each pivot not yet in the union, stop when
 *     the union holds n_mu points; if one channel stops the other continues;
 *     if both stop the union is short (rank exhausted).
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  const double* phi;   /* [n_orb][n_g] */
  const double* dphi;  /* [3][n_orb][n_g] */
  const double* w;     /* [n_g] */
  long n_g;
  int n_orb;
} pv_in;

/* column t1(., h) into out[g].  The loops over g may run on several threads
 * (OpenMP, static partition): each point's sum keeps its order, p ascending. */
static void col_t1(const pv_in* in, long h, double* out) {
  long n_g = in->n_g;
#pragma omp parallel
  {
#pragma omp for schedule(static)
    for (long g = 0; g < n_g; ++g) out[g] = 0.0;
    for (int p = 0; p < in->n_orb; ++p) {
      const double* row = in->phi + (long)p * n_g;
      double b = row[h];
#pragma omp for schedule(static)
      for (long g = 0; g < n_g; ++g) out[g] = fma(row[g], b, out[g]);
    }
  }
}

static void col_t2(const pv_in* in, long h, double* out) {
  long n_g = in->n_g;
#pragma omp parallel
  {
#pragma omp for schedule(static)
    for (long g = 0; g < n_g; ++g) out[g] = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < in->n_orb; ++p) {
        const double* row = in->dphi + ((long)c * in->n_orb + p) * n_g;
        double b = row[h];
#pragma omp for schedule(static)
        for (long g = 0; g < n_g; ++g) out[g] = fma(row[g], b, out[g]);
      }
  }
}

/* diagonal: t(g,g) computed in the same order as a column */
static void diag_init(const pv_in* in, int grad, double* d) {
  long n_g = in->n_g;
  double* t1 = (double*)calloc(n_g, sizeof(double));
  double* t2 = (double*)calloc(n_g, sizeof(double));
  for (int p = 0; p < in->n_orb; ++p) {
    const double* row = in->phi + (long)p * n_g;
    for (long g = 0; g < n_g; ++g) t1[g] = fma(row[g], row[g], t1[g]);
  }
  if (grad)
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < in->n_orb; ++p) {
        const double* row = in->dphi + ((long)c * in->n_orb + p) * n_g;
        for (long g = 0; g < n_g; ++g) t2[g] = fma(row[g], row[g], t2[g]);
      }
  for (long g = 0; g < n_g; ++g) {
    double ww = in->w[g] * in->w[g];
    d[g] = grad ? ww * (t1[g] * t2[g]) : ww * (t1[g] * t1[g]);
  }
  free(t1);
  free(t2);
}

static long argmax_first(const double* d, long n) {
  long best = 0;
  double bv = d[0];
  for (long g = 1; g < n; ++g)
    if (d[g] > bv) { bv = d[g]; best = g; }
  return best;
}

typedef struct {
  int grad;
  double* d;     /* [n_g] residual diagonal */
  double* L;     /* [cap][n_g] Cholesky columns */
  int* piv;      /* [cap] */
  int k;         /* columns so far */
  int cap;
  int done;
  double tol;
} pv_chan;

/* One pivoted-Cholesky step of a channel; returns the pivot or -1 if the
 * channel has stopped. */
static long chan_step(const pv_in* in, pv_chan* ch, double* t1, double* t2) {
  long n_g = in->n_g;
  if (ch->done) return -1;
  if (ch->k >= ch->cap) { ch->done = 1; return -1; }
  long gs = argmax_first(ch->d, n_g);
  double dgs = ch->d[gs];
  if (!(dgs > ch->tol)) { ch->done = 1; return -1; }
  col_t1(in, gs, t1);
  if (ch->grad) col_t2(in, gs, t2);
  double* Lk = ch->L + (long)ch->k * n_g;
  double wg = in->w[gs];
  double sq = sqrt(dgs);
#pragma omp parallel
  {
#pragma omp for schedule(static)
    for (long g = 0; g < n_g; ++g) {
      double s = ch->grad ? (in->w[g] * wg) * (t1[g] * t2[g])
                          : (in->w[g] * wg) * (t1[g] * t1[g]);
      Lk[g] = s;
    }
    for (int l = 0; l < ch->k; ++l) {
      const double* Ll = ch->L + (long)l * n_g;
      double b = Ll[gs];
#pragma omp for schedule(static)
      for (long g = 0; g < n_g; ++g) Lk[g] = fma(-Ll[g], b, Lk[g]);
    }
#pragma omp for schedule(static)
    for (long g = 0; g < n_g; ++g) {
      double v = Lk[g] / sq;
      Lk[g] = v;
      double nd = fma(-v, v, ch->d[g]);
      ch->d[g] = nd > 0.0 ? nd : 0.0;
    }
  }
  ch->d[gs] = 0.0;
  ch->piv[ch->k] = (int)gs;
  ch->k += 1;
  return gs;
}

/*
 * Fused selection.  Outputs:
 *   piv_union[n_mu]   union in append order; *n_union its size
 *   piv_s[cap], *n_s  scalar-channel pivots;  piv_v, *n_v gradient channel
 *   d_s, d_v [n_g]    final residual diagonals (may be NULL)
 *   L_s, L_v [cap][n_g] Cholesky columns (may be NULL: then allocated here)
 * mode 0 = fused alternating to n_mu; mode 1 = scalar channel only to n_mu;
 * mode 2 = gradient channel only to n_mu.
 * Returns 0 when n_mu points were found, 1 when the rank was exhausted.
 */
int oracle_pivots(const double* phi, const double* dphi, const double* w,
                  long n_g, int n_orb, int n_mu, int cap, int mode,
                  int* piv_union, int* n_union, int* piv_s, int* n_s,
                  int* piv_v, int* n_v, double* d_s, double* d_v,
                  double* L_s, double* L_v) {
  pv_in in = {phi, dphi, w, n_g, n_orb};
  pv_chan ch[2];
  double* own[4] = {NULL, NULL, NULL, NULL};
  for (int c = 0; c < 2; ++c) {
    ch[c].grad = c;
    ch[c].d = (c == 0 ? d_s : d_v);
    if (!ch[c].d) ch[c].d = own[c] = (double*)malloc(n_g * sizeof(double));
    ch[c].L = (c == 0 ? L_s : L_v);
    if (!ch[c].L) ch[c].L = own[2 + c] = (double*)malloc((size_t)cap * n_g * sizeof(double));
    ch[c].piv = (c == 0 ? piv_s : piv_v);
    ch[c].k = 0;
    ch[c].cap = cap;
    ch[c].done = 0;
    diag_init(&in, c, ch[c].d);
    double mx = 0.0;
    for (long g = 0; g < n_g; ++g) if (ch[c].d[g] > mx) mx = ch[c].d[g];
    ch[c].tol = 64.0 * DBL_EPSILON * mx;
  }
  if (mode == 1) ch[1].done = 1;
  if (mode == 2) ch[0].done = 1;
  char* in_union = (char*)calloc(n_g, 1);
  double* t1 = (double*)malloc(n_g * sizeof(double));
  double* t2 = (double*)malloc(n_g * sizeof(double));
  int nu = 0;
  int turn = 0;
  while (nu < n_mu) {
    if (ch[0].done && ch[1].done) break;
    int c = turn;
    if (ch[c].done) c = 1 - c;
    long gs = chan_step(&in, &ch[c], t1, t2);
    if (gs >= 0 && !in_union[gs]) {
      in_union[gs] = 1;
      piv_union[nu++] = (int)gs;
    }
    turn = 1 - turn;
  }
  *n_union = nu;
  *n_s = ch[0].k;
  *n_v = ch[1].k;
  free(in_union);
  free(t1);
  free(t2);
  for (int i = 0; i < 4; ++i) free(own[i]);
  return nu < n_mu ? 1 : 0;
}

/*
 * The paper's own fusion (Sec. II.D, pivot-fusion paragraph): each channel runs
 * on its own to a fixed rank -- n_phi scalar steps, then n_grad gradient steps,
 * fewer where a channel stops -- and the interpolation set is their union, the
 * scalar list in its order followed by each gradient pivot not already in it.
 * The union size is an outcome (at most n_phi + n_grad).
 * Outputs as oracle_pivots; piv_union needs n_phi + n_grad entries.
 * Returns 0 when both channels reached their ranks, 1 when either stopped
 * early (rank exhausted).
 */
int oracle_pivots_ranks(const double* phi, const double* dphi, const double* w,
                        long n_g, int n_orb, int n_phi, int n_grad,
                        int* piv_union, int* n_union, int* piv_s, int* n_s,
                        int* piv_v, int* n_v) {
  pv_in in = {phi, dphi, w, n_g, n_orb};
  const int rank[2] = {n_phi, n_grad};
  int* piv[2] = {piv_s, piv_v};
  int* nk[2] = {n_s, n_v};
  char* in_union = (char*)calloc(n_g, 1);
  double* t1 = (double*)malloc(n_g * sizeof(double));
  double* t2 = (double*)malloc(n_g * sizeof(double));
  int nu = 0;
  int short_rank = 0;
  for (int c = 0; c < 2; ++c) {
    pv_chan ch;
    ch.grad = c;
    ch.d = (double*)malloc(n_g * sizeof(double));
    ch.L = (double*)malloc((size_t)(rank[c] > 0 ? rank[c] : 1) * n_g * sizeof(double));
    ch.piv = piv[c];
    ch.k = 0;
    ch.cap = rank[c];
    ch.done = rank[c] <= 0;
    diag_init(&in, c, ch.d);
    double mx = 0.0;
    for (long g = 0; g < n_g; ++g) if (ch.d[g] > mx) mx = ch.d[g];
    ch.tol = 64.0 * DBL_EPSILON * mx;
    for (;;) {
      long gs = chan_step(&in, &ch, t1, t2);
      if (gs < 0) break;
      if (!in_union[gs]) {
        in_union[gs] = 1;
        piv_union[nu++] = (int)gs;
      }
    }
    if (ch.k < rank[c]) short_rank = 1;
    *nk[c] = ch.k;
    free(ch.d);
    free(ch.L);
  }
  *n_union = nu;
  free(in_union);
  free(t1);
  free(t2);
  return short_rank;
}
