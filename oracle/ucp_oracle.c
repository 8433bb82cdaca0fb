/*
 * ucp_oracle.c -- plain FP64 CPU oracle for critical-point probabilities of
 * 2D uncertain scalar fields (Athawale et al., "Uncertainty Visualization of
 * Critical Points of 2D Scalar Fields for Parametric and Nonparametric
 * Probabilistic Models", arXiv 2407.18015).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; it
 * is never part of the product path.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or constant with the CUDA sources.
 *
 * What it computes (all arithmetic in double precision unless stated):
 *
 *   P_min(v) = Pr[X_v < X_n for every in-grid axis neighbour n]
 *            = integral of pdf_v(x) * prod_n G_n(x) dx,  G_n = survival of X_n
 *   P_max(v) = integral of pdf_v(x) * prod_n F_n(x) dx,  F_n = CDF of X_n
 *
 * These are the paper's Eq. (localMinimumProb) (Sec. "Critical Point
 * Probability (Four-Pixel Neighborhood)") with the inner integrals carried
 * out (the integral of pdf_n from max(x1,a_n) to b_n is G_n(x1)), and the
 * local maximum as the same integral with every comparison reversed (the
 * paper obtains it by negating the variables, Sec. "Local Maximum
 * Probability"; the oracle writes the definition out directly so that the
 * negation identity can be tested against it).
 *
 * Method: the plain definition.  Every factor (the centre's density and each
 * neighbour's CDF or survival) is a piecewise polynomial.  All breakpoints of
 * all factors are merged and sorted; on each resulting piece every factor is
 * one polynomial, which is re-expanded in the piece-local variable
 * t = x - x_left, multiplied out in the monomial basis and integrated with its
 * exact antiderivative.  There is no quadrature, no blocking and no fusion.
 *
 * Saddle (Eq. saddleProb): with the neighbours e, n, w, s as X_2..X_5,
 *   t1 = Pr[X_1 < X_e, X_1 > X_n, X_1 < X_w, X_1 > X_s] = int pdf_1 G_e F_n G_w F_s
 *   t2 = Pr[X_1 > X_e, X_1 < X_n, X_1 > X_w, X_1 < X_s] = int pdf_1 F_e G_n F_w G_s
 *   P_saddle = t1 + t2.  A vertex without all four neighbours has no
 *   alternating neighbourhood: 0, except on a 1 x W or H x 1 grid, where the
 *   two-neighbour form (Eq. 1D-saddleProb) is used with X_2 the next
 *   neighbour (e, or s on a column) and X_3 the previous one (w, or n).
 *
 * Independent Gaussians (the parametric model the paper compares with):
 * orc_gauss, the same integrals over the real line by adaptive quadrature.
 *
 * Larger neighbourhoods and 3D grids (the extension named in Sec.
 * "Conclusion"): orc_prob_stencil evaluates the same P_min / P_max with the
 * neighbour set of a 6- or 8-neighbour 2D stencil or of the 6 axis
 * neighbours of a 3D grid (offsets listed at that function).
 *
 * Distribution models (Sec. "Parametric Noise Models",
 * Sec. "Nonparametric Noise Models"):
 *   uniform      params (a, b):     pdf 1/(b-a) on [a, b]
 *   Epanechnikov params (m, w):     pdf 3/(4w) (1 - ((x-m)/w)^2) on [m-w, m+w]
 *                                   (the paper's 3/(2(b-a)) with b-a = 2w)
 *   histogram    params (lo, hi, w_0..w_{B-1}): B equal bins on [lo, hi],
 *                pdf = sum_j w_j K_h(x - c_j), the mixture of non-overlapping
 *                uniform kernels of Eq. (localMinProbHistogram)'s text; the
 *                survival is used in the same mixture form, sum_j w_j S_j(x).
 *   multivariate Gaussian over (X_v, X_e, X_n, X_w, X_s): plain Monte Carlo.
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - neighbours are the in-grid axis neighbours e=(y,x+1), n=(y-1,x),
 *     w=(y,x-1), s=(y+1,x); a boundary vertex simply has fewer of them
 *     (boundary mode 0), or its probability is 0 (boundary mode 1);
 *   - a vertex whose support collapses (a == b, w == 0, lo == hi) is a point
 *     mass; comparisons are strict, so two equal point masses give 0;
 *   - Epanechnikov fit: m = sample mean, w = scale * sample std (N-1), the
 *     scale being sqrt(5) by default (variance of the kernel is w^2/5);
 *   - histogram fit: lo = min, hi = max, bin index computed in IEEE binary32
 *     as floor((x - lo) * s) with s = B / (hi - lo), clamped to [0, B-1]
 *     (this file must be compiled with -ffp-contract=off), mass = count / N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_UNIFORM 0
#define ORC_EPAN 1
#define ORC_HIST 2
#define ORC_MVN 3
#define ORC_GAUSS 5

#define ST_DEGENERATE 1
#define ST_NONFINITE 2
#define ST_BAD_PARAMS 4
#define ST_CHOL_JITTER 8
#define ST_CHOL_FAIL 16

#define MAXB 64
#define MAXE (MAXB + 1)
#define MAXC 4   /* a factor is a polynomial of degree <= 3 on each interval */
#define MAXK 8   /* neighbours per vertex, largest stencil                */
#define MAXPROD 32  /* Epanechnikov with 8 neighbours: degree 2 + 3*8 = 26 */

/* ------------------------------------------------------------------------ */
/* threads                                                                  */

static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* polynomials in the monomial basis                                        */

/* out(t) = p(d + t); p has n coefficients. */
static void poly_shift(const double *p, int n, double d, double *out) {
  double q[MAXC + 1];
  int i, j, nq = 1;
  q[0] = p[n - 1];
  for (i = n - 2; i >= 0; --i) {
    /* q <- q * (d + t) + p[i] */
    q[nq] = 0.0;
    for (j = nq; j >= 1; --j) q[j] = q[j] * d + q[j - 1];
    q[0] = q[0] * d + p[i];
    ++nq;
  }
  for (i = 0; i < n; ++i) out[i] = q[i];
}

static int poly_mul(const double *a, int na, const double *b, int nb, double *out) {
  double r[MAXPROD];
  int i, j;
  for (i = 0; i < na + nb - 1; ++i) r[i] = 0.0;
  for (i = 0; i < na; ++i)
    for (j = 0; j < nb; ++j) r[i + j] += a[i] * b[j];
  for (i = 0; i < na + nb - 1; ++i) out[i] = r[i];
  return na + nb - 1;
}

/* integral_0^L p(t) dt */
static double poly_int(const double *p, int n, double L) {
  double s = 0.0, Lp = L;
  int i;
  for (i = 0; i < n; ++i) {
    s += p[i] * Lp / (double)(i + 1);
    Lp *= L;
  }
  return s;
}

static double poly_eval(const double *p, int n, double t) {
  double s = 0.0;
  int i;
  for (i = n - 1; i >= 0; --i) s = s * t + p[i];
  return s;
}

/* ------------------------------------------------------------------------ */
/* piecewise polynomials                                                    */

typedef struct {
  int m;                   /* bounded intervals [e[j], e[j+1]], j < m      */
  double e[MAXE];
  double c[MAXB][MAXC];    /* coefficients in t = x - e[j]                 */
  int n[MAXB];             /* number of coefficients per interval          */
  double left, right;      /* constant value for x < e[0] and x > e[m]     */
} pw_t;

/* the polynomial of f on a piece [s, t] whose midpoint is mid, in the local
 * variable tau = x - s */
static int pw_poly_on(const pw_t *f, double s, double mid, double *out) {
  int j;
  if (mid < f->e[0]) {
    out[0] = f->left;
    return 1;
  }
  if (f->m == 0 || mid > f->e[f->m]) {
    out[0] = f->right;
    return 1;
  }
  for (j = 0; j < f->m - 1; ++j)
    if (mid < f->e[j + 1]) break;
  poly_shift(f->c[j], f->n[j], s - f->e[j], out);
  return f->n[j];
}

/* value of a continuous piecewise polynomial at x (right limit at a step) */
static double pw_eval(const pw_t *f, double x) {
  int j;
  if (f->m == 0) return x < f->e[0] ? f->left : f->right;
  if (x < f->e[0]) return f->left;
  if (x > f->e[f->m]) return f->right;
  for (j = 0; j < f->m - 1; ++j)
    if (x < f->e[j + 1]) break;
  return poly_eval(f->c[j], f->n[j], x - f->e[j]);
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* integral over [lo, hi] of the product of nf piecewise polynomials */
static double integrate_product(const pw_t *const *f, int nf, double lo, double hi) {
  double pts[2 + (1 + MAXK) * MAXE + 8];
  int np = 0, i, j, k;
  double total = 0.0;
  if (!(hi > lo)) return 0.0;
  pts[np++] = lo;
  pts[np++] = hi;
  for (i = 0; i < nf; ++i) {
    int ne = f[i]->m + 1;
    for (j = 0; j < ne; ++j) {
      double e = f[i]->e[j];
      if (e > lo && e < hi) pts[np++] = e;
    }
  }
  qsort(pts, (size_t)np, sizeof(double), cmp_double);
  for (k = 0; k + 1 < np; ++k) {
    double s = pts[k], t = pts[k + 1];
    double prod[MAXPROD], q[MAXC];
    int nprod = 1, nq;
    if (!(t > s)) continue;
    prod[0] = 1.0;
    for (i = 0; i < nf; ++i) {
      nq = pw_poly_on(f[i], s, 0.5 * (s + t), q);
      nprod = poly_mul(prod, nprod, q, nq, prod);
    }
    total += poly_int(prod, nprod, t - s);
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* per-vertex distributions                                                 */

typedef struct {
  int model, B, point, status;
  double lo, hi, total;   /* support; total mass (1 except mixture form)   */
  double p0, p1, h;       /* (a,b) / (m,w) / histogram bin width           */
  double w[MAXB];
  pw_t pdf, F, G;         /* density, CDF, survival (G = total - F)        */
} dist_t;

static void pw_step(pw_t *f, double c, double left, double right) {
  f->m = 0;
  f->e[0] = c;
  f->left = left;
  f->right = right;
}

static int all_finite(const double *p, int n) {
  int i;
  for (i = 0; i < n; ++i)
    if (!isfinite(p[i])) return 0;
  return 1;
}

/* Build the distribution of one vertex from its parameters.  Returns the
 * status bits: ST_NONFINITE / ST_BAD_PARAMS make the vertex unusable. */
static int dist_make(int model, const double *p, int B, dist_t *d) {
  int np = (model == ORC_HIST) ? 2 + B : 2, j;
  memset(d, 0, sizeof(*d));
  d->model = model;
  d->B = B;
  if (!all_finite(p, np)) return d->status = ST_NONFINITE;
  if (model == ORC_UNIFORM) {
    double a = p[0], b = p[1];
    if (a > b) return d->status = ST_BAD_PARAMS;
    d->p0 = a; d->p1 = b; d->lo = a; d->hi = b; d->total = 1.0;
    if (a == b) {
      d->point = 1;
    } else {
      double r = 1.0 / (b - a);
      d->pdf.m = 1; d->pdf.e[0] = a; d->pdf.e[1] = b;
      d->pdf.c[0][0] = r; d->pdf.n[0] = 1;
      d->F = d->pdf; d->F.c[0][0] = 0.0; d->F.c[0][1] = r; d->F.n[0] = 2;
      d->F.right = 1.0;
      d->G = d->pdf; d->G.c[0][0] = 1.0; d->G.c[0][1] = -r; d->G.n[0] = 2;
      d->G.left = 1.0;
    }
  } else if (model == ORC_EPAN) {
    double m = p[0], w = p[1];
    if (w < 0.0) return d->status = ST_BAD_PARAMS;
    d->p0 = m; d->p1 = w; d->lo = m - w; d->hi = m + w; d->total = 1.0;
    if (w == 0.0) {
      d->point = 1;
    } else {
      /* t = x - (m - w):  pdf = 3/(4w) (2t/w - t^2/w^2),
       *                   CDF = 3 t^2/(4 w^2) - t^3/(4 w^3)            */
      d->pdf.m = 1; d->pdf.e[0] = m - w; d->pdf.e[1] = m + w;
      d->pdf.c[0][0] = 0.0;
      d->pdf.c[0][1] = 3.0 / (2.0 * w * w);
      d->pdf.c[0][2] = -3.0 / (4.0 * w * w * w);
      d->pdf.n[0] = 3;
      d->F = d->pdf;
      d->F.c[0][0] = 0.0; d->F.c[0][1] = 0.0;
      d->F.c[0][2] = 3.0 / (4.0 * w * w);
      d->F.c[0][3] = -1.0 / (4.0 * w * w * w);
      d->F.n[0] = 4; d->F.right = 1.0;
      d->G = d->F;
      for (j = 0; j < 4; ++j) d->G.c[0][j] = -d->F.c[0][j];
      d->G.c[0][0] = 1.0; d->G.left = 1.0; d->G.right = 0.0;
    }
  } else if (model == ORC_HIST) {
    double lo = p[0], hi = p[1], T = 0.0, C = 0.0;
    if (B < 1 || B > MAXB) return d->status = ST_BAD_PARAMS;
    if (lo > hi) return d->status = ST_BAD_PARAMS;
    for (j = 0; j < B; ++j) {
      if (p[2 + j] < 0.0) return d->status = ST_BAD_PARAMS;
      d->w[j] = p[2 + j];
      T += p[2 + j];
    }
    d->lo = lo; d->hi = hi; d->total = T;
    if (lo == hi) {
      d->point = 1;
    } else {
      double h = (hi - lo) / (double)B;
      d->h = h;
      d->pdf.m = B; d->F.m = B; d->G.m = B;
      for (j = 0; j <= B; ++j) {
        double e = (j == B) ? hi : lo + (hi - lo) * (double)j / (double)B;
        d->pdf.e[j] = d->F.e[j] = d->G.e[j] = e;
      }
      for (j = 0; j < B; ++j) {
        double bw = d->pdf.e[j + 1] - d->pdf.e[j];
        d->pdf.c[j][0] = d->w[j] / bw; d->pdf.n[j] = 1;
        /* exact linear CDF of the mixture inside bin j */
        d->F.c[j][0] = C; d->F.c[j][1] = d->w[j] / bw; d->F.n[j] = 2;
        d->G.c[j][0] = T - C; d->G.c[j][1] = -d->w[j] / bw; d->G.n[j] = 2;
        C += d->w[j];
      }
      d->F.left = 0.0; d->F.right = T;
      d->G.left = T; d->G.right = 0.0;
    }
  } else {
    return d->status = ST_BAD_PARAMS;
  }
  if (d->point) {
    pw_step(&d->F, d->lo, 0.0, d->total);
    pw_step(&d->G, d->lo, d->total, 0.0);
    d->status = ST_DEGENERATE;
  }
  return d->status;
}

/* Pr[X > c] and Pr[X < c] (strict) */
static double prob_greater(const dist_t *d, double c) {
  if (d->point) return d->lo > c ? d->total : 0.0;
  return pw_eval(&d->G, c);
}
static double prob_less(const dist_t *d, double c) {
  if (d->point) return d->lo < c ? d->total : 0.0;
  return pw_eval(&d->F, c);
}

/* P_min (want_max = 0) or P_max (want_max = 1) of a centre with k neighbours */
static double prob_vertex(const dist_t *v, const dist_t *nb, int k, int want_max) {
  const pw_t *f[1 + MAXK];
  int n;
  if (v->point) {
    double p = v->total;
    for (n = 0; n < k; ++n)
      p *= want_max ? prob_less(&nb[n], v->lo) : prob_greater(&nb[n], v->lo);
    return p;
  }
  f[0] = &v->pdf;
  for (n = 0; n < k; ++n) f[1 + n] = want_max ? &nb[n].F : &nb[n].G;
  return integrate_product(f, 1 + k, v->lo, v->hi);
}

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */

static int nparams(int model, int B) {
  if (model == ORC_HIST) return 2 + B;
  if (model == ORC_MVN) return 20;
  return 2;
}

/* in-grid axis neighbours of (y, x) in the order e, n, w, s; returns count
 * and writes their linear indices; slot[] receives the direction 0..3 */
static int neighbours(int H, int W, int y, int x, int64_t *idx, int *slot) {
  static const int dy[4] = {0, -1, 0, 1};
  static const int dx[4] = {1, 0, -1, 0};
  int d, k = 0;
  for (d = 0; d < 4; ++d) {
    int yy = y + dy[d], xx = x + dx[d];
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    idx[k] = (int64_t)yy * W + xx;
    if (slot) slot[k] = d;
    ++k;
  }
  return k;
}

static void gather_params(const double *params, int64_t plane, int np, int64_t i, double *out) {
  int j;
  for (j = 0; j < np; ++j) out[j] = params[(int64_t)j * plane + i];
}

/* probability of one vertex; writes status */
static void vertex_min_max(const double *params, int H, int W, int model, int B,
                           int boundary, int y, int x, double *pmin, double *pmax,
                           uint8_t *status) {
  int64_t plane = (int64_t)H * W, nidx[4];
  int k = neighbours(H, W, y, x, nidx, NULL), n, st;
  double pv[2 + MAXB];
  dist_t v, nb[4];
  int np = nparams(model, B);
  gather_params(params, plane, np, (int64_t)y * W + x, pv);
  st = dist_make(model, pv, B, &v);
  for (n = 0; n < k; ++n) {
    double pn[2 + MAXB] = {0};
    gather_params(params, plane, np, nidx[n], pn);
    st |= dist_make(model, pn, B, &nb[n]) & (ST_NONFINITE | ST_BAD_PARAMS);
  }
  if (status) *status = (uint8_t)st;
  if (st & (ST_NONFINITE | ST_BAD_PARAMS)) {
    *pmin = *pmax = NAN;
    return;
  }
  if (boundary == 1 && k < 4) {
    *pmin = *pmax = 0.0;
    return;
  }
  *pmin = prob_vertex(&v, nb, k, 0);
  *pmax = prob_vertex(&v, nb, k, 1);
}

/* integral of pdf_v times, per neighbour, its survival (sign +1) or its CDF
 * (sign -1); a point-mass centre gives the product of the strict tail
 * probabilities */
static double prob_mixed(const dist_t *v, const dist_t *nb, const int *sign, int k) {
  const pw_t *f[5];
  int n;
  if (v->point) {
    double p = v->total;
    for (n = 0; n < k; ++n)
      p *= sign[n] > 0 ? prob_greater(&nb[n], v->lo) : prob_less(&nb[n], v->lo);
    return p;
  }
  f[0] = &v->pdf;
  for (n = 0; n < k; ++n) f[1 + n] = sign[n] > 0 ? &nb[n].G : &nb[n].F;
  return integrate_product(f, 1 + k, v->lo, v->hi);
}

static double vertex_saddle(const double *params, int H, int W, int model, int B, int y, int x,
                            uint8_t *status) {
  int64_t plane = (int64_t)H * W, nidx[4];
  int slot[4], k = neighbours(H, W, y, x, nidx, slot), n, st;
  int np = nparams(model, B), s1[4], s2[4];
  double pv[2 + MAXB];
  dist_t v, nb[4];
  gather_params(params, plane, np, (int64_t)y * W + x, pv);
  st = dist_make(model, pv, B, &v);
  for (n = 0; n < k; ++n) {
    double pn[2 + MAXB] = {0};
    gather_params(params, plane, np, nidx[n], pn);
    st |= dist_make(model, pn, B, &nb[n]) & (ST_NONFINITE | ST_BAD_PARAMS);
  }
  if (status) *status = (uint8_t)st;
  if (st & (ST_NONFINITE | ST_BAD_PARAMS)) return NAN;
  if (k == 4) {
    /* slots are e, n, w, s in this order: t1 wants G, F, G, F */
    for (n = 0; n < 4; ++n) {
      s1[n] = (slot[n] == 0 || slot[n] == 2) ? 1 : -1;
      s2[n] = -s1[n];
    }
  } else if (k == 2 && (H == 1 || W == 1)) {
    /* the line case: next = e or s (slots 0, 3), previous = w or n */
    for (n = 0; n < 2; ++n) {
      s1[n] = (slot[n] == 0 || slot[n] == 3) ? 1 : -1;
      s2[n] = -s1[n];
    }
  } else {
    return 0.0;
  }
  return prob_mixed(&v, nb, s1, k) + prob_mixed(&v, nb, s2, k);
}

/* ------------------------------------------------------------------------ */
/* exported: closed-form probability fields                                 */

/* Whole field.  params: [P][H][W] doubles (P = 2 or 2+B).  out_min/out_max
 * may be NULL.  status may be NULL. */
int orc_prob(const double *params, int H, int W, int model, int B, int boundary,
             double *out_min, double *out_max, uint8_t *status) {
  int y;
  if (model != ORC_UNIFORM && model != ORC_EPAN && model != ORC_HIST) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
  for (y = 0; y < H; ++y) {
    int x;
    for (x = 0; x < W; ++x) {
      double a, b;
      int64_t i = (int64_t)y * W + x;
      vertex_min_max(params, H, W, model, B, boundary, y, x, &a, &b,
                     status ? status + i : NULL);
      if (out_min) out_min[i] = a;
      if (out_max) out_max[i] = b;
    }
  }
  return 0;
}

/* Selected vertices only (linear indices idx[0..n-1]). */
int orc_prob_at(const double *params, int H, int W, int model, int B, int boundary,
                const int64_t *idx, int64_t n, double *out_min, double *out_max,
                uint8_t *status) {
  int64_t t;
  if (model != ORC_UNIFORM && model != ORC_EPAN && model != ORC_HIST) return -1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int y = (int)(idx[t] / W), x = (int)(idx[t] % W);
    double a, b;
    vertex_min_max(params, H, W, model, B, boundary, y, x, &a, &b,
                   status ? status + t : NULL);
    if (out_min) out_min[t] = a;
    if (out_max) out_max[t] = b;
  }
  return 0;
}

/* Saddle probability of every vertex (or of idx[0..n-1] when idx != NULL). */
int orc_saddle(const double *params, int H, int W, int model, int B, const int64_t *idx,
               int64_t n, double *out, uint8_t *status) {
  int64_t t, total = idx ? n : (int64_t)H * W;
  if (model != ORC_UNIFORM && model != ORC_EPAN && model != ORC_HIST) return -1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(orc_get_threads())
  for (t = 0; t < total; ++t) {
    int64_t i = idx ? idx[t] : t;
    out[t] = vertex_saddle(params, H, W, model, B, (int)(i / W), (int)(i % W),
                           status ? status + t : NULL);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* larger neighbourhoods and 3D grids                                        */
/*                                                                          */
/* The paper's stated extension (Sec. "Conclusion"): six- or eight-pixel     */
/* neighbourhoods of a triangulated 2D grid, and 3D grids.  The definition   */
/* is unchanged -- P_min = int pdf_v prod_{n in N(v)} G_n, P_max with F_n -- */
/* only the neighbour set N(v) comes from a stencil.  A D x H x W grid is    */
/* stored slice-major ([P][D][H][W]); offsets are (dz, dy, dx):              */
/*   stencil 0 (4):  e (0,0,1), n (0,-1,0), w (0,0,-1), s (0,1,0)           */
/*   stencil 1 (6):  the 4 axis ones, ne (0,-1,1), sw (0,1,-1): the grid    */
/*                   triangulated by cutting every cell along its           */
/*                   lower-left to upper-right diagonal                     */
/*   stencil 2 (8):  the 4 axis ones, ne, nw (0,-1,-1), sw, se (0,1,1)      */
/*   stencil 3 (3D6): the 4 axis ones, below (-1,0,0), above (1,0,0)        */
/* In-grid neighbours only (boundary mode 0), or 0 wherever the stencil is  */
/* incomplete (boundary mode 1).                                            */

static int stencil_offsets(int stencil, int off[MAXK][3]) {
  static const int o4[4][3] = {{0, 0, 1}, {0, -1, 0}, {0, 0, -1}, {0, 1, 0}};
  static const int o6[2][3] = {{0, -1, 1}, {0, 1, -1}};
  static const int o8[4][3] = {{0, -1, 1}, {0, -1, -1}, {0, 1, -1}, {0, 1, 1}};
  static const int oz[2][3] = {{-1, 0, 0}, {1, 0, 0}};
  int k = 0, i, j;
  if (stencil < 0 || stencil > 3) return -1;
  for (i = 0; i < 4; ++i, ++k)
    for (j = 0; j < 3; ++j) off[k][j] = o4[i][j];
  if (stencil == 1)
    for (i = 0; i < 2; ++i, ++k)
      for (j = 0; j < 3; ++j) off[k][j] = o6[i][j];
  if (stencil == 2)
    for (i = 0; i < 4; ++i, ++k)
      for (j = 0; j < 3; ++j) off[k][j] = o8[i][j];
  if (stencil == 3)
    for (i = 0; i < 2; ++i, ++k)
      for (j = 0; j < 3; ++j) off[k][j] = oz[i][j];
  return k;
}

static void vertex_min_max_stencil(const double *params, int D, int H, int W, int model, int B,
                                   int stencil, int boundary, int64_t i, double *pmin,
                                   double *pmax, uint8_t *status) {
  int64_t plane = (int64_t)D * H * W, nidx[MAXK];
  int off[MAXK][3], kfull = stencil_offsets(stencil, off), k = 0, n, st;
  int z = (int)(i / ((int64_t)H * W)), y = (int)((i / W) % H), x = (int)(i % W);
  int np = nparams(model, B);
  double pv[2 + MAXB] = {0};
  dist_t v, nb[MAXK];
  for (n = 0; n < kfull; ++n) {
    int zz = z + off[n][0], yy = y + off[n][1], xx = x + off[n][2];
    if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
    nidx[k++] = ((int64_t)zz * H + yy) * W + xx;
  }
  gather_params(params, plane, np, i, pv);
  st = dist_make(model, pv, B, &v);
  for (n = 0; n < k; ++n) {
    double pn[2 + MAXB] = {0};
    gather_params(params, plane, np, nidx[n], pn);
    st |= dist_make(model, pn, B, &nb[n]) & (ST_NONFINITE | ST_BAD_PARAMS);
  }
  if (status) *status = (uint8_t)st;
  if (st & (ST_NONFINITE | ST_BAD_PARAMS)) {
    *pmin = *pmax = NAN;
    return;
  }
  if (boundary == 1 && k < kfull) {
    *pmin = *pmax = 0.0;
    return;
  }
  *pmin = prob_vertex(&v, nb, k, 0);
  *pmax = prob_vertex(&v, nb, k, 1);
}

/* Minimum and maximum probability with a stencil on a D x H x W grid
 * (params [P][D][H][W] doubles), at every vertex (idx == NULL, outputs
 * [D][H][W]) or at the linear indices idx[0..n-1].  Closed-form models
 * only.  Returns -1 for an invalid model, stencil or shape. */
int orc_prob_stencil(const double *params, int D, int H, int W, int model, int B, int stencil,
                     int boundary, const int64_t *idx, int64_t n, double *out_min,
                     double *out_max, uint8_t *status) {
  int64_t t, total = (int64_t)D * H * W;
  if (model != ORC_UNIFORM && model != ORC_EPAN && model != ORC_HIST) return -1;
  if (stencil < 0 || stencil > 3 || D < 1 || H < 1 || W < 1) return -1;
  if (stencil != 3 && D != 1) return -1;
  if (!idx) n = total;
#pragma omp parallel for schedule(dynamic, 64) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int64_t i = idx ? idx[t] : t;
    double a, b;
    vertex_min_max_stencil(params, D, H, W, model, B, stencil, boundary, i, &a, &b,
                           status ? status + t : NULL);
    if (out_min) out_min[t] = a;
    if (out_max) out_max[t] = b;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* independent Gaussians                                                     */
/*                                                                          */
/* The parametric model the paper compares its closed forms with (Sec.       */
/* "Comparison of Parametric Vs. Nonparametric Models", there evaluated by   */
/* Monte Carlo): X_i ~ N(m_i, s_i^2) independent.  The definition is the     */
/* same integral, P_min = int pdf_v(x) prod_n Pr[X_n > x] dx (P_max with     */
/* Pr[X_n < x]), over the real line.  It is evaluated by adaptive Simpson    */
/* quadrature on [m_v - 12 s_v, m_v + 12 s_v] (the centre's mass outside is  */
/* below 1e-32), cut at m_v and at every neighbour's m_n and m_n +- 4 s_n,   */
/* with 16 starting panels per piece.  A point-mass centre (s_v = 0) gives   */
/* the product of the strict tail probabilities at m_v; a point-mass         */
/* neighbour is a step at its mean.  params: (m, s) planes.                  */

typedef struct {
  double m1, s1;
  int k;
  double m[4], s[4];
  int sign[4]; /* +1: Pr[X_n > x], -1: Pr[X_n < x] */
} gint_t;

static double g_tail(double m, double s, double x, int sign) {
  if (s == 0.0) return sign > 0 ? (m > x ? 1.0 : 0.0) : (m < x ? 1.0 : 0.0);
  /* Pr[X > x] = erfc((x - m) / (s sqrt 2)) / 2, Pr[X < x] = erfc((m - x) / (s sqrt 2)) / 2 */
  return 0.5 * erfc((sign > 0 ? (x - m) : (m - x)) / (s * sqrt(2.0)));
}

static double g_integrand(const gint_t *g, double x) {
  double z = (x - g->m1) / g->s1, f = exp(-0.5 * z * z) / (g->s1 * sqrt(2.0 * 3.14159265358979323846));
  int n;
  for (n = 0; n < g->k; ++n) f *= g_tail(g->m[n], g->s[n], x, g->sign[n]);
  return f;
}

static double g_simpson(const gint_t *g, double a, double b, double fa, double fm, double fb,
                        double whole, double tol, int depth) {
  double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = g_integrand(g, lm), frm = g_integrand(g, rm);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * tol) return left + right + delta / 15.0;
  return g_simpson(g, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         g_simpson(g, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

static double g_integral(const gint_t *g) {
  double lo = g->m1 - 12.0 * g->s1, hi = g->m1 + 12.0 * g->s1;
  double pts[3 + 3 * 4];
  int np = 0, n, i, j;
  double total = 0.0;
  pts[np++] = lo;
  pts[np++] = hi;
  pts[np++] = g->m1;
  for (n = 0; n < g->k; ++n) {
    double c[3] = {g->m[n] - 4.0 * g->s[n], g->m[n], g->m[n] + 4.0 * g->s[n]};
    for (i = 0; i < 3; ++i)
      if (c[i] > lo && c[i] < hi) pts[np++] = c[i];
  }
  qsort(pts, (size_t)np, sizeof(double), cmp_double);
  for (i = 0; i + 1 < np; ++i) {
    double a = pts[i], b = pts[i + 1];
    if (!(b > a)) continue;
    for (j = 0; j < 16; ++j) {
      double x0 = a + (b - a) * j / 16.0, x1 = a + (b - a) * (j + 1) / 16.0;
      double f0 = g_integrand(g, x0), f1 = g_integrand(g, x1), fm = g_integrand(g, 0.5 * (x0 + x1));
      double whole = (x1 - x0) / 6.0 * (f0 + 4.0 * fm + f1);
      total += g_simpson(g, x0, x1, f0, fm, f1, whole, 1e-15, 40);
    }
  }
  return total;
}

static int g_status(double m, double s) {
  if (!isfinite(m) || !isfinite(s)) return ST_NONFINITE;
  return s < 0.0 ? ST_BAD_PARAMS : (s == 0.0 ? ST_DEGENERATE : 0);
}

/* the integral with the given signs, or the product of tails at a
 * point-mass centre */
static double g_prob(gint_t *g) {
  int n;
  if (g->s1 == 0.0) {
    double p = 1.0;
    for (n = 0; n < g->k; ++n) p *= g_tail(g->m[n], g->s[n], g->m1, g->sign[n]);
    return p;
  }
  return g_integral(g);
}

/* Minimum, maximum and saddle probabilities of independent Gaussians at
 * every vertex (idx == NULL) or at idx[0..n-1]; any output may be NULL.
 * Neighbours and boundary modes as for the closed-form models. */
int orc_gauss(const double *params, int H, int W, int boundary, const int64_t *idx, int64_t n,
              double *out_min, double *out_max, double *out_saddle, uint8_t *status) {
  int64_t t, plane = (int64_t)H * W;
  if (H < 1 || W < 1) return -1;
  if (!idx) n = plane;
#pragma omp parallel for schedule(dynamic, 16) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int64_t i = idx ? idx[t] : t, nidx[4];
    int y = (int)(i / W), x = (int)(i % W), slot[4];
    int k = neighbours(H, W, y, x, nidx, slot), q, st;
    gint_t g;
    double pmin, pmax, psad = 0.0;
    g.m1 = params[i];
    g.s1 = params[plane + i];
    g.k = k;
    st = g_status(g.m1, g.s1);
    for (q = 0; q < k; ++q) {
      g.m[q] = params[nidx[q]];
      g.s[q] = params[plane + nidx[q]];
      st |= g_status(g.m[q], g.s[q]) & (ST_NONFINITE | ST_BAD_PARAMS);
    }
    if (status) status[t] = (uint8_t)st;
    if (st & (ST_NONFINITE | ST_BAD_PARAMS)) {
      if (out_min) out_min[t] = NAN;
      if (out_max) out_max[t] = NAN;
      if (out_saddle) out_saddle[t] = NAN;
      continue;
    }
    for (q = 0; q < k; ++q) g.sign[q] = 1;
    pmin = g_prob(&g);
    for (q = 0; q < k; ++q) g.sign[q] = -1;
    pmax = g_prob(&g);
    if (boundary == 1 && k < 4) pmin = pmax = 0.0;
    if (out_saddle) {
      /* Eq. saddleProb: e, w below / n, s above, and the reverse; the line
       * case with the next (e, or s) and previous (w, or n) neighbour */
      int ok = k == 4 || (k == 2 && (H == 1 || W == 1));
      if (ok) {
        double t1, t2;
        for (q = 0; q < k; ++q)
          g.sign[q] = k == 4 ? ((slot[q] == 0 || slot[q] == 2) ? 1 : -1)
                             : ((slot[q] == 0 || slot[q] == 3) ? 1 : -1);
        t1 = g_prob(&g);
        for (q = 0; q < k; ++q) g.sign[q] = -g.sign[q];
        t2 = g_prob(&g);
        psad = t1 + t2;
      }
      out_saddle[t] = psad;
    }
    if (out_min) out_min[t] = pmin;
    if (out_max) out_max[t] = pmax;
  }
  return 0;
}

/* The paper's second route for histograms, Eq. (localMinProbHistogram):
 * sum over every combination of one bin per variable of the product of the
 * bin masses times the uniform-kernel probability of that combination.
 * O(B^(k+1)) per vertex; meant for small B.  Point masses are not supported
 * (returns NaN there). */
int orc_prob_hist_h5_at(const double *params, int H, int W, int B, const int64_t *idx,
                        int64_t n, double *out_min, double *out_max) {
  int64_t t, plane = (int64_t)H * W;
  if (B < 1 || B > MAXB) return -1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int y = (int)(idx[t] / W), x = (int)(idx[t] % W);
    int64_t ids[5];
    int k = neighbours(H, W, y, x, ids + 1, NULL), nv = k + 1, i, bad = 0;
    double lo[5], hi[5], w[5][MAXB], smin = 0.0, smax = 0.0;
    int combo[5];
    ids[0] = idx[t];
    for (i = 0; i < nv; ++i) {
      int j;
      lo[i] = params[ids[i]];
      hi[i] = params[plane + ids[i]];
      if (!(hi[i] > lo[i])) bad = 1;
      for (j = 0; j < B; ++j) w[i][j] = params[(int64_t)(2 + j) * plane + ids[i]];
    }
    if (bad) {
      out_min[t] = out_max[t] = NAN;
      continue;
    }
    for (i = 0; i < nv; ++i) combo[i] = 0;
    for (;;) {
      double wt = 1.0, pa[2];
      dist_t v, nb[4];
      for (i = 0; i < nv; ++i) wt *= w[i][combo[i]];
      if (wt != 0.0) {
        for (i = 0; i < nv; ++i) {
          pa[0] = lo[i] + (hi[i] - lo[i]) * (double)combo[i] / (double)B;
          pa[1] = (combo[i] == B - 1) ? hi[i]
                                      : lo[i] + (hi[i] - lo[i]) * (double)(combo[i] + 1) / (double)B;
          dist_make(ORC_UNIFORM, pa, 1, i == 0 ? &v : &nb[i - 1]);
        }
        smin += wt * prob_vertex(&v, nb, k, 0);
        smax += wt * prob_vertex(&v, nb, k, 1);
      }
      for (i = 0; i < nv; ++i) {
        if (++combo[i] < B) break;
        combo[i] = 0;
      }
      if (i == nv) break;
    }
    out_min[t] = smin;
    out_max[t] = smax;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* exported: model fitting from an ensemble ens[N][H][W] (float32)           */

static int hist_bin_f32(float x, float lo, float scale, int B) {
  /* IEEE binary32, one rounding per operation, no contraction:
   * scale = B / (hi - lo) is formed once per vertex by the caller */
  float d = x - lo;
  float q = d * scale;
  int i = (int)floorf(q);
  if (i < 0) i = 0;
  if (i > B - 1) i = B - 1;
  return i;
}

/* params: [P][H][W] doubles; status may be NULL.
 * model 0: (a,b) = (min,max); 1: (m,w) = (mean, scale*std); 2: (lo,hi,masses);
 * 3: mean of (v,e,n,w,s) in planes 0..4 and their covariance (unbiased) in
 *    planes 5..19, packed lower triangle row by row: (0,0),(1,0),(1,1),(2,0)...
 *    Entries of absent neighbours are 0. */
int orc_fit(const float *ens, int N, int H, int W, int model, int B, double epan_scale,
            double *params, uint8_t *status) {
  int64_t plane = (int64_t)H * W;
  int y;
  if (N < 1 || H < 1 || W < 1) return -1;
  if (model == ORC_HIST && (B < 1 || B > MAXB)) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
  for (y = 0; y < H; ++y) {
    int x;
    for (x = 0; x < W; ++x) {
      int64_t i = (int64_t)y * W + x;
      int k, st = 0;
      float mn = ens[i], mx = ens[i];
      for (k = 0; k < N; ++k) {
        float v = ens[(int64_t)k * plane + i];
        if (!isfinite(v)) st |= ST_NONFINITE;
        if (v < mn) mn = v;
        if (v > mx) mx = v;
      }
      /* a vertex with a non-finite member has no distribution (its
       * parameters are NaN): not degenerate, whatever min and max are */
      if (model != ORC_MVN && mn == mx && !(st & ST_NONFINITE)) st |= ST_DEGENERATE;
      if (st & ST_NONFINITE) {
        /* parameters are written as NaN below */
      } else if (model == ORC_UNIFORM) {
        params[i] = mn;
        params[plane + i] = mx;
      } else if (model == ORC_EPAN || model == ORC_GAUSS) {
        /* Gaussian: m = mean, s = sample std (the scale is 1) */
        double s = 0.0, m, ss = 0.0;
        for (k = 0; k < N; ++k) s += ens[(int64_t)k * plane + i];
        m = s / N;
        for (k = 0; k < N; ++k) {
          double d = ens[(int64_t)k * plane + i] - m;
          ss += d * d;
        }
        if (mn == mx) {
          params[i] = mn;
          params[plane + i] = 0.0;
        } else {
          params[i] = m;
          params[plane + i] = (model == ORC_GAUSS ? 1.0 : epan_scale) * sqrt(ss / (N - 1));
        }
      } else if (model == ORC_HIST) {
        int cnt[MAXB], j;
        for (j = 0; j < B; ++j) cnt[j] = 0;
        if (mn == mx) {
          cnt[0] = N;
        } else {
          float scale = (float)B / (mx - mn);
          for (k = 0; k < N; ++k) cnt[hist_bin_f32(ens[(int64_t)k * plane + i], mn, scale, B)]++;
        }
        params[i] = mn;
        params[plane + i] = mx;
        for (j = 0; j < B; ++j) params[(int64_t)(2 + j) * plane + i] = (double)cnt[j] / (double)N;
      } else if (model == ORC_MVN) {
        int64_t ids[5];
        int slot[4], present[5] = {1, 0, 0, 0, 0}, kn, a, b, r;
        double mu[5] = {0, 0, 0, 0, 0};
        kn = neighbours(H, W, y, x, ids + 1, slot);
        ids[0] = i;
        /* map to fixed slots v,e,n,w,s */
        {
          int64_t full[5];
          full[0] = i;
          for (a = 1; a < 5; ++a) full[a] = -1;
          for (a = 0; a < kn; ++a) full[1 + slot[a]] = ids[1 + a];
          for (a = 0; a < 5; ++a) {
            ids[a] = full[a];
            present[a] = full[a] >= 0;
          }
        }
        for (a = 0; a < 5; ++a) {
          if (!present[a]) continue;
          for (k = 0; k < N; ++k) {
            float v = ens[(int64_t)k * plane + ids[a]];
            if (!isfinite(v)) st |= ST_NONFINITE;
            mu[a] += v;
          }
          mu[a] /= N;
        }
        for (a = 0; a < 5; ++a) params[(int64_t)a * plane + i] = present[a] ? mu[a] : 0.0;
        r = 5;
        for (a = 0; a < 5; ++a) {
          for (b = 0; b <= a; ++b) {
            double c = 0.0;
            if (present[a] && present[b] && N > 1) {
              for (k = 0; k < N; ++k)
                c += (ens[(int64_t)k * plane + ids[a]] - mu[a]) *
                     (ens[(int64_t)k * plane + ids[b]] - mu[b]);
              c /= (N - 1);
            }
            params[(int64_t)r * plane + i] = c;
            ++r;
          }
        }
      }
      if (st & ST_NONFINITE) {
        int j, np = nparams(model, B);
        for (j = 0; j < np; ++j) params[(int64_t)j * plane + i] = NAN;
      }
      if (status) status[i] = (uint8_t)st;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box with the   */
/* Weyl key schedule.                                                        */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  int r;
  for (r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0, p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* multivariate Gaussian Monte Carlo                                        */

static int cholesky(const double *A, int n, double *L) {
  int i, j, k;
  for (i = 0; i < n * n; ++i) L[i] = 0.0;
  for (j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return 0;
    L[j * n + j] = sqrt(s);
    for (i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  return 1;
}

/* Monte Carlo for selected vertices.  params: [20][H][W] doubles (see
 * orc_fit).  Sample s of vertex i uses two Philox4x32-10 blocks with
 * counter (s, i, field, j), j = 0, 1, and key (seed_lo, seed_hi); the eight
 * words give uniforms u = ((r >> 9) + 0.5) / 2^23 (exact in binary32 as in
 * binary64, and strictly inside (0, 1)), and Box-Muller on the
 * pairs (u0,u1), (u2,u3), (u4,u5) gives z_0..z_5, of which z_0..z_k are used
 * (k = number of in-grid neighbours): x = mu + L z with L the Cholesky factor
 * of the covariance of the vertex and its present neighbours (in the order
 * v, e, n, w, s).  Hits count x_0 < every x_n (min) and x_0 > every x_n (max).
 * near_ties counts samples with min_n |x_0 - x_n| < 1e-4 * sqrt(Sigma_00).
 * Cholesky failure adds eps*I, eps = 1e-6 * trace / (k+1), times 10 per
 * retry, three retries; a vertex whose covariance has zero trace is
 * deterministic. */
int orc_mvn_mc_at(const double *params, int H, int W, int boundary, const int64_t *idx,
                  int64_t n, int S, uint64_t seed, uint32_t field, int64_t *hits_min,
                  int64_t *hits_max, int64_t *hits_saddle, int64_t *near_ties,
                  uint8_t *status) {
  int64_t t, plane = (int64_t)H * W;
  if (S < 1) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int64_t i = idx[t], nidx[4];
    int y = (int)(i / W), x = (int)(i % W), slot[4], k, a, b, nv, st = 0, s;
    int sl[5];
    double mu[5], A[25], L[25], full[5][5], tr = 0.0;
    int64_t hmin = 0, hmax = 0, hsad = 0, ties = 0;
    int ssg[5] = {0, 0, 0, 0, 0}, saddle_ok;
    k = neighbours(H, W, y, x, nidx, slot);
    /* saddle sign of each present neighbour (see vertex_saddle): +1 wants
     * x_v < x_n in t1, -1 wants x_v > x_n */
    saddle_ok = (k == 4) || (k == 2 && (H == 1 || W == 1));
    for (a = 0; a < k; ++a)
      ssg[1 + a] = (k == 4) ? ((slot[a] == 0 || slot[a] == 2) ? 1 : -1)
                            : ((slot[a] == 0 || slot[a] == 3) ? 1 : -1);
    /* unpack the packed covariance */
    {
      int r = 5;
      for (a = 0; a < 5; ++a)
        for (b = 0; b <= a; ++b) {
          full[a][b] = full[b][a] = params[(int64_t)r * plane + i];
          ++r;
        }
    }
    sl[0] = 0;
    for (a = 0; a < k; ++a) sl[1 + a] = 1 + slot[a];
    nv = k + 1;
    for (a = 0; a < nv; ++a) {
      mu[a] = params[(int64_t)sl[a] * plane + i];
      for (b = 0; b < nv; ++b) A[a * nv + b] = full[sl[a]][sl[b]];
      tr += A[a * nv + a];
    }
    for (a = 0; a < nv; ++a)
      if (!isfinite(mu[a])) st |= ST_NONFINITE;
    for (a = 0; a < nv * nv; ++a)
      if (!isfinite(A[a])) st |= ST_NONFINITE;
    if (st) {
      hits_min[t] = hits_max[t] = -1;
      if (hits_saddle) hits_saddle[t] = -1;
      near_ties[t] = 0;
      if (status) status[t] = (uint8_t)st;
      continue;
    }
    /* zero boundary mode: minimum and maximum are 0 where a neighbour is
     * missing; the saddle and the flags are computed as usual */
    if (tr == 0.0) {
      int lt = 1, gt = 1;
      for (a = 1; a < nv; ++a) {
        lt &= mu[0] < mu[a];
        gt &= mu[0] > mu[a];
      }
      hits_min[t] = (lt && !(boundary == 1 && k < 4)) ? S : 0;
      hits_max[t] = (gt && !(boundary == 1 && k < 4)) ? S : 0;
      if (hits_saddle) {
        int t1 = saddle_ok, t2 = saddle_ok;
        for (a = 1; a < nv; ++a) {
          t1 &= ssg[a] > 0 ? mu[0] < mu[a] : mu[0] > mu[a];
          t2 &= ssg[a] > 0 ? mu[0] > mu[a] : mu[0] < mu[a];
        }
        hits_saddle[t] = (t1 || t2) ? S : 0;
      }
      near_ties[t] = 0;
      if (status) status[t] = ST_DEGENERATE;
      continue;
    }
    if (!cholesky(A, nv, L)) {
      double eps = 1e-6 * tr / nv, B2[25];
      int r, ok = 0;
      for (r = 0; r < 3 && !ok; ++r) {
        memcpy(B2, A, sizeof(double) * nv * nv);
        for (a = 0; a < nv; ++a) B2[a * nv + a] += eps;
        ok = cholesky(B2, nv, L);
        eps *= 10.0;
      }
      st |= ok ? ST_CHOL_JITTER : ST_CHOL_FAIL;
      if (!ok) {
        hits_min[t] = hits_max[t] = -1;
        if (hits_saddle) hits_saddle[t] = -1;
        near_ties[t] = 0;
        if (status) status[t] = (uint8_t)st;
        continue;
      }
    }
    {
      const double tie_tol = 1e-4 * sqrt(A[0]);
      const double two_pi = 6.283185307179586476925286766559;
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      for (s = 0; s < S; ++s) {
        uint32_t ctr[4], r8[8];
        double u[6], z[6], xv[5];
        int lt = 1, gt = 1, t1 = saddle_ok, t2 = saddle_ok;
        double dmin = INFINITY;
        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)i; ctr[2] = field; ctr[3] = 0;
        orc_philox4x32_10(ctr, key, r8);
        ctr[3] = 1;
        orc_philox4x32_10(ctr, key, r8 + 4);
        for (a = 0; a < 6; ++a) u[a] = ((double)(r8[a] >> 9) + 0.5) / 8388608.0;
        for (a = 0; a < 3; ++a) {
          double rad = sqrt(-2.0 * log(u[2 * a]));
          double th = two_pi * u[2 * a + 1];
          z[2 * a] = rad * cos(th);
          z[2 * a + 1] = rad * sin(th);
        }
        for (a = 0; a < nv; ++a) {
          double acc = mu[a];
          for (b = 0; b <= a; ++b) acc += L[a * nv + b] * z[b];
          xv[a] = acc;
        }
        for (a = 1; a < nv; ++a) {
          double dd = fabs(xv[0] - xv[a]);
          lt &= xv[0] < xv[a];
          gt &= xv[0] > xv[a];
          t1 &= ssg[a] > 0 ? xv[0] < xv[a] : xv[0] > xv[a];
          t2 &= ssg[a] > 0 ? xv[0] > xv[a] : xv[0] < xv[a];
          if (dd < dmin) dmin = dd;
        }
        hmin += lt;
        hmax += gt;
        hsad += (t1 || t2);
        ties += (nv > 1 && dmin < tie_tol);
      }
    }
    hits_min[t] = (boundary == 1 && k < 4) ? 0 : hmin;
    hits_max[t] = (boundary == 1 && k < 4) ? 0 : hmax;
    if (hits_saddle) hits_saddle[t] = hsad;
    near_ties[t] = ties;
    if (status) status[t] = (uint8_t)st;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* semianalytical histogram estimator (Sec. "Semianalytical Solution")       */
/*                                                                          */
/* c samples x_s are drawn from the centre's histogram; for each, the        */
/* probability of being below (above) every neighbour is exact: the product */
/* of the neighbours' mixture survivals G_n(x_s) (CDFs F_n(x_s)); the        */
/* estimate is T_1 times the mean over the samples (T_1 = the centre's total */
/* mass).  Sampling: sample s uses Philox4x32-10 with counter (s >> 1, i,    */
/* field, 2) and the seed as key; words 0, 1 (even s) or 2, 3 (odd s) give    */
/* uniforms ua, ub as for the Gaussian path.  The bin is an integer decision */
/* taken in IEEE binary32 on both sides: t = ua * T_1 (T_1 summed in bin     */
/* order in binary32), j = the number of running sums C_1..C_B (binary32,    */
/* in bin order) that are <= t, clamped to B-1; then x = lo + (j + ub) h.    */
/* A point-mass centre is exact (every sample is its position).             */

static double semi_sample_x(const dist_t *v, float ua, float ub) {
  float T = 0.0f, C = 0.0f, t;
  int j, cnt = 0, B = v->B;
  for (j = 0; j < B; ++j) T += (float)v->w[j];
  t = ua * T;
  for (j = 0; j < B; ++j) {
    C += (float)v->w[j];
    cnt += (C <= t);
  }
  if (cnt > B - 1) cnt = B - 1;
  return v->lo + ((double)cnt + (double)ub) * (v->hi - v->lo) / (double)B;
}

/* Estimates of P_min, P_max, P_saddle at vertices idx (histogram params);
 * sd_* (nullable) receive the sample standard deviation of each mean. */
int orc_semi_at(const double *params, int H, int W, int B, int boundary, const int64_t *idx,
                int64_t n, int c, uint64_t seed, uint32_t field, double *out_min,
                double *out_max, double *out_saddle, double *sd_min, double *sd_max) {
  int64_t t, plane = (int64_t)H * W;
  if (c < 1 || B < 1 || B > MAXB) return -1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(orc_get_threads())
  for (t = 0; t < n; ++t) {
    int64_t i = idx[t], nidx[4];
    int y = (int)(i / W), x = (int)(i % W), slot[4], k, q, st, ssg[4] = {0, 0, 0, 0}, has_sad;
    double pv[2 + MAXB], smin = 0, smax = 0, ssad = 0, qmin = 0, qmax = 0;
    dist_t v, nb[4];
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    k = neighbours(H, W, y, x, nidx, slot);
    gather_params(params, plane, 2 + B, i, pv);
    st = dist_make(ORC_HIST, pv, B, &v);
    for (q = 0; q < k; ++q) {
      double pn[2 + MAXB];
      gather_params(params, plane, 2 + B, nidx[q], pn);
      st |= dist_make(ORC_HIST, pn, B, &nb[q]);
    }
    if (st & (ST_NONFINITE | ST_BAD_PARAMS)) {
      out_min[t] = out_max[t] = out_saddle[t] = NAN;
      continue;
    }
    has_sad = (k == 4) || (k == 2 && (H == 1 || W == 1));
    for (q = 0; q < k; ++q)
      ssg[q] = (k == 4) ? ((slot[q] == 0 || slot[q] == 2) ? 1 : -1)
                        : ((slot[q] == 0 || slot[q] == 3) ? 1 : -1);
    if (v.point) {
      double pm = v.total, pM = v.total, t1 = v.total, t2 = v.total;
      for (q = 0; q < k; ++q) {
        double g = prob_greater(&nb[q], v.lo), f = prob_less(&nb[q], v.lo);
        pm *= g;
        pM *= f;
        t1 *= ssg[q] > 0 ? g : f;
        t2 *= ssg[q] > 0 ? f : g;
      }
      smin = pm * c;
      smax = pM * c;
      ssad = has_sad ? (t1 + t2) * c : 0.0;
      qmin = pm * pm * c;
      qmax = pM * pM * c;
    } else {
      int s;
      for (s = 0; s < c; ++s) {
        uint32_t ctr[4] = {(uint32_t)(s >> 1), (uint32_t)i, field, 2u}, r[4];
        float ua, ub;
        double xs, pm = v.total, pM = v.total, t1 = v.total, t2 = v.total;
        orc_philox4x32_10(ctr, key, r);
        ua = (float)(((double)(r[(s & 1) * 2] >> 8) + 0.5) / 16777216.0);
        ub = (float)(((double)(r[(s & 1) * 2 + 1] >> 8) + 0.5) / 16777216.0);
        xs = semi_sample_x(&v, ua, ub);
        for (q = 0; q < k; ++q) {
          /* G_n(x) = Pr[X_n > x], F_n(x) = Pr[X_n < x] in the mixture form */
          double g = prob_greater(&nb[q], xs), f = prob_less(&nb[q], xs);
          pm *= g;
          pM *= f;
          t1 *= ssg[q] > 0 ? g : f;
          t2 *= ssg[q] > 0 ? f : g;
        }
        smin += pm;
        smax += pM;
        qmin += pm * pm;
        qmax += pM * pM;
        if (has_sad) ssad += t1 + t2;
      }
    }
    out_min[t] = smin / c;
    out_max[t] = smax / c;
    out_saddle[t] = ssad / c;
    if (boundary == 1 && k < 4) out_min[t] = out_max[t] = 0.0;
    if (sd_min) sd_min[t] = sqrt(fmax(qmin / c - (smin / c) * (smin / c), 0.0) / c);
    if (sd_max) sd_max[t] = sqrt(fmax(qmax / c - (smax / c) * (smax / c), 0.0) / c);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* gradients of L = sum_v W_v P_v with respect to every vertex's parameters  */
/*                                                                          */
/* P_v depends on the parameters of v and of its in-grid neighbours only.   */
/* For a neighbour n, G_n (or F_n) is continuous in its parameters and the  */
/* derivative is taken under the integral sign.  For the centre, the uniform */
/* density jumps at the moving support ends, which adds the Leibniz boundary */
/* terms; the Epanechnikov density vanishes there and adds none; histogram   */
/* masses do not move any breakpoint.  Histogram gradients are with respect  */
/* to the masses only, in the mixture form (P_v is linear in each vertex's   */
/* masses).  Parameters of point masses get zero own-derivatives.            */

/* derivative factor for a neighbour parameter q (0,1 for uniform/Epan, bin j
 * for histogram), for the survival (want_max = 0) or the CDF (want_max = 1) */
static void neighbour_dfactor(const dist_t *d, int q, int want_max, pw_t *out) {
  double sg = want_max ? -1.0 : 1.0;
  memset(out, 0, sizeof(*out));
  if (d->point) {
    if (d->model == ORC_HIST) {
      /* G = T [x < c]: dG/dw_j = [x < c] */
      if (want_max) pw_step(out, d->lo, 0.0, 1.0);
      else pw_step(out, d->lo, 1.0, 0.0);
    } else {
      pw_step(out, d->lo, 0.0, 0.0);
    }
    return;
  }
  if (d->model == ORC_UNIFORM) {
    double a = d->p0, b = d->p1, r2 = 1.0 / ((b - a) * (b - a));
    out->m = 1; out->e[0] = a; out->e[1] = b; out->n[0] = 2;
    if (q == 0) { /* dG/da = (b - x)/(b-a)^2, t = x - a */
      out->c[0][0] = sg * (b - a) * r2; out->c[0][1] = -sg * r2;
    } else {      /* dG/db = (x - a)/(b-a)^2 */
      out->c[0][0] = 0.0; out->c[0][1] = sg * r2;
    }
  } else if (d->model == ORC_EPAN) {
    double m = d->p0, w = d->p1;
    out->m = 1; out->e[0] = m - w; out->e[1] = m + w;
    if (q == 0) { /* dG/dm = pdf(x) */
      int j;
      out->n[0] = 3;
      for (j = 0; j < 3; ++j) out->c[0][j] = sg * d->pdf.c[0][j];
    } else {      /* dG/dw = pdf(x) (x - m)/w,  x - m = t - w */
      double tmp[MAXPROD], lin[2] = {-1.0, 1.0 / w};
      int j, nn = poly_mul(d->pdf.c[0], 3, lin, 2, tmp);
      out->n[0] = nn;
      for (j = 0; j < nn; ++j) out->c[0][j] = sg * tmp[j];
    }
  } else { /* histogram bin q: dG/dw_q = survival of the uniform bin q */
    double e0 = d->pdf.e[q], e1 = d->pdf.e[q + 1];
    out->m = 1; out->e[0] = e0; out->e[1] = e1; out->n[0] = 2;
    if (want_max) {
      out->c[0][0] = 0.0; out->c[0][1] = 1.0 / (e1 - e0);
      out->left = 0.0; out->right = 1.0;
    } else {
      out->c[0][0] = 1.0; out->c[0][1] = -1.0 / (e1 - e0);
      out->left = 1.0; out->right = 0.0;
    }
  }
}

/* dP_v / d(parameter q of participant p), p = 0 for the centre, 1..k for the
 * neighbours (in the order returned by neighbours()) */
static double vertex_partial(const dist_t *v, const dist_t *nb, int k, int want_max, int p,
                             int q) {
  const pw_t *f[5];
  pw_t dfac;
  int n;
  if (v->point) {
    double c = v->lo, prod = v->total;
    if (p == 0) {
      if (v->model != ORC_HIST) return 0.0;
      prod = 1.0; /* d(total)/dw_q = 1 */
      for (n = 0; n < k; ++n)
        prod *= want_max ? prob_less(&nb[n], c) : prob_greater(&nb[n], c);
      return prod;
    }
    for (n = 0; n < k; ++n) {
      if (n == p - 1) {
        neighbour_dfactor(&nb[n], q, want_max, &dfac);
        prod *= pw_eval(&dfac, c);
      } else {
        prod *= want_max ? prob_less(&nb[n], c) : prob_greater(&nb[n], c);
      }
    }
    return prod;
  }
  for (n = 0; n < k; ++n) f[1 + n] = want_max ? &nb[n].F : &nb[n].G;
  if (p == 0) {
    if (v->model == ORC_UNIFORM) {
      double a = v->p0, b = v->p1, P, Ha = 1.0, Hb = 1.0;
      f[0] = &v->pdf;
      P = integrate_product(f, 1 + k, a, b);
      for (n = 0; n < k; ++n) {
        Ha *= pw_eval(f[1 + n], a);
        Hb *= pw_eval(f[1 + n], b);
      }
      return q == 0 ? (P - Ha) / (b - a) : (Hb - P) / (b - a);
    } else if (v->model == ORC_EPAN) {
      double m = v->p0, w = v->p1;
      memset(&dfac, 0, sizeof(dfac));
      dfac.m = 1; dfac.e[0] = m - w; dfac.e[1] = m + w;
      if (q == 0) { /* d pdf/dm = 3 (x - m)/(2 w^3), x - m = t - w */
        dfac.n[0] = 2;
        dfac.c[0][0] = -3.0 / (2.0 * w * w);
        dfac.c[0][1] = 3.0 / (2.0 * w * w * w);
      } else {      /* d pdf/dw = -3/(4 w^2) (1 - 3 u^2), u = (t - w)/w */
        double c2 = -3.0 / (4.0 * w * w);
        /* 1 - 3 (t/w - 1)^2 = -2 + 6 t/w - 3 t^2/w^2 */
        dfac.n[0] = 3;
        dfac.c[0][0] = c2 * -2.0;
        dfac.c[0][1] = c2 * 6.0 / w;
        dfac.c[0][2] = c2 * -3.0 / (w * w);
      }
      f[0] = &dfac;
      return integrate_product(f, 1 + k, m - w, m + w);
    } else { /* histogram: (1/h) integral over bin q of the product */
      memset(&dfac, 0, sizeof(dfac));
      dfac.m = 1; dfac.e[0] = v->pdf.e[q]; dfac.e[1] = v->pdf.e[q + 1];
      dfac.n[0] = 1; dfac.c[0][0] = 1.0 / (dfac.e[1] - dfac.e[0]);
      f[0] = &dfac;
      return integrate_product(f, 1 + k, dfac.e[0], dfac.e[1]);
    }
  }
  neighbour_dfactor(&nb[p - 1], q, want_max, &dfac);
  f[0] = &v->pdf;
  f[p] = &dfac;
  return integrate_product(f, 1 + k, v->lo, v->hi);
}

/* grad: [Q][H][W] with Q = 2 (uniform, Epanechnikov) or B (histogram masses).
 * weight: [H][W].  cptype: 1 = minimum, 2 = maximum. */
int orc_grad(const double *params, int H, int W, int model, int B, int boundary, int cptype,
             const double *weight, double *grad) {
  int64_t plane = (int64_t)H * W;
  int Q = (model == ORC_HIST) ? B : 2, np = nparams(model, B), want_max = (cptype == 2);
  int y;
  if (model != ORC_UNIFORM && model != ORC_EPAN && model != ORC_HIST) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
  for (y = 0; y < H; ++y) {
    int x;
    for (x = 0; x < W; ++x) {
      int64_t u = (int64_t)y * W + x, vids[5];
      int nv, t, q;
      double acc[MAXB];
      for (q = 0; q < Q; ++q) acc[q] = 0.0;
      /* the vertices whose probability depends on u: u itself and its
       * in-grid neighbours */
      vids[0] = u;
      nv = 1 + neighbours(H, W, y, x, vids + 1, NULL);
      for (t = 0; t < nv; ++t) {
        int64_t v = vids[t], nidx[4];
        int vy = (int)(v / W), vx = (int)(v % W), k, n, p = -1, st;
        double pv[2 + MAXB];
        dist_t dv, nb[4];
        k = neighbours(H, W, vy, vx, nidx, NULL);
        if (boundary == 1 && k < 4) continue;
        gather_params(params, plane, np, v, pv);
        st = dist_make(model, pv, B, &dv);
        for (n = 0; n < k; ++n) {
          double pn[2 + MAXB];
          gather_params(params, plane, np, nidx[n], pn);
          st |= dist_make(model, pn, B, &nb[n]);
          if (nidx[n] == u) p = 1 + n;
        }
        if (t == 0) p = 0;
        if (st & (ST_NONFINITE | ST_BAD_PARAMS)) {
          for (q = 0; q < Q; ++q) acc[q] = NAN;
          continue;
        }
        for (q = 0; q < Q; ++q) acc[q] += weight[v] * vertex_partial(&dv, nb, k, want_max, p, q);
      }
      for (q = 0; q < Q; ++q) grad[(int64_t)q * plane + u] = acc[q];
    }
  }
  return 0;
}
