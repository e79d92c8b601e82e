/*
 * nbref.c — CPU oracle of the hybrid symplectic step (test infrastructure).
 *
 * Plain C11, FP64, compiled with -O2 -ffp-contract=off and no fast-math.
 * Sums over j run in ascending order for each i; OpenMP splits only the
 * outer i loop, so results do not depend on the thread count.
 *
 * Paper passages followed (Grimm & Stadel, section "The hybrid symplectic
 * integrator"):
 *   Eq. H   H = H_A + H_B + H_C                         -> the step's split
 *   Eq. Ha  Kepler part + (1 - K) close part            -> Kepler drift, BS
 *   Eq. Hb  interaction part weighted by K              -> kick
 *   Eq. Hc  momentum part |sum p|^2 / (2 m0)           -> linear drift
 *   Eq. rcrit  r_crit = max(3 R_Hill, 0.4 dt v)         -> changeover radius
 * and "Detailing the outcomes of collisions" (perfect mergers).
 *
 * Where the paper is silent the following readings are taken (each is
 * repeated at the function that implements it):
 *   - operator order B(h/2) C(h/2) A(h) C(h/2) B(h/2);
 *   - K(y) = f(y) / (f(y) + f(1 - y)), f(y) = exp(-1/y), y = (r - 0.1 rc) / (0.9 rc);
 *   - kick weight w = K - r dK/dr (exact gradient of Eq. Hb), close weight 1 - w;
 *   - rc_ij = max(rc_i, rc_j); a pair is in encounter when r^2 < rc_ij^2 at the
 *     start of the step (flags of the previous force evaluation) or after the
 *     trial Kepler drift;
 *   - r^2 = fma(dz, dz, fma(dy, dy, dx*dx)) (correctly rounded fused form);
 *   - Kepler drift in universal variables, Newton iteration with a
 *     Laguerre-Conway fallback;
 *   - the close-encounter "direct solver" is Gragg-Bulirsch-Stoer;
 *   - R_Hill = |x| (m / (3 m0))^(1/3); v in Eq. rcrit is the speed relative to
 *     the local circular prograde orbit (vel_mode 0) or |v| (vel_mode 1).
 */
#include "nbref.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Changeover function (Eq. Hb and the paragraph after Eq. Hc).        */
/* The paper states that K is smooth, goes from 0 to 1, and that the    */
/* transition must be smooth enough. Reading: the infinitely            */
/* differentiable switch K(y) = f(y) / (f(y) + f(1 - y)),               */
/* f(y) = exp(-1/y) for y > 0, with y = (r - 0.1 rc) / (0.9 rc).        */
/* dK/dy = f(y) f(1-y) (1/y^2 + 1/(1-y)^2) / (f(y) + f(1-y))^2.          */
/* ------------------------------------------------------------------ */
void nbref_changeover(double r, double rc, double* K, double* dKdr) {
  double y = (r - 0.1 * rc) / (0.9 * rc);
  if (y <= 0.0) {
    *K = 0.0;
    *dKdr = 0.0;
  } else if (y >= 1.0) {
    *K = 1.0;
    *dKdr = 0.0;
  } else {
    double f = exp(-1.0 / y);
    double g = exp(-1.0 / (1.0 - y));
    double s = f + g;
    *K = f / s;
    double fg = f * g;
    double dKdy = 0.0;
    if (fg > 0.0) dKdy = fg * (1.0 / (y * y) + 1.0 / ((1.0 - y) * (1.0 - y))) / (s * s);
    *dKdr = dKdy / (0.9 * rc);
  }
}

/* Kick weight of a pair: -grad of -G mi mj K(r)/r gives G mi mj (K - r K') dx / r^3. */
static double kick_weight(double r, double rc) {
  double K, dK;
  nbref_changeover(r, rc, &K, &dK);
  return K - r * dK;
}

/* ------------------------------------------------------------------ */
/* Stumpff functions c_k(z) = sum_j (-z)^j / (2j + k)!                 */
/* Series for |z| < 1, trigonometric / hyperbolic closed forms beyond. */
/* ------------------------------------------------------------------ */
void nbref_stumpff(double z, double c[4]) {
  if (fabs(z) < 1.0) {
    for (int k = 0; k < 4; ++k) {
      /* term_0 = 1/k!, term_{j+1} = term_j * (-z) / ((2j+k+1)(2j+k+2)) */
      double fact = 1.0;
      for (int q = 2; q <= k; ++q) fact *= q;
      double term = 1.0 / fact;
      double sum = term;
      for (int j = 0; j < 30; ++j) {
        term = term * (-z) / ((double)(2 * j + k + 1) * (double)(2 * j + k + 2));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      c[k] = sum;
    }
  } else if (z > 0.0) {
    double u = sqrt(z);
    double sh = sin(0.5 * u);
    c[0] = cos(u);
    c[1] = sin(u) / u;
    c[2] = 2.0 * sh * sh / z;
    c[3] = (u - sin(u)) / (u * z);
  } else {
    double u = sqrt(-z);
    double sh = sinh(0.5 * u);
    c[0] = cosh(u);
    c[1] = sinh(u) / u;
    c[2] = 2.0 * sh * sh / (-z);
    c[3] = (sinh(u) - u) / (u * (-z));
  }
}

/* G_k(s) = s^k c_k(beta s^2) */
static void gfun(double beta, double s, double G[4]) {
  double c[4];
  nbref_stumpff(beta * s * s, c);
  G[0] = c[0];
  G[1] = s * c[1];
  G[2] = s * s * c[2];
  G[3] = s * s * s * c[3];
}

/* ------------------------------------------------------------------ */
/* Kepler flow of H_A's first sum (Eq. Ha), mu = G m0: "solved          */
/* analytically" (section "The symplectic integrator"). Universal      */
/* variable s solves t(s) = r0 G1 + eta G2 + mu G3 = h. Newton's method */
/* first; if it has not converged after 10 updates, Laguerre-Conway    */
/* (n = 5) from the same start. An update smaller than 1e-10 |s| is    */
/* followed by one more update, after which the iteration stops.       */
/* ------------------------------------------------------------------ */
static int solve_universal(double mu, double r0, double eta, double beta, double h,
                           int max_iter, double* s_out, int* iters) {
  /* Start: the second-order expansion t(s) = r0 s + eta s^2 / 2 + ... For an
   * unbound orbit (beta < 0) deep in the exponential regime, where
   * t(s) ~ exp(g|s|) (r0 + sgn(h) eta/g + mu/g^2) / (2g) with g = sqrt(-beta),
   * the asymptotic inverse is used when it is the smaller of the two. */
  double s0 = h / r0 - eta * h * h / (2.0 * r0 * r0 * r0);
  if (beta < 0.0) {
    double g = sqrt(-beta);
    if (g * fabs(s0) > 2.0) {
      double sg = h > 0.0 ? 1.0 : -1.0;
      double c = r0 + sg * eta / g + mu / (g * g);
      double arg = 2.0 * g * fabs(h) / c;
      if (c > 0.0 && arg > 1.0) {
        double sa = sg * log(arg) / g;
        if (fabs(sa) < fabs(s0)) s0 = sa;
      }
    }
  }
  int it = 0;
  for (int method = 0; method < 2; ++method) {
    double s = s0;
    int last = 0;
    int cap = (method == 0) ? 10 : max_iter;
    for (int k = 0; k < cap && it < max_iter; ++k, ++it) {
      double G[4];
      gfun(beta, s, G);
      double F = r0 * G[1] + eta * G[2] + mu * G[3] - h;
      double Fp = r0 * G[0] + eta * G[1] + mu * G[2];
      double ds;
      if (method == 0) {
        ds = F / Fp;
      } else {
        double Fpp = eta * G[0] + (mu - beta * r0) * G[1];
        const double n = 5.0;
        double disc = fabs((n - 1.0) * (n - 1.0) * Fp * Fp - n * (n - 1.0) * F * Fpp);
        double den = Fp + (Fp >= 0.0 ? 1.0 : -1.0) * sqrt(disc);
        ds = n * F / den;
      }
      s -= ds;
      if (!isfinite(s)) break;
      if (last) {
        *s_out = s;
        *iters = it + 1;
        return NBREF_OK;
      }
      if (fabs(ds) <= 1e-10 * fabs(s)) last = 1;
    }
    if (it >= max_iter) break;
  }
  *iters = it;
  return NBREF_E_NOCONV;
}

int nbref_kepler_fg(double mu, const double x[3], const double v[3], double h, int max_iter,
                    double fg[4]) {
  double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double eta = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  double beta = 2.0 * mu / r0 - v2;
  double s;
  int iters;
  if (h == 0.0) {
    fg[0] = 1.0; fg[1] = 0.0; fg[2] = 0.0; fg[3] = 1.0;
    return NBREF_OK;
  }
  int st = solve_universal(mu, r0, eta, beta, h, max_iter, &s, &iters);
  if (st) return st;
  double G[4];
  gfun(beta, s, G);
  double r = r0 * G[0] + eta * G[1] + mu * G[2];
  fg[0] = 1.0 - mu * G[2] / r0;
  fg[1] = r0 * G[1] + eta * G[2];
  fg[2] = -mu * G[1] / (r * r0);
  fg[3] = 1.0 - mu * G[2] / r;
  return NBREF_OK;
}

int nbref_kepler_drift(double mu, double x[3], double v[3], double h, int max_iter, int* iters) {
  *iters = 0;
  if (h == 0.0) return NBREF_OK;
  double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double eta = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  double beta = 2.0 * mu / r0 - v2;
  double s;
  int st = solve_universal(mu, r0, eta, beta, h, max_iter, &s, iters);
  if (st) return st;
  double G[4];
  gfun(beta, s, G);
  double r = r0 * G[0] + eta * G[1] + mu * G[2];
  /* f - 1, g, fdot, gdot - 1 (Gauss f and g functions) */
  double fm1 = -mu * G[2] / r0;
  double g = r0 * G[1] + eta * G[2];
  double fd = -mu * G[1] / (r * r0);
  double gdm1 = -mu * G[2] / r;
  double xn[3], vn[3];
  for (int k = 0; k < 3; ++k) {
    xn[k] = x[k] + (fm1 * x[k] + g * v[k]);
    vn[k] = v[k] + (fd * x[k] + gdm1 * v[k]);
  }
  for (int k = 0; k < 3; ++k) {
    x[k] = xn[k];
    v[k] = vn[k];
  }
  return NBREF_OK;
}

/* ------------------------------------------------------------------ */
/* Eq. rcrit: r_crit = max(hill_factor R_Hill, vel_factor |dt| v).     */
/* ------------------------------------------------------------------ */
double nbref_rcrit(const nbref_params* p, const double x[3], const double v[3], double m) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double rhill = r * cbrt(m / (3.0 * p->m0));
  double vrel;
  if (p->vel_mode == 0) {
    double rxy = sqrt(x[0] * x[0] + x[1] * x[1]);
    double vc[3] = {0.0, 0.0, 0.0};
    if (rxy > 0.0 && r > 0.0) {
      double vk = sqrt(p->G * p->m0 / r);
      vc[0] = -vk * x[1] / rxy;
      vc[1] = vk * x[0] / rxy;
    }
    double d0 = v[0] - vc[0], d1 = v[1] - vc[1], d2 = v[2] - vc[2];
    vrel = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  } else {
    vrel = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  }
  double a = p->hill_factor * rhill;
  double b = p->vel_factor * fabs(p->dt_rcrit) * vrel;
  return a > b ? a : b;
}

void nbref_default_params(nbref_params* p) {
  p->G = 2.959122082855911e-4; /* k^2, k = 0.01720209895 */
  p->m0 = 1.0;
  p->dt_rcrit = 6.0;
  p->hill_factor = 3.0;
  p->vel_factor = 0.4;
  p->vel_mode = 0;
  p->merge = 1;
  p->bs_tol = 1e-14;
  p->bs_kmax = 8;
  p->bs_max_halvings = 20;
  p->kepler_max_iter = 30;
  p->rcrit_refresh = 0;
  p->gas = 0;
  p->gas_rho0 = 2.36e-3; /* 1.4e-9 g cm^-3 (minimum-mass nebula at 1 AU) */
  p->gas_p = 2.75;
  p->gas_eta = 2e-3;
  p->gas_cd = 1.0;
  p->gas_iter = 30;
  p->eject_r = 0.0;
  p->ml_levels = 0;
  p->ml_factor = 3;
}

/* ------------------------------------------------------------------ */
/* Dynamic pair list                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
  int* ij; /* 2 ints per pair */
  int n, cap;
} pairlist;

static void pl_push(pairlist* l, int i, int j) {
  if (l->n == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 64;
    l->ij = (int*)realloc(l->ij, sizeof(int) * 2 * (size_t)l->cap);
  }
  l->ij[2 * l->n] = i;
  l->ij[2 * l->n + 1] = j;
  l->n++;
}

static int pair_cmp(const void* a, const void* b) {
  const int* p = (const int*)a;
  const int* q = (const int*)b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Kick accelerations from Eq. Hb and the encounter flags, over bodies  */
/* with alive[k] != 0 (alive may be NULL = all).                        */
/* ------------------------------------------------------------------ */
static void forces_flags(int n, const double* x, const double* m, const double* rc,
                         const int* alive, double G, double* a, pairlist* flags) {
  int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
  int** loc = (int**)calloc((size_t)n + 1, sizeof(int*));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    a[3 * i] = a[3 * i + 1] = a[3 * i + 2] = 0.0;
    if (alive && !alive[i]) continue;
    double ax = 0.0, ay = 0.0, az = 0.0;
    int mycap = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i || (alive && !alive[j])) continue;
      double dx = x[3 * j] - x[3 * i];
      double dy = x[3 * j + 1] - x[3 * i + 1];
      double dz = x[3 * j + 2] - x[3 * i + 2];
      double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      double rc_ij = rc[i] > rc[j] ? rc[i] : rc[j];
      double rc2 = rc_ij * rc_ij;
      if (r2 < rc2 && i < j) {
        if (cnt[i] == mycap) {
          mycap = mycap ? 2 * mycap : 4;
          loc[i] = (int*)realloc(loc[i], sizeof(int) * (size_t)mycap);
        }
        loc[i][cnt[i]++] = j;
      }
      if (r2 == 0.0) continue; /* coincident bodies exert no kick */
      double r = sqrt(r2);
      double w = 1.0;
      if (r2 < rc2) w = kick_weight(r, rc_ij);
      double f = G * m[j] * w / (r2 * r);
      ax += f * dx;
      ay += f * dy;
      az += f * dz;
    }
    a[3 * i] = ax;
    a[3 * i + 1] = ay;
    a[3 * i + 2] = az;
  }
  if (flags) {
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < cnt[i]; ++k) pl_push(flags, i, loc[i][k]);
  }
  for (int i = 0; i < n; ++i) free(loc[i]);
  free(loc);
  free(cnt);
}

int nbref_forces(int n, const double* x, const double* m, const double* rc, double G,
                 double* a, int* pairs, int cap, int* npairs) {
  if (n < 0) return NBREF_E_INVALID;
  pairlist l = {0, 0, 0};
  forces_flags(n, x, m, rc, NULL, G, a, &l);
  *npairs = l.n;
  for (int k = 0; k < l.n && k < cap; ++k) {
    pairs[2 * k] = l.ij[2 * k];
    pairs[2 * k + 1] = l.ij[2 * k + 1];
  }
  free(l.ij);
  return NBREF_OK;
}

/* Kick acceleration of selected targets only (all sources), and the flagged
 * pairs that involve a selected target, as (min, max) index pairs sorted and
 * unique. Same pair expression as forces_flags. */
int nbref_forces_targets(int n, const double* x, const double* m, const double* rc, double G,
                         const int* targets, int nt, double* a, int* pairs, int cap,
                         int* npairs) {
  pairlist l = {0, 0, 0};
  for (int q = 0; q < nt; ++q) {
    int i = targets[q];
    if (i < 0 || i >= n) return NBREF_E_INVALID;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = x[3 * j] - x[3 * i];
      double dy = x[3 * j + 1] - x[3 * i + 1];
      double dz = x[3 * j + 2] - x[3 * i + 2];
      double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      double rc_ij = rc[i] > rc[j] ? rc[i] : rc[j];
      double rc2 = rc_ij * rc_ij;
      if (r2 < rc2) pl_push(&l, i < j ? i : j, i < j ? j : i);
      if (r2 == 0.0) continue;
      double r = sqrt(r2);
      double w = 1.0;
      if (r2 < rc2) w = kick_weight(r, rc_ij);
      double f = G * m[j] * w / (r2 * r);
      ax += f * dx;
      ay += f * dy;
      az += f * dz;
    }
    a[3 * q] = ax;
    a[3 * q + 1] = ay;
    a[3 * q + 2] = az;
  }
  if (l.n) qsort(l.ij, (size_t)l.n, 2 * sizeof(int), pair_cmp);
  int ne = 0;
  for (int k = 0; k < l.n; ++k) {
    if (ne > 0 && l.ij[2 * k] == l.ij[2 * (ne - 1)] && l.ij[2 * k + 1] == l.ij[2 * (ne - 1) + 1])
      continue;
    l.ij[2 * ne] = l.ij[2 * k];
    l.ij[2 * ne + 1] = l.ij[2 * k + 1];
    ne++;
  }
  *npairs = ne;
  for (int k = 0; k < ne && k < cap; ++k) {
    pairs[2 * k] = l.ij[2 * k];
    pairs[2 * k + 1] = l.ij[2 * k + 1];
  }
  free(l.ij);
  return NBREF_OK;
}

/* ------------------------------------------------------------------ */
/* Bulirsch-Stoer integration of H_A restricted to a group: the paper's */
/* "direct solver" for close encounters (the paragraph after Eq. rcrit).*/
/* Equations of motion of Eq. Ha for group members:                    */
/*   dx_i/dt = v_i                                                      */
/*   dv_i/dt = -G m0 x_i / |x_i|^3 + sum_j G m_j (1 - w_ij) dx / r^3    */
/* Gragg modified midpoint with n_k = 2k substeps, polynomial            */
/* extrapolation in (step)^2 by Neville's scheme (Hairer, Norsett &     */
/* Wanner 1993, section II.9).                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  const nbref_params* p;
  int n;
  const double* m;
  const double* rc;
  const int* alive;
  long long derivs;
  double rc_scale; /* the level's critical radii are rc * rc_scale */
} bs_sys;

/* y layout: per body [x, y, z, vx, vy, vz] */
static void bs_deriv(bs_sys* S, const double* y, double* dy) {
  const double G = S->p->G, mu = S->p->G * S->p->m0;
  int n = S->n;
  S->derivs++;
  for (int i = 0; i < n; ++i) {
    const double* yi = y + 6 * i;
    double* di = dy + 6 * i;
    if (!S->alive[i]) {
      for (int k = 0; k < 6; ++k) di[k] = 0.0;
      continue;
    }
    di[0] = yi[3];
    di[1] = yi[4];
    di[2] = yi[5];
    double r2 = yi[0] * yi[0] + yi[1] * yi[1] + yi[2] * yi[2];
    double r = sqrt(r2);
    double ks = -mu / (r2 * r);
    double ax = ks * yi[0], ay = ks * yi[1], az = ks * yi[2];
    for (int j = 0; j < n; ++j) {
      if (j == i || !S->alive[j]) continue;
      const double* yj = y + 6 * j;
      double dx = yj[0] - yi[0], dyy = yj[1] - yi[1], dz = yj[2] - yi[2];
      double q2 = fma(dz, dz, fma(dyy, dyy, dx * dx));
      if (q2 == 0.0) continue;
      double q = sqrt(q2);
      double rc = (S->rc[i] > S->rc[j] ? S->rc[i] : S->rc[j]) * S->rc_scale;
      double w = (q2 < rc * rc) ? kick_weight(q, rc) : 1.0;
      double f = G * S->m[j] * (1.0 - w) / (q2 * q);
      ax += f * dx;
      ay += f * dyy;
      az += f * dz;
    }
    di[3] = ax;
    di[4] = ay;
    di[5] = az;
  }
}

/* Modified midpoint over H with nsub substeps (Gragg). */
static void bs_midpoint(bs_sys* S, const double* y0, double H, int nsub, double* out, double* zm,
                        double* zc, double* f) {
  int d = 6 * S->n;
  double hs = H / nsub;
  bs_deriv(S, y0, f);
  for (int k = 0; k < d; ++k) {
    zm[k] = y0[k];
    zc[k] = y0[k] + hs * f[k];
  }
  for (int m = 1; m < nsub; ++m) {
    bs_deriv(S, zc, f);
    for (int k = 0; k < d; ++k) {
      double zn = zm[k] + 2.0 * hs * f[k];
      zm[k] = zc[k];
      zc[k] = zn;
    }
  }
  bs_deriv(S, zc, f);
  for (int k = 0; k < d; ++k) out[k] = 0.5 * (zc[k] + zm[k] + hs * f[k]);
}

/* Scaled error between the two highest extrapolation columns: for each live
 * body, the max-norm of the position (velocity) difference divided by the
 * max-norm of its position (velocity); the maximum over bodies. */
static double bs_error(const bs_sys* S, const double* a, const double* b) {
  double err = 0.0;
  for (int i = 0; i < S->n; ++i) {
    if (!S->alive[i]) continue;
    for (int part = 0; part < 2; ++part) {
      double dmax = 0.0, ymax = 0.0;
      for (int k = 0; k < 3; ++k) {
        int idx = 6 * i + 3 * part + k;
        double d = fabs(a[idx] - b[idx]);
        double y = fabs(a[idx]);
        if (d > dmax) dmax = d;
        if (y > ymax) ymax = y;
      }
      double e = dmax / (ymax + 1e-300);
      if (e > err) err = e;
    }
  }
  return err;
}

/* Energy of two bodies relative to the star and each other (used for the
 * energy removed by a perfect merger). */
static double pair_energy(const nbref_params* p, const double* xi, const double* vi, double mi,
                          const double* xj, const double* vj, double mj) {
  double vi2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
  double vj2 = vj[0] * vj[0] + vj[1] * vj[1] + vj[2] * vj[2];
  double ri = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
  double rj = sqrt(xj[0] * xj[0] + xj[1] * xj[1] + xj[2] * xj[2]);
  double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
  double rij = sqrt(dx * dx + dy * dy + dz * dz);
  return 0.5 * mi * vi2 + 0.5 * mj * vj2 - p->G * p->m0 * mi / ri - p->G * p->m0 * mj / rj -
         p->G * mi * mj / rij;
}

static double body_energy(const nbref_params* p, const double* x, const double* v, double m) {
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  return 0.5 * m * v2 - p->G * p->m0 * m / r;
}

/* Perfect merging on contact (section "Detailing the outcomes of
 * collisions"): after each accepted substep, pairs (i < j) of live members
 * are scanned in ascending order; r_ij < R_i + R_j merges j into i. */
static void bs_merge_scan(const nbref_params* p, int n, double* y, double* m, double* R,
                          double* rc, int* alive, double* E_lost, nbref_stats* st) {
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      if (!alive[i] || !alive[j]) continue;
      double* yi = y + 6 * i;
      double* yj = y + 6 * j;
      double dx = yj[0] - yi[0], dy = yj[1] - yi[1], dz = yj[2] - yi[2];
      double rij = sqrt(dx * dx + dy * dy + dz * dz);
      if (!(rij < R[i] + R[j])) continue;
      double e_before = pair_energy(p, yi, yi + 3, m[i], yj, yj + 3, m[j]);
      double M = m[i] + m[j];
      double xn[6];
      for (int k = 0; k < 6; ++k) xn[k] = (m[i] * yi[k] + m[j] * yj[k]) / M;
      double Rn = cbrt(R[i] * R[i] * R[i] + R[j] * R[j] * R[j]);
      for (int k = 0; k < 6; ++k) yi[k] = xn[k];
      m[i] = M;
      R[i] = Rn;
      alive[j] = 0;
      double e_after = body_energy(p, yi, yi + 3, M);
      *E_lost += e_before - e_after;
      rc[i] = nbref_rcrit(p, yi, yi + 3, M);
      if (st) st->merges++;
    }
  }
}

static int bs_group_scaled(const nbref_params* p, int n, double* x, double* v, double* m,
                           double* R, double* rc, int* alive, double h, double rc_scale,
                           double* E_lost, nbref_stats* st);

int nbref_bs_group(const nbref_params* p, int n, double* x, double* v, double* m, double* R,
                   double* rc, int* alive, double h, double* E_lost, nbref_stats* st) {
  return bs_group_scaled(p, n, x, v, m, R, rc, alive, h, 1.0, E_lost, st);
}

/* The direct solver with the critical radii of the changeover scaled by
 * rc_scale (the last level of the multi-level changeover); r_crit itself,
 * and a merged survivor's recomputed r_crit, stay unscaled. */
static int bs_group_scaled(const nbref_params* p, int n, double* x, double* v, double* m,
                           double* R, double* rc, int* alive, double h, double rc_scale,
                           double* E_lost, nbref_stats* st) {
  int d = 6 * n;
  int kmax = p->bs_kmax;
  if (kmax < 3) kmax = 3;
  double* y = (double*)malloc(sizeof(double) * d);
  double* T = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(kmax + 1) * (size_t)(kmax + 1));
  double* zm = (double*)malloc(sizeof(double) * d);
  double* zc = (double*)malloc(sizeof(double) * d);
  double* f = (double*)malloc(sizeof(double) * d);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      y[6 * i + k] = x[3 * i + k];
      y[6 * i + 3 + k] = v[3 * i + k];
    }
  bs_sys S = {p, n, m, rc, alive, 0, rc_scale};
#define TT(j, k) (T + ((size_t)(j) * (kmax + 1) + (k)) * d)
  int level = 0;          /* substep = h / 2^level */
  long long done = 0;     /* substeps completed at the current level */
  int status = NBREF_OK;
  while (done < (1LL << level)) {
    double H = ldexp(h, -level);
    int accepted = 0, accepted_k = 0;
    for (int j = 1; j <= kmax; ++j) {
      int nj = 2 * j;
      bs_midpoint(&S, y, H, nj, TT(j, 1), zm, zc, f);
      for (int k = 1; k < j; ++k) {
        double ratio = (double)nj / (double)(2 * (j - k));
        double den = ratio * ratio - 1.0;
        double* Tjk = TT(j, k);
        double* Tj1k = TT(j - 1, k);
        double* out = TT(j, k + 1);
        for (int q = 0; q < d; ++q) out[q] = Tjk[q] + (Tjk[q] - Tj1k[q]) / den;
      }
      if (j >= 3) {
        double err = bs_error(&S, TT(j, j), TT(j, j - 1));
        if (err <= p->bs_tol) {
          for (int q = 0; q < d; ++q) y[q] = TT(j, j)[q];
          accepted = 1;
          accepted_k = j;
          break;
        }
      }
    }
    if (accepted) {
      done++;
      if (st) st->bs_substeps++;
      if (p->merge) bs_merge_scan(p, n, y, m, R, rc, alive, E_lost, st);
      /* Step back up a level (double the substep) when the substep converged
       * early and the position is aligned with the coarser grid. */
      if (level > 0 && (done & 1) == 0 && accepted_k <= kmax - 2) {
        level--;
        done >>= 1;
      }
    } else {
      if (level >= p->bs_max_halvings) {
        status = NBREF_E_NOCONV;
        break;
      }
      level++;
      done *= 2;
      if (st) st->bs_halvings++;
    }
  }
#undef TT
  if (st) st->bs_derivs += S.derivs;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      x[3 * i + k] = y[6 * i + k];
      v[3 * i + k] = y[6 * i + 3 + k];
    }
  free(y);
  free(T);
  free(zm);
  free(zc);
  free(f);
  return status;
}

/* ------------------------------------------------------------------ */
/* Multi-level changeover (section "Increasing N": the step is reduced  */
/* level by level for the bodies concerned, each level with its own     */
/* smooth changeover, and only the last level uses the direct solver).  */
/* Level l has critical radii r_crit * f^-l and substeps tau / f.       */
/* ml_integrate(S, l, tau) moves the bodies S over tau under their       */
/* Kepler motion and the close part of their mutual interaction with    */
/* weight 1 - w_l; at l = L (ml_levels) that is the direct solver with  */
/* radii scaled by f^-L, below it is f substeps of                      */
/*   K_{l+1}(tau'/2) A_{l+1}(tau') K_{l+1}(tau'/2),  tau' = tau / f,     */
/* K_{l+1} the kick with weight w_{l+1} - w_l (the split                  */
/* 1 - w_l = (w_{l+1} - w_l) + (1 - w_{l+1}) of the close part), and    */
/* A_{l+1} the Kepler drift of S except for the level-(l+1) groups:      */
/* pairs within r_crit f^-(l+1) at the substep's start or after the     */
/* trial drift, joined into connected components, each restarted from  */
/* the substep's start and integrated by ml_integrate at level l + 1.   */
/* ------------------------------------------------------------------ */
static int uf_find(int* parent, int k);

typedef struct {
  const nbref_params* p;
  double *x, *v, *m, *R, *rc; /* group-local arrays, x and v 3 per body */
  int* alive;
  double* E_lost;
  nbref_stats* st;
} ml_ctx;

/* f^-level by repeated division (the same rounding on every side) */
static double ml_scale(const nbref_params* p, int level) {
  double s = 1.0;
  for (int l = 0; l < level; ++l) s /= (double)p->ml_factor;
  return s;
}

static double pair_w(double q2, double q, double rcl) {
  return (q2 < rcl * rcl) ? kick_weight(q, rcl) : 1.0;
}

/* K_level(tau): v_i += tau sum_j G m_j (w_level - w_{level-1}) d_ij / r_ij^3 over
 * the live pairs of S (accelerations from the positions first, then applied). */
static void ml_kick(ml_ctx* c, const int* S, int ns, int level, double tau) {
  const double G = c->p->G;
  const double sl = ml_scale(c->p, level), sp = ml_scale(c->p, level - 1);
  double* acc = (double*)calloc(3 * (size_t)ns, sizeof(double));
  for (int a = 0; a < ns; ++a) {
    const int i = S[a];
    if (!c->alive[i]) continue;
    for (int b = 0; b < ns; ++b) {
      const int j = S[b];
      if (j == i || !c->alive[j]) continue;
      const double dx = c->x[3 * j] - c->x[3 * i], dy = c->x[3 * j + 1] - c->x[3 * i + 1],
                   dz = c->x[3 * j + 2] - c->x[3 * i + 2];
      const double q2 = fma(dz, dz, fma(dy, dy, dx * dx));
      if (q2 == 0.0) continue;
      const double q = sqrt(q2);
      const double rcp = c->rc[i] > c->rc[j] ? c->rc[i] : c->rc[j];
      const double dw = pair_w(q2, q, rcp * sl) - pair_w(q2, q, rcp * sp);
      if (dw == 0.0) continue;
      const double f = G * c->m[j] * dw / (q2 * q);
      acc[3 * a] += f * dx;
      acc[3 * a + 1] += f * dy;
      acc[3 * a + 2] += f * dz;
    }
  }
  for (int a = 0; a < ns; ++a) {
    const int i = S[a];
    if (!c->alive[i]) continue;
    for (int k = 0; k < 3; ++k) c->v[3 * i + k] += tau * acc[3 * a + k];
  }
  free(acc);
}

/* pairs (a < b) of S within the level's radii join in parent[] */
static void ml_flag(ml_ctx* c, const int* S, int ns, int level, int* parent) {
  const double sl = ml_scale(c->p, level);
  for (int a = 0; a < ns; ++a) {
    const int i = S[a];
    if (!c->alive[i]) continue;
    for (int b = a + 1; b < ns; ++b) {
      const int j = S[b];
      if (!c->alive[j]) continue;
      const double dx = c->x[3 * j] - c->x[3 * i], dy = c->x[3 * j + 1] - c->x[3 * i + 1],
                   dz = c->x[3 * j + 2] - c->x[3 * i + 2];
      const double q2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double rcl = (c->rc[i] > c->rc[j] ? c->rc[i] : c->rc[j]) * sl;
      if (!(q2 < rcl * rcl)) continue;
      const int ra = uf_find(parent, a), rb = uf_find(parent, b);
      if (ra < rb)
        parent[rb] = ra;
      else if (rb < ra)
        parent[ra] = rb;
    }
  }
}

static int ml_integrate(ml_ctx* c, const int* S, int ns, int level, double tau) {
  const nbref_params* p = c->p;
  if (level >= p->ml_levels) {
    /* the direct solver on S with the level's radii */
    double* gx = (double*)malloc(sizeof(double) * 3 * (size_t)ns);
    double* gv = (double*)malloc(sizeof(double) * 3 * (size_t)ns);
    double* gm = (double*)malloc(sizeof(double) * (size_t)ns);
    double* gR = (double*)malloc(sizeof(double) * (size_t)ns);
    double* grc = (double*)malloc(sizeof(double) * (size_t)ns);
    int* ga = (int*)malloc(sizeof(int) * (size_t)ns);
    for (int a = 0; a < ns; ++a) {
      const int i = S[a];
      for (int k = 0; k < 3; ++k) {
        gx[3 * a + k] = c->x[3 * i + k];
        gv[3 * a + k] = c->v[3 * i + k];
      }
      gm[a] = c->m[i]; gR[a] = c->R[i]; grc[a] = c->rc[i]; ga[a] = c->alive[i];
    }
    const int st = bs_group_scaled(p, ns, gx, gv, gm, gR, grc, ga, tau, ml_scale(p, level),
                                   c->E_lost, c->st);
    for (int a = 0; a < ns; ++a) {
      const int i = S[a];
      for (int k = 0; k < 3; ++k) {
        c->x[3 * i + k] = gx[3 * a + k];
        c->v[3 * i + k] = gv[3 * a + k];
      }
      c->m[i] = gm[a]; c->R[i] = gR[a]; c->rc[i] = grc[a]; c->alive[i] = ga[a];
    }
    free(gx); free(gv); free(gm); free(gR); free(grc); free(ga);
    return st;
  }
  const int f = p->ml_factor;
  const double t1 = tau / (double)f;
  const double mu = p->G * p->m0;
  double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)ns);
  double* vs = (double*)malloc(sizeof(double) * 3 * (size_t)ns);
  int* parent = (int*)malloc(sizeof(int) * (size_t)ns);
  int* sub = (int*)malloc(sizeof(int) * (size_t)ns);
  int status = NBREF_OK;
  for (int k = 0; k < f && status == NBREF_OK; ++k) {
    ml_kick(c, S, ns, level + 1, 0.5 * t1);
    for (int a = 0; a < ns; ++a) parent[a] = a;
    ml_flag(c, S, ns, level + 1, parent);
    for (int a = 0; a < ns; ++a)
      for (int q = 0; q < 3; ++q) {
        xs[3 * a + q] = c->x[3 * S[a] + q];
        vs[3 * a + q] = c->v[3 * S[a] + q];
      }
    for (int a = 0; a < ns; ++a) {
      const int i = S[a];
      if (!c->alive[i]) continue;
      int it;
      const int kst = nbref_kepler_drift(mu, c->x + 3 * i, c->v + 3 * i, t1, p->kepler_max_iter, &it);
      if (c->st) c->st->kepler_iters += it;
      if (kst) status = kst;
    }
    if (status) break;
    ml_flag(c, S, ns, level + 1, parent);
    for (int a = 0; a < ns; ++a) parent[a] = uf_find(parent, a);
    for (int a = 0; a < ns && status == NBREF_OK; ++a) {
      if (parent[a] != a) continue;
      int nsub = 0;
      for (int b = a; b < ns; ++b)
        if (parent[b] == a) sub[nsub++] = S[b];
      if (nsub < 2) continue;
      for (int b = a; b < ns; ++b) {
        if (parent[b] != a) continue;
        for (int q = 0; q < 3; ++q) {
          c->x[3 * S[b] + q] = xs[3 * b + q];
          c->v[3 * S[b] + q] = vs[3 * b + q];
        }
      }
      if (c->st) c->st->ml_groups++;
      status = ml_integrate(c, sub, nsub, level + 1, t1);
    }
    if (status) break;
    ml_kick(c, S, ns, level + 1, 0.5 * t1);
    if (c->st) c->st->ml_substeps++;
  }
  free(xs); free(vs); free(parent); free(sub);
  return status;
}

int nbref_ml_group(const nbref_params* p, int n, double* x, double* v, double* m, double* R,
                   double* rc, int* alive, double h, double* E_lost, nbref_stats* st) {
  ml_ctx mc = {p, x, v, m, R, rc, alive, E_lost, st};
  int* idx = (int*)malloc(sizeof(int) * (size_t)n);
  for (int q = 0; q < n; ++q) idx[q] = q;
  const int status = ml_integrate(&mc, idx, n, 0, h);
  free(idx);
  return status;
}

/* ------------------------------------------------------------------ */
/* System                                                              */
/* ------------------------------------------------------------------ */
struct nbref_system {
  nbref_params p;
  int n;
  double *x, *v, *m, *R, *rc, *a;
  int *id, *alive;
  pairlist fprev; /* flags of the last force evaluation */
  /* encounter log of the last nbref_step call: (step, id_i, id_j) */
  int* log;
  int nlog, caplog;
  double E_lost;
  long long step_index;
  nbref_stats st;
};

static int bad(double q) { return !isfinite(q); }

nbref_system* nbref_create(const nbref_params* p, int n, const double* x, const double* v,
                           const double* m, const double* R, const double* rc_override,
                           const int* ids, int* status) {
  *status = NBREF_E_INVALID;
  if (n < 1 || !p || !x || !v || !m || !R) return NULL;
  if (!(p->m0 > 0.0) || !(p->G > 0.0)) return NULL;
  for (int i = 0; i < 3 * n; ++i)
    if (bad(x[i]) || bad(v[i])) return NULL;
  for (int i = 0; i < n; ++i) {
    if (bad(m[i]) || !(m[i] > 0.0) || bad(R[i]) || R[i] < 0.0) return NULL;
    if (rc_override && (bad(rc_override[i]) || !(rc_override[i] > 0.0))) return NULL;
    if (ids && i > 0 && ids[i] <= ids[i - 1]) return NULL;
  }
  nbref_system* s = (nbref_system*)calloc(1, sizeof(nbref_system));
  s->p = *p;
  s->n = n;
  size_t b3 = sizeof(double) * 3 * (size_t)n, b1 = sizeof(double) * (size_t)n;
  s->x = (double*)malloc(b3);
  s->v = (double*)malloc(b3);
  s->a = (double*)malloc(b3);
  s->m = (double*)malloc(b1);
  s->R = (double*)malloc(b1);
  s->rc = (double*)malloc(b1);
  s->id = (int*)malloc(sizeof(int) * (size_t)n);
  s->alive = (int*)malloc(sizeof(int) * (size_t)n);
  memcpy(s->x, x, b3);
  memcpy(s->v, v, b3);
  memcpy(s->m, m, b1);
  memcpy(s->R, R, b1);
  for (int i = 0; i < n; ++i) {
    s->id[i] = ids ? ids[i] : i;
    s->alive[i] = 1;
    s->rc[i] = rc_override ? rc_override[i] : nbref_rcrit(p, x + 3 * i, v + 3 * i, m[i]);
  }
  forces_flags(n, s->x, s->m, s->rc, s->alive, p->G, s->a, &s->fprev);
  s->st.force_evals++;
  *status = NBREF_OK;
  return s;
}

static void log_push(nbref_system* s, int step, int i, int j) {
  if (s->nlog == s->caplog) {
    s->caplog = s->caplog ? 2 * s->caplog : 256;
    s->log = (int*)realloc(s->log, sizeof(int) * 3 * (size_t)s->caplog);
  }
  s->log[3 * s->nlog] = step;
  s->log[3 * s->nlog + 1] = i;
  s->log[3 * s->nlog + 2] = j;
  s->nlog++;
}

static int uf_find(int* parent, int k) {
  while (parent[k] != k) {
    parent[k] = parent[parent[k]];
    k = parent[k];
  }
  return k;
}

/* C(h/2): x_i += (h/2) P / m0 with P = sum m_i v_i (Eq. Hc). */
static void momentum_drift(nbref_system* s, double hh) {
  double P[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) P[k] += s->m[i] * s->v[3 * i + k];
  }
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) s->x[3 * i + k] += hh * P[k] / s->p.m0;
  }
}

/* B(h/2): v_i += (h/2) a_i (Eq. Hb flow, acceleration cached from the last
 * force evaluation). */
static void kick(nbref_system* s, double hh) {
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) s->v[3 * i + k] += hh * s->a[3 * i + k];
  }
}

/* Gas drag acceleration on body i (section "Modelling additional dynamical
 * effects", gas effects; the paper names no drag law, this reading takes the
 * quadratic law of Adachi et al. 1976 used by Morishima et al. 2010, the
 * model the paper cites): the gas rotates about the star on circles at
 * (1 - eta) times the circular speed sqrt(G m0 / s), s the cylindrical
 * radius, with midplane density rho0 (s / 1 AU)^-p; the body's velocity
 * relative to the star is its barycentric velocity plus P / m0 (the star
 * moves at -P / m0); a = -(C_D pi R^2 rho / (2 m)) |u| u with u the velocity
 * relative to the gas. */
static void drag_acc(const nbref_params* p, const double* x, const double* vb, const double* Pm0,
                     double m, double R, double out[3]) {
  const double sxy = sqrt(x[0] * x[0] + x[1] * x[1]);
  double vg[3] = {0.0, 0.0, 0.0};
  if (sxy > 0.0) {
    const double vk = (1.0 - p->gas_eta) * sqrt(p->G * p->m0 / sxy);
    vg[0] = -vk * x[1] / sxy;
    vg[1] = vk * x[0] / sxy;
  }
  double u[3];
  for (int k = 0; k < 3; ++k) u[k] = vb[k] + Pm0[k] - vg[k];
  const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double rho = p->gas_rho0 * pow(sxy, -p->gas_p);
  const double kd = p->gas_cd * 3.14159265358979323846 * R * R * rho / (2.0 * m);
  for (int k = 0; k < 3; ++k) out[k] = -kd * un * u[k];
}

/* One body's implicit-midpoint drag update (Eq. implicit):
 * v' = v + tau a_f(x, (v + v') / 2), fixed-point iteration from v' = v until
 * successive iterates agree to 1e-15 of |v'| (max-norm) or gas_iter
 * iterations (NBREF_E_NOCONV). Pm0 = P / m0, held for the whole operator. */
int nbref_implicit_drag(const nbref_params* p, const double x[3], const double v[3],
                        const double Pm0[3], double m, double R, double tau, double vout[3]) {
  double w[3] = {v[0], v[1], v[2]};
  int ok = 0;
  for (int it = 0; it < p->gas_iter; ++it) {
    double vm[3], a[3];
    for (int k = 0; k < 3; ++k) vm[k] = 0.5 * (v[k] + w[k]);
    drag_acc(p, x, vm, Pm0, m, R, a);
    double dmax = 0.0, wmax = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double wn = v[k] + tau * a[k];
      dmax = fmax(dmax, fabs(wn - w[k]));
      wmax = fmax(wmax, fabs(wn));
      w[k] = wn;
    }
    if (dmax <= 1e-15 * wmax) {
      ok = 1;
      break;
    }
  }
  for (int k = 0; k < 3; ++k) vout[k] = w[k];
  return ok ? NBREF_OK : NBREF_E_NOCONV;
}

/* G(tau): the implicit-midpoint drag update of every live body with a
 * radius; P is the momentum at the start of the operator. */
static int gas_drag(nbref_system* s, double tau) {
  const nbref_params* p = &s->p;
  double P[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) P[k] += s->m[i] * s->v[3 * i + k];
  }
  const double Pm0[3] = {P[0] / p->m0, P[1] / p->m0, P[2] / p->m0};
  int status = NBREF_OK;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i] || !(s->R[i] > 0.0)) continue;
    double w[3];
    const int st = nbref_implicit_drag(p, s->x + 3 * i, s->v + 3 * i, Pm0, s->m[i], s->R[i], tau, w);
    if (st) {
#pragma omp atomic write
      status = st;
    }
    for (int k = 0; k < 3; ++k) s->v[3 * i + k] = w[k];
  }
  return status;
}

/* Bodies beyond eject_r leave the system (the ejected mass of the
 * resolution study, section on the comparison of resolutions): in ascending
 * order each is deactivated, its mass and the count recorded, and the energy
 * it takes away added to E_lost: its kinetic and star-potential energy, its
 * mutual potential with the bodies still present, and the change of the
 * |P|^2 / (2 m0) term of Eq. Hc. Returns the number removed. */
static int eject(nbref_system* s) {
  const nbref_params* p = &s->p;
  const double r2max = p->eject_r * p->eject_r;
  int ne = 0;
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    const double* x = s->x + 3 * i;
    if (!(x[0] * x[0] + x[1] * x[1] + x[2] * x[2] > r2max)) continue;
    const double* v = s->v + 3 * i;
    const double mi = s->m[i];
    double P[3] = {0.0, 0.0, 0.0}, mutual = 0.0;
    for (int j = 0; j < s->n; ++j) {
      if (!s->alive[j]) continue;
      for (int k = 0; k < 3; ++k) P[k] += s->m[j] * s->v[3 * j + k];
      if (j == i) continue;
      const double dx = s->x[3 * j] - x[0], dy = s->x[3 * j + 1] - x[1], dz = s->x[3 * j + 2] - x[2];
      mutual -= p->G * mi * s->m[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    double Pn2 = 0.0, P2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      P2 += P[k] * P[k];
      Pn2 += (P[k] - mi * v[k]) * (P[k] - mi * v[k]);
    }
    s->E_lost += body_energy(p, x, v, mi) + mutual + (P2 - Pn2) / (2.0 * p->m0);
    s->st.m_ejected += mi;
    s->st.ejections++;
    s->alive[i] = 0;
    ++ne;
  }
  return ne;
}

static int one_step(nbref_system* s, double h) {
  int n = s->n;
  const nbref_params* p = &s->p;
  double mu = p->G * p->m0;
  int ejected = p->eject_r > 0.0 ? eject(s) : 0;
  if (p->rcrit_refresh) {
    /* Eq. rcrit evaluated afresh for every body at the start of the step. */
    for (int i = 0; i < n; ++i)
      if (s->alive[i]) s->rc[i] = nbref_rcrit(p, s->x + 3 * i, s->v + 3 * i, s->m[i]);
  }
  if (p->rcrit_refresh || ejected) {
    /* the cached force and flags anew (new radii, or bodies removed) */
    s->fprev.n = 0;
    forces_flags(n, s->x, s->m, s->rc, s->alive, p->G, s->a, &s->fprev);
    s->st.force_evals++;
  }
  if (p->gas) {
    int gs = gas_drag(s, 0.5 * h);
    if (gs) return gs;
  }
  kick(s, 0.5 * h);
  momentum_drift(s, 0.5 * h);
  size_t b3 = sizeof(double) * 3 * (size_t)n;
  double* xs = (double*)malloc(b3);
  double* vs = (double*)malloc(b3);
  memcpy(xs, s->x, b3);
  memcpy(vs, s->v, b3);
  int status = NBREF_OK;
  long long kit = 0;
#pragma omp parallel for reduction(+ : kit) schedule(static)
  for (int i = 0; i < n; ++i) {
    if (!s->alive[i]) continue;
    int it;
    int st = nbref_kepler_drift(mu, s->x + 3 * i, s->v + 3 * i, h, p->kepler_max_iter, &it);
    kit += it;
    if (st) {
#pragma omp atomic write
      status = st;
    }
  }
  s->st.kepler_iters += kit;
  if (status) {
    free(xs);
    free(vs);
    return status;
  }
  /* Trial force and flags at the drifted positions. */
  pairlist ftrial = {0, 0, 0};
  double* atrial = (double*)malloc(b3);
  forces_flags(n, s->x, s->m, s->rc, s->alive, p->G, atrial, &ftrial);
  s->st.force_evals++;
  /* E = F_prev U F_trial, sorted and unique. */
  pairlist E = {0, 0, 0};
  for (int k = 0; k < s->fprev.n; ++k) pl_push(&E, s->fprev.ij[2 * k], s->fprev.ij[2 * k + 1]);
  for (int k = 0; k < ftrial.n; ++k) pl_push(&E, ftrial.ij[2 * k], ftrial.ij[2 * k + 1]);
  if (E.n) qsort(E.ij, (size_t)E.n, 2 * sizeof(int), pair_cmp);
  int ne = 0;
  for (int k = 0; k < E.n; ++k) {
    if (ne > 0 && E.ij[2 * k] == E.ij[2 * (ne - 1)] && E.ij[2 * k + 1] == E.ij[2 * (ne - 1) + 1])
      continue;
    E.ij[2 * ne] = E.ij[2 * k];
    E.ij[2 * ne + 1] = E.ij[2 * k + 1];
    ne++;
  }
  E.n = ne;
  s->st.encounter_pairs += ne;
  for (int k = 0; k < ne; ++k)
    log_push(s, (int)s->step_index, s->id[E.ij[2 * k]], s->id[E.ij[2 * k + 1]]);
  if (ne > 0) {
    /* Independent close-encounter groups: connected components of E
     * (section "Increasing N"). Union by smaller index, so a root is the
     * smallest member. */
    int* parent = (int*)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) parent[i] = i;
    for (int k = 0; k < ne; ++k) {
      int ra = uf_find(parent, E.ij[2 * k]), rb = uf_find(parent, E.ij[2 * k + 1]);
      if (ra == rb) continue;
      if (ra < rb)
        parent[rb] = ra;
      else
        parent[ra] = rb;
    }
    char* in_e = (char*)calloc((size_t)n, 1);
    for (int k = 0; k < 2 * ne; ++k) in_e[E.ij[k]] = 1;
    int* ebod = (int*)malloc(sizeof(int) * (size_t)n); /* bodies in E, ascending */
    int nb = 0;
    for (int i = 0; i < n; ++i)
      if (in_e[i]) ebod[nb++] = i;
    /* Groups in ascending order of their smallest member (its root). */
    int* members = (int*)malloc(sizeof(int) * (size_t)n);
    for (int q0 = 0; q0 < nb && status == NBREF_OK; ++q0) {
      int root = ebod[q0];
      if (uf_find(parent, root) != root) continue;
      int gn = 0;
      for (int q = q0; q < nb; ++q)
        if (uf_find(parent, ebod[q]) == root) members[gn++] = ebod[q];
      double* gx = (double*)malloc(sizeof(double) * 3 * (size_t)gn);
      double* gv = (double*)malloc(sizeof(double) * 3 * (size_t)gn);
      double* gm = (double*)malloc(sizeof(double) * (size_t)gn);
      double* gR = (double*)malloc(sizeof(double) * (size_t)gn);
      double* grc = (double*)malloc(sizeof(double) * (size_t)gn);
      int* ga = (int*)malloc(sizeof(int) * (size_t)gn);
      for (int q = 0; q < gn; ++q) {
        int b = members[q];
        for (int k = 0; k < 3; ++k) {
          gx[3 * q + k] = xs[3 * b + k]; /* restart from the saved state */
          gv[3 * q + k] = vs[3 * b + k];
        }
        gm[q] = s->m[b];
        gR[q] = s->R[b];
        grc[q] = s->rc[b];
        ga[q] = 1;
      }
      if (p->ml_levels > 0) {
        ml_ctx mc = {p, gx, gv, gm, gR, grc, ga, &s->E_lost, &s->st};
        int* idx = (int*)malloc(sizeof(int) * (size_t)gn);
        for (int q = 0; q < gn; ++q) idx[q] = q;
        status = ml_integrate(&mc, idx, gn, 0, h);
        free(idx);
      } else {
        status = nbref_bs_group(p, gn, gx, gv, gm, gR, grc, ga, h, &s->E_lost, &s->st);
      }
      s->st.groups++;
      for (int q = 0; q < gn; ++q) {
        int b = members[q];
        for (int k = 0; k < 3; ++k) {
          s->x[3 * b + k] = gx[3 * q + k];
          s->v[3 * b + k] = gv[3 * q + k];
        }
        s->m[b] = gm[q];
        s->R[b] = gR[q];
        s->rc[b] = grc[q];
        s->alive[b] = ga[q];
      }
      free(gx); free(gv); free(gm); free(gR); free(grc); free(ga);
    }
    free(members);
    free(ebod);
    free(in_e);
    free(parent);
    /* Force and flags at the final positions. */
    s->fprev.n = 0;
    forces_flags(n, s->x, s->m, s->rc, s->alive, p->G, s->a, &s->fprev);
    s->st.force_evals++;
  } else {
    memcpy(s->a, atrial, b3);
    s->fprev.n = 0;
    for (int k = 0; k < ftrial.n; ++k) pl_push(&s->fprev, ftrial.ij[2 * k], ftrial.ij[2 * k + 1]);
  }
  free(atrial);
  free(ftrial.ij);
  free(E.ij);
  free(xs);
  free(vs);
  if (status) return status;
  momentum_drift(s, 0.5 * h);
  kick(s, 0.5 * h);
  if (p->gas) {
    int gs = gas_drag(s, 0.5 * h);
    if (gs) return gs;
  }
  s->step_index++;
  s->st.steps++;
  return NBREF_OK;
}

int nbref_step(nbref_system* s, int nsteps, double dt) {
  if (!s || nsteps < 0 || bad(dt)) return NBREF_E_INVALID;
  s->nlog = 0;
  for (int k = 0; k < nsteps; ++k) {
    int st = one_step(s, dt);
    if (st) return st;
  }
  return NBREF_OK;
}

/* Neumaier-compensated sum */
typedef struct {
  double s, c;
} csum;
static void cs_add(csum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

/* E = H_A + H_B + H_C (Eqs. Ha, Hb, Hc): K cancels between the close part
 * of H_A and H_B, leaving the Newtonian pair sum. */
int nbref_energy_momentum(const nbref_system* s, double* E, double L[3], double P[3],
                          double* E_lost) {
  const nbref_params* p = &s->p;
  int n = s->n;
  csum e = {0, 0}, l[3] = {{0, 0}, {0, 0}, {0, 0}}, pp[3] = {{0, 0}, {0, 0}, {0, 0}};
  double* pairsum = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    if (!s->alive[i]) continue;
    csum ci = {0, 0};
    for (int j = i + 1; j < n; ++j) {
      if (!s->alive[j]) continue;
      double dx = s->x[3 * j] - s->x[3 * i];
      double dy = s->x[3 * j + 1] - s->x[3 * i + 1];
      double dz = s->x[3 * j + 2] - s->x[3 * i + 2];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      cs_add(&ci, -p->G * s->m[i] * s->m[j] / r);
    }
    pairsum[i] = ci.s + ci.c;
  }
  for (int i = 0; i < n; ++i) {
    if (!s->alive[i]) continue;
    const double* x = s->x + 3 * i;
    const double* v = s->v + 3 * i;
    double mi = s->m[i];
    cs_add(&e, body_energy(p, x, v, mi));
    cs_add(&e, pairsum[i]);
    cs_add(&l[0], mi * (x[1] * v[2] - x[2] * v[1]));
    cs_add(&l[1], mi * (x[2] * v[0] - x[0] * v[2]));
    cs_add(&l[2], mi * (x[0] * v[1] - x[1] * v[0]));
    for (int k = 0; k < 3; ++k) cs_add(&pp[k], mi * v[k]);
  }
  free(pairsum);
  double Pv[3];
  for (int k = 0; k < 3; ++k) Pv[k] = pp[k].s + pp[k].c;
  cs_add(&e, (Pv[0] * Pv[0] + Pv[1] * Pv[1] + Pv[2] * Pv[2]) / (2.0 * p->m0));
  *E = e.s + e.c;
  for (int k = 0; k < 3; ++k) {
    L[k] = l[k].s + l[k].c;
    P[k] = Pv[k];
  }
  *E_lost = s->E_lost;
  return NBREF_OK;
}

int nbref_n_active(const nbref_system* s) {
  int c = 0;
  for (int i = 0; i < s->n; ++i) c += s->alive[i] ? 1 : 0;
  return c;
}

int nbref_get_state(const nbref_system* s, double* x, double* v, double* m, double* R,
                    double* rc, int* ids, int* n_active) {
  int c = 0;
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) {
      if (x) x[3 * c + k] = s->x[3 * i + k];
      if (v) v[3 * c + k] = s->v[3 * i + k];
    }
    if (m) m[c] = s->m[i];
    if (R) R[c] = s->R[i];
    if (rc) rc[c] = s->rc[i];
    if (ids) ids[c] = s->id[i];
    c++;
  }
  *n_active = c;
  return NBREF_OK;
}

int nbref_get_accel(const nbref_system* s, double* a) {
  int c = 0;
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int k = 0; k < 3; ++k) a[3 * c + k] = s->a[3 * i + k];
    c++;
  }
  return NBREF_OK;
}

int nbref_encounter_list(const nbref_system* s, int* step_ij, int cap, int* count) {
  *count = s->nlog;
  for (int k = 0; k < s->nlog && k < cap; ++k)
    for (int q = 0; q < 3; ++q) step_ij[3 * k + q] = s->log[3 * k + q];
  return NBREF_OK;
}

int nbref_stats_get(const nbref_system* s, nbref_stats* st) {
  *st = s->st;
  return NBREF_OK;
}

long long nbref_step_index(const nbref_system* s) { return s->step_index; }

void nbref_destroy(nbref_system* s) {
  if (!s) return;
  free(s->x); free(s->v); free(s->a); free(s->m); free(s->R); free(s->rc);
  free(s->id); free(s->alive); free(s->fprev.ij); free(s->log);
  free(s);
}

void nbref_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
