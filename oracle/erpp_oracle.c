/*
 * erpp_oracle.c -- plain, slow FP64 CPU oracle of the ERPP two-way coupling
 * step (Gualtieri, Picano, Sardina & Casciola, "Exact regularized point
 * particle method for multi-phase flows in the two-way coupling regime").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the timed
 * CPU baseline of the benchmark load this library.  It shares no code, header
 * or constant with the CUDA library: it is written independently from the
 * paper so that the two can be compared.  Compile with -ffp-contract=off so
 * that every product and sum is rounded exactly as written.
 *
 * Everything is double precision, in plain loops, particles in index order.
 *
 * Notation (nodes x_j = j * dx_a, j = 0..N_a-1 per axis, periodic box
 * [0, L_a), dx_a = L_a / N_a, dV = dx dy dz):
 *   sigma_R   = sqrt(2 nu eps_R)        regularisation width (Sec. 2.3)
 *   r_c       = cutoff * sigma_R         stencil radius (Sec. 3.1 uses 3 sigma_R)
 *   s         = x_p * (N_a / L_a)        particle position in grid units
 *   window    j_lo = ceil(s - r_c/dx) .. j_hi = floor(s + r_c/dx): every
 *             node whose signed distance d_j = (j - s) dx obeys |d_j| <= r_c.
 *             Node indices wrap modulo N_a; d_j is taken from the unwrapped j.
 *   w_a(j)    = (2 pi sigma_R^2)^(-1/2) exp(-d_j^2 / (2 sigma_R^2)): the heat
 *             kernel of App. A.1 (Eq. fundamental_phys) at t = eps_R,
 *             factored per axis.
 *   normalised weights w~_a(j) = w_a(j) / (dx_a sum_window w_a), so that the
 *             discrete kernel carries unit mass on every axis.
 *
 * Functions (each cites the passage it follows):
 *   orc_windows        stencil windows per particle and axis
 *   orc_scatter        S_j = -(1/rho_f) sum_p D_p W_p(j)          (Sec. 2.4, Eq. ns_regularized_filtered)
 *   orc_gather         u_p = sum_j dV W_p(j) u_j + shear y_p e_x   (matching kernel gather, Sec. 2.5)
 *   orc_self_velocity  closed-form regularised self disturbance    (App. A.5, Eq. disturbance_velo)
 *   orc_self_velocity_s2  the same at a given variance s2 (a point-value gather
 *                      sees it at 2 nu (eps_R + dt), without the gather's sigma_R^2)
 *   orc_advance        self removal, Stokes drag, explicit Euler   (Sec. 2.5, Eqs. particle_motion, force_stokes_drag)
 *   orc_step           gather + advance + scatter                  (Sec. 2.4-2.5)
 *   orc_momentum       grid and particle momentum of the source   (impulse, Sec. 3.1)
 *   orc_scatter_backward / orc_gather_backward  adjoints of scatter and gather
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n[3];          /* nx, ny, nz                                     */
  int32_t normalize;     /* 1: per-axis normalised weights                 */
  int32_t self_removal;  /* 1: subtract the closed-form self disturbance   */
  int32_t untruncated;   /* 1: stencil radius 12 sigma_R, windows may wrap */
  double L[3];
  double nu, rho_f, eps_R, cutoff, dt;
  double gravity[3];
  double shear_rate;     /* mean flow shear_rate * y e_x added at particles */
} orc_params;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

typedef struct {
  int64_t n[3];
  double L[3], dx[3], inv_dx[3], cp[3];
  double sigR2, sigR, raw_norm, dV;
} orc_geom;

static const double ORC_PI = 3.14159265358979323846;

static int orc_geom_init(const orc_params* p, orc_geom* g) {
  if (!p) return ORC_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (p->n[a] < 1 || !(p->L[a] > 0.0)) return ORC_EINVAL;
  }
  if (!(p->nu > 0.0) || !(p->rho_f > 0.0) || !(p->eps_R > 0.0) || !(p->cutoff > 0.0))
    return ORC_EINVAL;
  g->sigR2 = (2.0 * p->nu) * p->eps_R;
  g->sigR = sqrt(g->sigR2);
  double rc = (p->untruncated ? 12.0 : p->cutoff) * g->sigR;
  g->raw_norm = 1.0 / sqrt(2.0 * ORC_PI * g->sigR2);
  g->dV = 1.0;
  for (int a = 0; a < 3; ++a) {
    g->n[a] = p->n[a];
    g->L[a] = p->L[a];
    g->inv_dx[a] = (double)p->n[a] / p->L[a];
    g->dx[a] = p->L[a] / (double)p->n[a];
    g->cp[a] = rc * g->inv_dx[a];
    g->dV = g->dV * g->dx[a];
    if (!p->untruncated && !(2.0 * rc < p->L[a])) return ORC_EINVAL;
  }
  return ORC_OK;
}

static int64_t orc_wrap_index(int64_t j, int64_t n) {
  int64_t r = j % n;
  return r < 0 ? r + n : r;
}

/* Window of one coordinate: every node j with |(j - s) dx| <= r_c. */
static void orc_window(const orc_geom* g, int a, double xa, int64_t* jlo, int64_t* jhi,
                       double* s_out) {
  double s = xa * g->inv_dx[a];
  *jlo = (int64_t)ceil(s - g->cp[a]);
  *jhi = (int64_t)floor(s + g->cp[a]);
  *s_out = s;
}

/* Weights of one axis over the window; returns their plain sum through
 * *sum_raw (unit-mass normalisation needs it) and leaves in w[] either the raw
 * or the normalised weights.  d[] receives the signed distances. */
static void orc_axis_weights(const orc_geom* g, int a, int normalize, double s, int64_t jlo,
                             int64_t jhi, double* w, double* d, double* mass_out) {
  int64_t m = jhi - jlo + 1;
  double sum = 0.0;
  for (int64_t k = 0; k < m; ++k) {
    double dj = ((double)(jlo + k) - s) * g->dx[a];
    double wk = g->raw_norm * exp(-(dj * dj) / (2.0 * g->sigR2));
    d[k] = dj;
    w[k] = wk;
    sum += wk;
  }
  double mass = g->dx[a] * sum; /* discrete mass of the raw kernel on this axis */
  if (normalize) {
    for (int64_t k = 0; k < m; ++k) w[k] = w[k] / mass;
  }
  if (mass_out) *mass_out = normalize ? 1.0 : mass;
}

static int64_t orc_max_window(const orc_geom* g) {
  int64_t m = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t ma = (int64_t)floor(2.0 * g->cp[a]) + 2;
    if (ma > m) m = ma;
  }
  return m;
}

int orc_windows(const orc_params* p, int64_t np, const double* x, int32_t* jlo, int32_t* jhi) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  for (int64_t i = 0; i < np; ++i) {
    for (int a = 0; a < 3; ++a) {
      int64_t lo, hi;
      double s;
      orc_window(&g, a, x[(size_t)a * np + i], &lo, &hi, &s);
      jlo[(size_t)a * np + i] = (int32_t)lo;
      jhi[(size_t)a * np + i] = (int32_t)hi;
    }
  }
  return ORC_OK;
}

/* Per-particle stencil: windows, weights (raw or normalised), distances. */
typedef struct {
  int64_t jlo[3], m[3];
  double* w[3];
  double* d[3];
  double s[3];
  double mass; /* M_p = prod_a (dx_a sum w_a), 1 when normalised */
} orc_stencil;

static int orc_stencil_alloc(orc_stencil* st, int64_t mmax) {
  for (int a = 0; a < 3; ++a) {
    st->w[a] = (double*)malloc(sizeof(double) * (size_t)mmax);
    st->d[a] = (double*)malloc(sizeof(double) * (size_t)mmax);
    if (!st->w[a] || !st->d[a]) return ORC_ENOMEM;
  }
  return ORC_OK;
}

static void orc_stencil_free(orc_stencil* st) {
  for (int a = 0; a < 3; ++a) {
    free(st->w[a]);
    free(st->d[a]);
  }
}

static void orc_stencil_build(const orc_geom* g, int normalize, const double* x, int64_t np,
                              int64_t i, orc_stencil* st) {
  st->mass = 1.0;
  for (int a = 0; a < 3; ++a) {
    int64_t lo, hi;
    double s, mass_a;
    orc_window(g, a, x[(size_t)a * np + i], &lo, &hi, &s);
    st->jlo[a] = lo;
    st->m[a] = hi - lo + 1;
    st->s[a] = s;
    orc_axis_weights(g, a, normalize, s, lo, hi, st->w[a], st->d[a], &mass_a);
    st->mass = st->mass * mass_a;
  }
}

static size_t orc_node(const orc_geom* g, int64_t jx, int64_t jy, int64_t jz) {
  int64_t ix = orc_wrap_index(jx, g->n[0]);
  int64_t iy = orc_wrap_index(jy, g->n[1]);
  int64_t iz = orc_wrap_index(jz, g->n[2]);
  return ((size_t)iz * (size_t)g->n[1] + (size_t)iy) * (size_t)g->n[0] + (size_t)ix;
}

/* Eq. ns_regularized_filtered: the source added to the momentum equation is
 * -(1/rho_f) sum_p D_p g(x - x_p, eps_R); on the grid, with the separable
 * truncated kernel, S_j = -(1/rho_f) sum_p D_p prod_a w_a(j_a).  S is
 * overwritten. */
int orc_scatter(const orc_params* p, int64_t np, const double* x, const double* D, double* S) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  size_t nn = (size_t)g.n[0] * (size_t)g.n[1] * (size_t)g.n[2];
  memset(S, 0, sizeof(double) * 3 * nn);
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, orc_max_window(&g))) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  double inv_rho = 1.0 / p->rho_f;
  for (int64_t i = 0; i < np; ++i) {
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    double f[3];
    for (int c = 0; c < 3; ++c) f[c] = -inv_rho * D[(size_t)c * np + i];
    for (int64_t kz = 0; kz < sc.m[2]; ++kz)
      for (int64_t ky = 0; ky < sc.m[1]; ++ky)
        for (int64_t kx = 0; kx < sc.m[0]; ++kx) {
          double W = sc.w[0][kx] * sc.w[1][ky] * sc.w[2][kz];
          size_t j = orc_node(&g, sc.jlo[0] + kx, sc.jlo[1] + ky, sc.jlo[2] + kz);
          for (int c = 0; c < 3; ++c) S[(size_t)c * nn + j] += f[c] * W;
        }
  }
  orc_stencil_free(&sc);
  return ORC_OK;
}

/* Matching kernel gather: the same truncated kernel, integrated against the
 * grid field, u_p = sum_j dV W_p(j) u_j, plus the analytic mean shear
 * shear_rate * y_p along x.  (The paper leaves the interpolation operator
 * open; this is the transpose of the scatter up to -dV/rho_f.) */
int orc_gather(const orc_params* p, int64_t np, const double* x, const double* u, double* up) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  size_t nn = (size_t)g.n[0] * (size_t)g.n[1] * (size_t)g.n[2];
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, orc_max_window(&g))) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  for (int64_t i = 0; i < np; ++i) {
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t kz = 0; kz < sc.m[2]; ++kz)
      for (int64_t ky = 0; ky < sc.m[1]; ++ky)
        for (int64_t kx = 0; kx < sc.m[0]; ++kx) {
          double W = g.dV * (sc.w[0][kx] * sc.w[1][ky] * sc.w[2][kz]);
          size_t j = orc_node(&g, sc.jlo[0] + kx, sc.jlo[1] + ky, sc.jlo[2] + kz);
          for (int c = 0; c < 3; ++c) acc[c] += W * u[(size_t)c * nn + j];
        }
    up[i] = acc[0] + p->shear_rate * x[(size_t)1 * np + i];
    up[(size_t)np + i] = acc[1];
    up[(size_t)2 * np + i] = acc[2];
  }
  orc_stencil_free(&sc);
  return ORC_OK;
}

/* F(eta) = f(eta) / (2 eta^3), f(eta) = (sqrt(pi)/2) erf(eta) - eta exp(-eta^2)
 * (App. A.5).  For small eta the two terms of f cancel; there the Taylor
 * series F = sum_k (-1)^k eta^(2k) / (k! (2k+3)) is summed instead (it
 * follows from the series of erf and of exp term by term). */
static double orc_F(double eta) {
  if (eta < 0.5) {
    double e2 = eta * eta, term = 1.0, sum = 0.0;
    for (int k = 0; k < 20; ++k) {
      /* term = (-1)^k eta^(2k) / k! */
      sum += term / (double)(2 * k + 3);
      term = -term * e2 / (double)(k + 1);
    }
    return sum;
  }
  double f = 0.5 * sqrt(ORC_PI) * erf(eta) - eta * exp(-eta * eta);
  return f / (2.0 * eta * eta * eta);
}

/* Closed-form disturbance of App. A.5 (Eq. disturbance_velo), with the
 * prefactor -dt/rho_f that Eq. pseudo_velo_num carries:
 *   v(r) = -(dt/rho_f) (2 pi s2)^(-3/2) { [e^(-eta^2) - F] D - (D.rhat)[e^(-eta^2) - 3F] rhat },
 *   eta = |r| / sqrt(2 s2).
 * s2 is the variance of the disturbance as seen by the gather (below).
 * r [3][n] and D [3][n] in, out [3][n]. */
void orc_self_velocity_s2(const orc_params* p, double s2, int64_t n, const double* r,
                          const double* D, double* out) {
  double pref = -(p->dt / p->rho_f) / pow(2.0 * ORC_PI * s2, 1.5);
  for (int64_t i = 0; i < n; ++i) {
    double rv[3], Dv[3];
    for (int a = 0; a < 3; ++a) {
      rv[a] = r[(size_t)a * n + i];
      Dv[a] = D[(size_t)a * n + i];
    }
    double rr = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    double eta = rr / sqrt(2.0 * s2);
    double F = orc_F(eta);
    double e = exp(-eta * eta);
    double Ddotr = 0.0;
    double rh[3] = {0.0, 0.0, 0.0};
    if (rr > 0.0) {
      for (int a = 0; a < 3; ++a) rh[a] = rv[a] / rr;
      Ddotr = Dv[0] * rh[0] + Dv[1] * rh[1] + Dv[2] * rh[2];
    }
    for (int a = 0; a < 3; ++a)
      out[(size_t)a * n + i] = pref * ((e - F) * Dv[a] - Ddotr * (e - 3.0 * F) * rh[a]);
  }
}

/* The disturbance as the matching kernel gather sees it:
 *   s2 = 2 nu (eps_R + dt)  (forcing diffused one step, App. A.5)
 *      + sigma_R^2           (the kernel gather filters it once more). */
void orc_self_velocity(const orc_params* p, int64_t n, const double* r, const double* D,
                       double* out) {
  double s2 = (2.0 * p->nu) * (p->eps_R + p->dt) + (2.0 * p->nu) * p->eps_R;
  orc_self_velocity_s2(p, s2, n, r, D, out);
}

static double orc_min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

static double orc_wrap_coord(double x, double L) {
  if (x < 0.0) x = x + L;
  if (x >= L) x = x - L;
  return x;
}

/* Self-disturbance removal, Stokes drag and one explicit Euler step
 * (Sec. 2.5: Eq. particle_motion, Eq. force_stokes_drag and the removal of
 * v_R[x_p(t) - x_p(t - dt), dt] for an explicit Euler scheme).
 *
 * In:  up = fluid velocity gathered at x^n; x = x^n; v = v^n;
 *      x_prev = x^(n-1); D = D^(n-1) (ignored when first_step or when
 *      self removal is off).
 * Out: x = x^(n+1) (wrapped into [0, L)), v = v^(n+1), x_prev = x^n,
 *      D = D^n = 6 pi mu a (u~ - v^n), u~ = up - v_self.
 *   v^(n+1) = v^n + dt [D^n / m_p + (1 - rho_f/rho_p) g]
 *   x^(n+1) = x^n + dt v^n,   m_p = (4/3) pi a^3 rho_p.
 * Gravity and buoyancy act on the particle only; the fluid receives -D. */
int orc_advance(const orc_params* p, int64_t np, const double* up, double* x, double* v,
                double* x_prev, double* D, const double* radius, const double* rho_p,
                int first_step) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  double mu = p->rho_f * p->nu;
  int remove = p->self_removal && !first_step;
  double* r = NULL;
  double* vs = NULL;
  if (remove) {
    r = (double*)malloc(sizeof(double) * 3 * (size_t)np);
    vs = (double*)malloc(sizeof(double) * 3 * (size_t)np);
    if ((!r || !vs) && np > 0) { free(r); free(vs); return ORC_ENOMEM; }
    for (int64_t i = 0; i < np; ++i)
      for (int a = 0; a < 3; ++a) {
        size_t k = (size_t)a * np + i;
        r[k] = orc_min_image(x[k] - x_prev[k], p->L[a]);
      }
    orc_self_velocity(p, np, r, D, vs);
  }
  for (int64_t i = 0; i < np; ++i) {
    double a_p = radius[i];
    double k_drag = 6.0 * ORC_PI * mu * a_p;
    double m_p = (4.0 / 3.0) * ORC_PI * a_p * a_p * a_p * rho_p[i];
    double buoy = 1.0 - p->rho_f / rho_p[i];
    for (int a = 0; a < 3; ++a) {
      size_t k = (size_t)a * np + i;
      double ut = up[k] - (remove ? vs[k] : 0.0);
      double Dn = k_drag * (ut - v[k]);
      double xn = x[k];
      double vn = v[k];
      v[k] = vn + p->dt * (Dn / m_p + buoy * p->gravity[a]);
      x[k] = orc_wrap_coord(xn + p->dt * vn, p->L[a]);
      x_prev[k] = xn;
      D[k] = Dn;
    }
  }
  free(r);
  free(vs);
  return ORC_OK;
}

/* One coupling step: gather at x^n, advance, scatter the new forces D^n at
 * x^n (stored in x_prev after the advance).  The source uses the force and
 * position of the same step (no eps_R history buffer). */
int orc_step(const orc_params* p, int64_t np, const double* u, double* x, double* v,
             double* x_prev, double* D, const double* radius, const double* rho_p,
             int first_step, double* S, double* up_out) {
  double* up = up_out;
  if (!up) {
    up = (double*)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    if (!up) return ORC_ENOMEM;
  }
  int st = orc_gather(p, np, x, u, up);
  if (!st) st = orc_advance(p, np, up, x, v, x_prev, D, radius, rho_p, first_step);
  if (!st) st = orc_scatter(p, np, x_prev, D, S);
  if (!up_out) free(up);
  return st;
}

/* Momentum of the source: out[0..2] = dV sum_j S_j (grid), out[3..5] =
 * -(1/rho_f) sum_p M_p D_p (particles), M_p the discrete kernel mass (1 with
 * normalised weights).  Equal up to rounding: the momentum handed to the
 * fluid is the impulse of the particle forces (Sec. 3.1). */
int orc_momentum(const orc_params* p, int64_t np, const double* x, const double* D,
                 const double* S, double* out) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  size_t nn = (size_t)g.n[0] * (size_t)g.n[1] * (size_t)g.n[2];
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (size_t j = 0; j < nn; ++j) s += S[(size_t)c * nn + j];
    out[c] = g.dV * s;
  }
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, orc_max_window(&g))) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < np; ++i) {
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    for (int c = 0; c < 3; ++c) acc[c] += sc.mass * D[(size_t)c * np + i];
  }
  for (int c = 0; c < 3; ++c) out[3 + c] = -acc[c] / p->rho_f;
  orc_stencil_free(&sc);
  return ORC_OK;
}

/* Derivative of the axis weights with respect to the particle coordinate.
 * Raw:        dw_j/dx_p = w_j d_j / sigma^2          (d_j = x_j - x_p)
 * Normalised: dw~_j/dx_p = w~_j (d_j - dx sum_k w~_k d_k) / sigma^2 */
static void orc_axis_dweights(const orc_geom* g, int a, int normalize, int64_t m,
                              const double* w, const double* d, double* dw) {
  double mean_d = 0.0;
  if (normalize) {
    for (int64_t k = 0; k < m; ++k) mean_d += w[k] * d[k];
    mean_d = g->dx[a] * mean_d;
  }
  for (int64_t k = 0; k < m; ++k) dw[k] = w[k] * (d[k] - mean_d) / g->sigR2;
}

/* Adjoint of the scatter for a cotangent R = dL/dS on the grid:
 *   dL/dD_pc = -(1/rho_f) sum_j R_jc W_p(j)
 *   dL/dx_pa = -(1/rho_f) sum_j (R_j . D_p) dW_p(j)/dx_pa
 * (stencil membership is held fixed; it is piecewise constant in x_p). */
int orc_scatter_backward(const orc_params* p, int64_t np, const double* x, const double* D,
                         const double* R, double* dD, double* dx) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  size_t nn = (size_t)g.n[0] * (size_t)g.n[1] * (size_t)g.n[2];
  int64_t mmax = orc_max_window(&g);
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, mmax)) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  double* dw[3];
  for (int a = 0; a < 3; ++a) dw[a] = (double*)malloc(sizeof(double) * (size_t)mmax);
  double inv_rho = 1.0 / p->rho_f;
  for (int64_t i = 0; i < np; ++i) {
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    for (int a = 0; a < 3; ++a) orc_axis_dweights(&g, a, p->normalize, sc.m[a], sc.w[a], sc.d[a], dw[a]);
    double Dp[3], gD[3] = {0, 0, 0}, gx[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) Dp[c] = D[(size_t)c * np + i];
    for (int64_t kz = 0; kz < sc.m[2]; ++kz)
      for (int64_t ky = 0; ky < sc.m[1]; ++ky)
        for (int64_t kx = 0; kx < sc.m[0]; ++kx) {
          size_t j = orc_node(&g, sc.jlo[0] + kx, sc.jlo[1] + ky, sc.jlo[2] + kz);
          double W = sc.w[0][kx] * sc.w[1][ky] * sc.w[2][kz];
          double RD = 0.0;
          for (int c = 0; c < 3; ++c) {
            double Rj = R[(size_t)c * nn + j];
            gD[c] += Rj * W;
            RD += Rj * Dp[c];
          }
          gx[0] += RD * (dw[0][kx] * sc.w[1][ky] * sc.w[2][kz]);
          gx[1] += RD * (sc.w[0][kx] * dw[1][ky] * sc.w[2][kz]);
          gx[2] += RD * (sc.w[0][kx] * sc.w[1][ky] * dw[2][kz]);
        }
    for (int c = 0; c < 3; ++c) {
      dD[(size_t)c * np + i] = -inv_rho * gD[c];
      dx[(size_t)c * np + i] = -inv_rho * gx[c];
    }
  }
  for (int a = 0; a < 3; ++a) free(dw[a]);
  orc_stencil_free(&sc);
  return ORC_OK;
}

/* Adjoint of the gather for a cotangent G = dL/du_p:
 *   dL/du_jc = sum_p dV W_p(j) G_pc        (du overwritten)
 *   dL/dx_pa = sum_j dV (u_j . G_p) dW_p(j)/dx_pa + [a = y] shear_rate G_px */
int orc_gather_backward(const orc_params* p, int64_t np, const double* x, const double* u,
                        const double* G, double* du, double* dx) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  size_t nn = (size_t)g.n[0] * (size_t)g.n[1] * (size_t)g.n[2];
  memset(du, 0, sizeof(double) * 3 * nn);
  int64_t mmax = orc_max_window(&g);
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, mmax)) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  double* dw[3];
  for (int a = 0; a < 3; ++a) dw[a] = (double*)malloc(sizeof(double) * (size_t)mmax);
  for (int64_t i = 0; i < np; ++i) {
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    for (int a = 0; a < 3; ++a) orc_axis_dweights(&g, a, p->normalize, sc.m[a], sc.w[a], sc.d[a], dw[a]);
    double Gp[3], gx[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) Gp[c] = G[(size_t)c * np + i];
    for (int64_t kz = 0; kz < sc.m[2]; ++kz)
      for (int64_t ky = 0; ky < sc.m[1]; ++ky)
        for (int64_t kx = 0; kx < sc.m[0]; ++kx) {
          size_t j = orc_node(&g, sc.jlo[0] + kx, sc.jlo[1] + ky, sc.jlo[2] + kz);
          double W = g.dV * (sc.w[0][kx] * sc.w[1][ky] * sc.w[2][kz]);
          double uG = 0.0;
          for (int c = 0; c < 3; ++c) {
            du[(size_t)c * nn + j] += W * Gp[c];
            uG += u[(size_t)c * nn + j] * Gp[c];
          }
          gx[0] += uG * g.dV * (dw[0][kx] * sc.w[1][ky] * sc.w[2][kz]);
          gx[1] += uG * g.dV * (sc.w[0][kx] * dw[1][ky] * sc.w[2][kz]);
          gx[2] += uG * g.dV * (sc.w[0][kx] * sc.w[1][ky] * dw[2][kz]);
        }
    gx[1] += p->shear_rate * Gp[0];
    for (int c = 0; c < 3; ++c) dx[(size_t)c * np + i] = gx[c];
  }
  for (int a = 0; a < 3; ++a) free(dw[a]);
  orc_stencil_free(&sc);
  return ORC_OK;
}

/* The source of Eq. ns_regularized_filtered at selected nodes only:
 * out[c][k] = -(1/rho_f) sum_p D_p prod_a w_a(j_a) for the nodes
 * nodes[k] = (jx, jy, jz), summed over every particle whose window contains
 * the node (after wrapping).  Same arithmetic as orc_scatter, for grids too
 * large to hold in full. */
int orc_scatter_nodes(const orc_params* p, int64_t np, const double* x, const double* D,
                      int64_t nnodes, const int32_t* nodes, double* out) {
  orc_geom g;
  int st = orc_geom_init(p, &g);
  if (st) return st;
  for (int64_t k = 0; k < 3 * nnodes; ++k) out[k] = 0.0;
  orc_stencil sc;
  if (orc_stencil_alloc(&sc, orc_max_window(&g))) { orc_stencil_free(&sc); return ORC_ENOMEM; }
  double inv_rho = 1.0 / p->rho_f;
  for (int64_t i = 0; i < np; ++i) {
    int hit = 0;
    int64_t kk[3];
    for (int64_t k = 0; k < nnodes && !hit; ++k) {
      hit = 1;
      for (int a = 0; a < 3; ++a) {
        int64_t lo, hi;
        double s;
        orc_window(&g, a, x[(size_t)a * np + i], &lo, &hi, &s);
        int64_t j = nodes[(size_t)a * nnodes + k];
        int64_t rel = orc_wrap_index(j - lo, g.n[a]);
        if (rel > hi - lo) hit = 0;
      }
    }
    if (!hit) continue;
    orc_stencil_build(&g, p->normalize, x, np, i, &sc);
    for (int64_t k = 0; k < nnodes; ++k) {
      double W = 1.0;
      for (int a = 0; a < 3; ++a) {
        int64_t j = nodes[(size_t)a * nnodes + k];
        int64_t rel = orc_wrap_index(j - sc.jlo[a], g.n[a]);
        if (rel >= sc.m[a]) { W = 0.0; break; }
        kk[a] = rel;
      }
      if (W == 0.0) continue;
      W = sc.w[0][kk[0]] * sc.w[1][kk[1]] * sc.w[2][kk[2]];
      for (int c = 0; c < 3; ++c) out[(size_t)c * nnodes + k] += (-inv_rho * D[(size_t)c * np + i]) * W;
    }
  }
  orc_stencil_free(&sc);
  return ORC_OK;
}
