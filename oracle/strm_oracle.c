/*
 * FP64 CPU oracle: right-hand side of the compressible Navier-Stokes equations and
 * Wray's low-storage RK3, following STREAmS (arXiv 2004.02276) Section 2 step by step.
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against. Only the
 * tests, the smoke check and the benchmark's CPU baseline leg may load this library.
 * It is compiled with -ffp-contract=off and without fast-math.
 *
 * Order of one right-hand-side evaluation (Section 2.1):
 *   ghost fill of w  ->  primitives at every node  ->  Ducros sensor (Eq. sensor) at the
 *   interior, ghost fill of theta and of the node divergence  ->  per direction: interface
 *   flags, central energy-consistent flux (Eqs. avg_operator, encflux) or characteristic
 *   Lax-Friedrichs WENO5 flux, wall interfaces, flux difference (Eq. num_flux)  ->  viscous
 *   terms in Laplacian form (Section 2.1, last equation)  ->  mass-flow forcing (Eqs. 1b-c).
 * Time integration: Eq. RK with alpha = (0, -17/60, -5/12), beta = (8/15, 5/12, 3/4).
 *
 * Readings taken where the paper is silent or garbled (each repeated at its use):
 *   - RK alpha_1 is printed +17/60; only -17/60 is first-order consistent.
 *   - The viscous formula's first sum is garbled; it is read as (D1 mu)(D1 u) + mu (D2 u).
 *   - The sensor's u_0^2/L_0 is read as (u_0/L_0)^2 (dimensionally required).
 *   - Pressure enters the momentum flux through the same conservative central form.
 *   - WENO is used at interface i+1/2 iff max theta over nodes i-L+1..i+L exceeds the threshold.
 *   - Staggered isothermal wall: mirrored ghosts, zero convective flux of mass, x/z momentum
 *     and energy through the wall interface.
 *   - Forcing is applied at every RK stage; the CFL step uses the convective limit only.
 *   - Characteristic (non-reflecting) faces, Section 3.2: ghost states from the eigenvectors at
 *     the boundary node; outgoing characteristic variables extrapolated at zeroth order,
 *     incoming ones taken from a reference state: at the top face the free stream (or the
 *     post-shock state), at an outflow face the boundary node's own state at the reference
 *     pressure (a subsonic outflow only prescribes the far-field pressure; the outflow plane
 *     crosses the boundary layer, where the free-stream state is not a valid reference).
 *   - Inflow: rescaled recycling (the paper's digital filtering needs a Reynolds-stress
 *     dataset): ghost planes copy planes upstream of a recycling plane with the wall-normal
 *     coordinate stretched by delta_r / delta_in (outer scaling only).
 *   - Oblique shock at the top, Section 3.3: top ghosts downstream of the shock foot see the
 *     weak-branch Rankine-Hugoniot post-shock state.
 */
#include "strm_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define G 3 /* ghost layers: enough for L <= 3 and for the six-node WENO5 stencil */

typedef struct {
  const orc_cfg* c;
  int nx, ny, nz;
  ptrdiff_t nxg, nyg, nzg, ng;
  ptrdiff_t sx, sy, sz; /* strides along x, y, z in ghosted arrays */
  double dx, deta, dz;
  double* y;
  double* yeta;
  double* yetaeta;
  double cv, cp;
  double a[4], b[4]; /* central first- and second-derivative coefficients, index 1..L */
} grid_t;

typedef struct {
  double *rho, *u, *v, *w, *p, *T, *H, *c, *mu;
} prims_t;

int orc_ghosts(void) { return G; }

#ifdef _OPENMP
#include <omp.h>
int orc_set_threads(int n) {
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
}
#else
int orc_set_threads(int n) {
  (void)n;
  return 1;
}
#endif

static ptrdiff_t gidx(const grid_t* g, int i, int j, int k) {
  return ((ptrdiff_t)(k + G) * g->nyg + (ptrdiff_t)(j + G)) * g->nxg + (ptrdiff_t)(i + G);
}

static ptrdiff_t iidx(const grid_t* g, int i, int j, int k) {
  return ((ptrdiff_t)k * g->ny + j) * g->nx + i;
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Standard central coefficients of order 2L (Section 2.1): first derivative a_l and second
 * derivative b_l, with f'' ~ sum_l b_l (f_{i+l} - 2 f_i + f_{i-l}) / dx^2. */
static int central_coeffs(int L, double* a, double* b) {
  memset(a, 0, 4 * sizeof(double));
  memset(b, 0, 4 * sizeof(double));
  if (L == 3) {
    a[1] = 3.0 / 4.0; a[2] = -3.0 / 20.0; a[3] = 1.0 / 60.0;
    b[1] = 3.0 / 2.0; b[2] = -3.0 / 20.0; b[3] = 1.0 / 90.0;
    return 0;
  }
  if (L == 2) {
    a[1] = 2.0 / 3.0; a[2] = -1.0 / 12.0;
    b[1] = 4.0 / 3.0; b[2] = -1.0 / 12.0;
    return 0;
  }
  return -1;
}

/* Wall-normal mapping y(eta), eta in [0,1], nodes at eta_j = (j+1/2)/ny (staggered: the
 * walls eta = 0, 1 are interfaces). Clustering toward both walls, y in [-ly/2, ly/2]:
 * tanh, y = (ly/2) tanh(beta (2 eta - 1)) / tanh beta, or the error function of Section 3.1,
 * y = (ly/2) erf(beta (2 eta - 1)) / erf beta. Toward the wall y = 0 only, y in [0, ly]:
 * y = ly (1 - tanh(beta (1-eta)) / tanh beta), or the hyperbolic sine of Section 3.2,
 * y = ly sinh(beta eta) / sinh beta. The derivatives are the analytic ones. */
void orc_metrics(const orc_cfg* c, double* y, double* yeta, double* yetaeta) {
  for (int j = 0; j < c->ny; ++j) {
    double eta = (j + 0.5) / c->ny;
    if (c->y_map == ORC_MAP_TANH_ONESIDED) {
      double s = c->beta * (1.0 - eta);
      double th = tanh(s);
      double sech2 = 1.0 - th * th;
      double A = c->ly / tanh(c->beta);
      y[j] = c->ly - A * th;
      yeta[j] = A * c->beta * sech2;
      yetaeta[j] = 2.0 * A * c->beta * c->beta * sech2 * th;
    } else if (c->y_map == ORC_MAP_TANH) {
      double s = c->beta * (2.0 * eta - 1.0);
      double A = 0.5 * c->ly / tanh(c->beta);
      double th = tanh(s);
      double sech2 = 1.0 - th * th;
      y[j] = A * th;
      yeta[j] = 2.0 * c->beta * A * sech2;
      yetaeta[j] = -8.0 * c->beta * c->beta * A * sech2 * th;
    } else if (c->y_map == ORC_MAP_ERF) {
      double s = 2.0 * eta - 1.0;
      double E = erf(c->beta);
      y[j] = 0.5 * c->ly * erf(c->beta * s) / E;
      /* d/deta erf(beta s) = (2/sqrt(pi)) exp(-beta^2 s^2) * 2 beta */
      yeta[j] = 0.5 * c->ly / E * (2.0 / sqrt(acos(-1.0))) * exp(-c->beta * c->beta * s * s) * 2.0 * c->beta;
      yetaeta[j] = yeta[j] * (-2.0 * c->beta * c->beta * s) * 2.0;
    } else if (c->y_map == ORC_MAP_SINH_ONESIDED) {
      double S = sinh(c->beta);
      y[j] = c->ly * sinh(c->beta * eta) / S;
      yeta[j] = c->ly * c->beta * cosh(c->beta * eta) / S;
      yetaeta[j] = c->ly * c->beta * c->beta * sinh(c->beta * eta) / S;
    } else {
      y[j] = c->ly * (eta - 0.5);
      yeta[j] = c->ly;
      yetaeta[j] = 0.0;
    }
  }
}

/* Height of the wall-side boundary eta = 0 in the mapping. */
static double map_y0(const orc_cfg* c) {
  return (c->y_map == ORC_MAP_TANH_ONESIDED || c->y_map == ORC_MAP_SINH_ONESIDED) ? 0.0 : -0.5 * c->ly;
}

static int grid_init(grid_t* g, const orc_cfg* c) {
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return -1;
  if ((c->bc_ymin == ORC_BC_WALL || c->bc_ymax == ORC_BC_WALL) && c->ny < G) return -1;
  if ((c->bc_xmin == ORC_BC_PERIODIC) != (c->bc_xmax == ORC_BC_PERIODIC)) return -1;
  if ((c->bc_ymin == ORC_BC_PERIODIC) != (c->bc_ymax == ORC_BC_PERIODIC)) return -1;
  if (c->bc_xmax == ORC_BC_RECYCLE || c->bc_ymin == ORC_BC_RECYCLE || c->bc_ymax == ORC_BC_RECYCLE) return -1;
  if (c->bc_xmin == ORC_BC_RECYCLE && (c->i_recycle < G - 1 || c->i_recycle >= c->nx || !(c->delta_in > 0)))
    return -1;
  if (c->bc_xmax == ORC_BC_DF || c->bc_ymin == ORC_BC_DF || c->bc_ymax == ORC_BC_DF) return -1;
  if (c->bc_xmin == ORC_BC_DF && (!c->df_prof || !c->df_psi || !c->df_count || c->df_ny < 1 ||
                                  c->df_nz < 1 || !(c->df_tau > 0)))
    return -1;
  g->c = c;
  g->nx = c->nx; g->ny = c->ny; g->nz = c->nz;
  g->nxg = c->nx + 2 * G; g->nyg = c->ny + 2 * G; g->nzg = c->nz + 2 * G;
  g->ng = g->nxg * g->nyg * g->nzg;
  g->sx = 1; g->sy = g->nxg; g->sz = g->nxg * g->nyg;
  g->dx = c->lx / c->nx;
  g->deta = 1.0 / c->ny;
  g->dz = c->lz / c->nz;
  g->cv = c->r_gas / (c->gamma - 1.0);
  g->cp = c->gamma * c->r_gas / (c->gamma - 1.0);
  if (central_coeffs(c->L, g->a, g->b)) return -1;
  g->y = malloc(sizeof(double) * c->ny);
  g->yeta = malloc(sizeof(double) * c->ny);
  g->yetaeta = malloc(sizeof(double) * c->ny);
  orc_metrics(c, g->y, g->yeta, g->yetaeta);
  return 0;
}

static void grid_free(grid_t* g) {
  free(g->y); free(g->yeta); free(g->yetaeta);
}

static double* alloc_nan(ptrdiff_t n) {
  double* p = malloc(sizeof(double) * (size_t)n);
  for (ptrdiff_t q = 0; q < n; ++q) p[q] = NAN; /* unfilled corners stay NaN */
  return p;
}

/* Viscosity law: power law mu_ref (T/t_ref)^exp, or Sutherland (Section 2). */
static double viscosity(const orc_cfg* c, double T) {
  double tr = T / c->t_ref;
  if (c->visc_law == ORC_VISC_SUTHERLAND)
    return c->mu_ref * pow(tr, 1.5) * (1.0 + c->suth_s) / (tr + c->suth_s);
  return c->mu_ref * pow(tr, c->visc_exp);
}

/* ---------------------------------------------------------------- ghost fill of w */

static void load_interior(const grid_t* g, const double* w, double* wg[5]);

/* Isothermal no-slip wall on the staggered mesh: the ghost node mirrors an interior node
 * across the wall interface; velocity changes sign, T_g = 2 T_w - T, p_g = p, rho_g from the
 * equation of state, E from E = cv T + |u|^2/2. */
static void wall_ghost(const grid_t* g, const double* win, double* wout) {
  const orc_cfg* c = g->c;
  double rho = win[0];
  double u = win[1] / rho, v = win[2] / rho, w = win[3] / rho;
  double E = win[4] / rho;
  double T = (E - 0.5 * (u * u + v * v + w * w)) / g->cv;
  double p = rho * c->r_gas * T;
  double Tg = 2.0 * c->t_wall - T;
  double pg = p;
  double rhog = pg / (c->r_gas * Tg);
  double ug = -u, vg = -v, wg = -w;
  wout[0] = rhog;
  wout[1] = rhog * ug;
  wout[2] = rhog * vg;
  wout[3] = rhog * wg;
  wout[4] = rhog * (g->cv * Tg + 0.5 * (ug * ug + vg * vg + wg * wg));
}

/* Conserved state from primitives (rho, u, v, w, p): T = p/(rho R), E = cv T + |u|^2/2. */
static void prim_to_cons(const grid_t* g, const double* q, double* w) {
  double T = q[4] / (q[0] * g->c->r_gas);
  w[0] = q[0];
  w[1] = q[0] * q[1];
  w[2] = q[0] * q[2];
  w[3] = q[0] * q[3];
  w[4] = q[0] * (g->cv * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]));
}

/* Primitives (rho, u, v, w, p) and T from the conserved state. */
static void cons_to_prim(const grid_t* g, const double* w, double* q, double* T) {
  double rho = w[0];
  double u = w[1] / rho, v = w[2] / rho, ww = w[3] / rho;
  double t = (w[4] / rho - 0.5 * (u * u + v * v + ww * ww)) / g->cv;
  q[0] = rho;
  q[1] = u;
  q[2] = v;
  q[3] = ww;
  q[4] = rho * g->c->r_gas * t;
  *T = t;
}

/* Weak-branch oblique shock (Section 3.3): theta(beta) = atan(2 cot(beta) (M^2 sin^2 beta - 1) /
 * (M^2 (gamma + cos 2 beta) + 2)) rises from 0 at the Mach angle to its maximum and falls back to
 * 0 at 90 degrees; the weak solution is the root on the rising part (bisection), then the
 * normal-shock relations with M1n = M sin(beta). */
static double oblique_theta(double gamma, double M, double b) {
  double sb = sin(b);
  return atan(2.0 / tan(b) * (M * M * sb * sb - 1.0) / (M * M * (gamma + cos(2.0 * b)) + 2.0));
}

int orc_oblique_shock(double gamma, double M, double theta, double* beta, double* p_ratio,
                      double* rho_ratio, double* mach2) {
  double pi = acos(-1.0);
  double lo = asin(1.0 / M), hi = 0.5 * pi;
  /* maximum of theta(beta) by ternary search */
  for (int it = 0; it < 200; ++it) {
    double m1 = lo + (hi - lo) / 3.0, m2 = hi - (hi - lo) / 3.0;
    if (oblique_theta(gamma, M, m1) < oblique_theta(gamma, M, m2)) lo = m1;
    else hi = m2;
  }
  double bmax = 0.5 * (lo + hi);
  if (theta > oblique_theta(gamma, M, bmax)) return -1;
  lo = asin(1.0 / M);
  hi = bmax;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (oblique_theta(gamma, M, mid) < theta) lo = mid;
    else hi = mid;
  }
  double b = 0.5 * (lo + hi);
  double m1n = M * sin(b);
  *beta = b;
  *p_ratio = 1.0 + 2.0 * gamma / (gamma + 1.0) * (m1n * m1n - 1.0);
  *rho_ratio = (gamma + 1.0) * m1n * m1n / ((gamma - 1.0) * m1n * m1n + 2.0);
  double m2n2 = (m1n * m1n + 2.0 / (gamma - 1.0)) / (2.0 * gamma / (gamma - 1.0) * m1n * m1n - 1.0);
  *mach2 = sqrt(m2n2) / sin(b - theta);
  return 0;
}

/* Post-shock primitives behind the incident shock: the upstream reference stream (u along x)
 * deflected by theta toward the wall; x position of the shock foot on the top boundary. */
static void shock_state(const grid_t* g, double* q2, double* x_foot) {
  const orc_cfg* c = g->c;
  const double* q1 = c->ref;
  double V1 = q1[1];
  double c1 = sqrt(c->gamma * q1[4] / q1[0]);
  double b, pr, rr, m2;
  orc_oblique_shock(c->gamma, V1 / c1, c->shock_theta, &b, &pr, &rr, &m2);
  double un1 = V1 * sin(b), ut = V1 * cos(b);
  double un2 = un1 / rr;
  q2[0] = q1[0] * rr;
  q2[1] = ut * cos(b) + un2 * sin(b);
  q2[2] = -ut * sin(b) + un2 * cos(b);
  q2[3] = 0.0;
  q2[4] = q1[4] * pr;
  /* the shock line descends at angle beta from the foot (x_foot, top) to (x_imp, wall); the
   * wall (eta = 0) and the top (eta = 1) are ly apart */
  *x_foot = c->shock_ximp - c->ly / tan(b);
}

/* Non-reflecting characteristic ghost (Section 3.2: characteristic decomposition normal to the
 * boundary). Eigenvectors at the boundary node state wb along dir; a characteristic variable
 * whose speed points out of the domain (outward = +1 for the max face, -1 for the min face) is
 * extrapolated from the boundary node at zeroth order, the others are taken from the reference
 * primitives qref. */
static void char_ghost(const grid_t* g, const double* wb, const double* qref, int dir, int outward,
                       double* wout) {
  double q[5], T, wr[5], Lm[25], Rm[25], W[5];
  cons_to_prim(g, wb, q, &T);
  double H = (wb[4] + q[4]) / q[0];
  orc_eigvecs(dir, g->c->gamma, q[1], q[2], q[3], H, Lm, Rm);
  double cs = sqrt(g->c->gamma * q[4] / q[0]);
  double un = q[1 + dir];
  double lam[5] = {un - cs, un, un, un, un + cs};
  prim_to_cons(g, qref, wr);
  for (int k = 0; k < 5; ++k) {
    const double* src = (outward * lam[k] > 0.0) ? wb : wr;
    double s = 0.0;
    for (int m = 0; m < 5; ++m) s += Lm[k * 5 + m] * src[m];
    W[k] = s;
  }
  for (int m = 0; m < 5; ++m) {
    double s = 0.0;
    for (int k = 0; k < 5; ++k) s += Rm[m * 5 + k] * W[k];
    wout[m] = s;
  }
}

/* Spanwise-mean streamwise velocity at the recycling plane and the thickness delta_r where it
 * first reaches 0.99 of the reference velocity (linear interpolation between nodes; heights
 * above the wall eta = 0). Returns s = delta_r / delta_in (1 if the profile never reaches it). */
static double recycle_scale_g(const grid_t* g, double* const wg[5]) {
  const orc_cfg* c = g->c;
  double y0 = map_y0(c), target = 0.99 * c->ref[1];
  double prev_u = 0.0, prev_h = 0.0; /* the wall: u = 0 at height 0 */
  for (int j = 0; j < g->ny; ++j) {
    double sum = 0.0;
    for (int k = 0; k < g->nz; ++k) {
      ptrdiff_t n = gidx(g, c->i_recycle, j, k);
      sum += wg[1][n] / wg[0][n];
    }
    double ub = sum / g->nz, h = g->y[j] - y0;
    if (ub >= target) {
      double dr = prev_h + (target - prev_u) * (h - prev_h) / (ub - prev_u);
      return dr / c->delta_in;
    }
    prev_u = ub;
    prev_h = h;
  }
  return 1.0;
}

double orc_recycle_scale(const orc_cfg* c, const double* w) {
  grid_t g;
  if (grid_init(&g, c)) return -1.0;
  if (c->bc_xmin != ORC_BC_RECYCLE) {
    grid_free(&g);
    return 1.0;
  }
  double* wg[5];
  for (int m = 0; m < 5; ++m) wg[m] = alloc_nan(g.ng);
  load_interior(&g, w, wg);
  double s = recycle_scale_g(&g, wg);
  for (int m = 0; m < 5; ++m) free(wg[m]);
  grid_free(&g);
  return s;
}

/* Rescaled recycling inflow: ghost plane i = -1-q copies interior plane i_recycle - q with the
 * wall-normal coordinate stretched, the value at height h being the recycled plane's value at
 * height s*h (primitives u, v, w, T, p interpolated linearly between nodes; below the first node
 * between the wall state u = v = w = 0, T = T_w, p = p_0 and the first node; above the last node
 * the last node's value). */
static void fill_recycle(const grid_t* g, double* wg[5], double s) {
  const orc_cfg* c = g->c;
  double y0 = map_y0(c);
  for (int q = 0; q < G; ++q) {
    int is = c->i_recycle - q;
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j) {
        double ht = s * (g->y[j] - y0);
        double a[5], b[5], Ta, Tb, alpha;
        double wa[5], wb[5];
        int jb;
        for (jb = 0; jb < g->ny && g->y[jb] - y0 < ht; ++jb) {}
        if (jb == g->ny) {
          for (int m = 0; m < 5; ++m) wb[m] = wg[m][gidx(g, is, g->ny - 1, k)];
          cons_to_prim(g, wb, b, &Tb);
          for (int m = 0; m < 5; ++m) a[m] = b[m];
          Ta = Tb;
          alpha = 1.0;
        } else {
          for (int m = 0; m < 5; ++m) wb[m] = wg[m][gidx(g, is, jb, k)];
          cons_to_prim(g, wb, b, &Tb);
          double ha, hb = g->y[jb] - y0;
          if (jb == 0) {
            a[1] = a[2] = a[3] = 0.0;
            a[4] = b[4];
            Ta = c->t_wall;
            ha = 0.0;
          } else {
            for (int m = 0; m < 5; ++m) wa[m] = wg[m][gidx(g, is, jb - 1, k)];
            cons_to_prim(g, wa, a, &Ta);
            ha = g->y[jb - 1] - y0;
          }
          alpha = (ht - ha) / (hb - ha);
        }
        double qg[5];
        double Tg = (1.0 - alpha) * Ta + alpha * Tb;
        for (int m = 1; m < 5; ++m) qg[m] = (1.0 - alpha) * a[m] + alpha * b[m];
        qg[0] = qg[4] / (c->r_gas * Tg);
        double out[5];
        prim_to_cons(g, qg, out);
        for (int m = 0; m < 5; ++m) wg[m][gidx(g, -1 - q, j, k)] = out[m];
      }
  }
}

/* ---------------------------------------------------------------- digital-filter inflow
 * Section 3.2 names the method (Klein et al. digital filter, extended to compressible flow by
 * the strong Reynolds analogy, the filter done as a sequence of one-dimensional convolutions)
 * without its formulas. Steps, as read from those methods:
 *  1. random numbers with zero mean and unit variance, r = sqrt(3) (2 u - 1), u uniform from
 *     SplitMix64, one per (draw, velocity component m, z index k, extended y index);
 *  2. a Gaussian-shaped filter b_l = exp(-pi l^2 / (2 n^2)) / sqrt(sum_l exp(-pi l^2 / n^2)),
 *     l = -2n..2n, applied along y (random plane extended by 2n on both sides), then along z
 *     (periodic);
 *  3. time correlation: Psi <- Psi exp(-pi dt / (2 tau)) + psi sqrt(1 - exp(-pi dt / tau)),
 *     once per time step with a fresh filtered plane psi;
 *  4. velocity fluctuations u'_i = a_ij Psi_j with a the Cholesky factor of the Reynolds stress
 *     tensor (R13 = R23 = 0);
 *  5. strong Reynolds analogy at constant pressure: cp T' + U u' = 0, p = ref p, rho = p/(R T).
 * Every ghost layer of the inflow face takes the same state. */

/* SplitMix64 (Steele, Lea, Flood 2014): output number k + 1 of the generator seeded with seed. */
static uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

unsigned long long orc_splitmix64(unsigned long long seed, unsigned long long k) {
  return (unsigned long long)splitmix64((uint64_t)seed, (uint64_t)k);
}

static double df_random(const orc_cfg* c, long long draw, int m, int k, int je) {
  uint64_t nye = (uint64_t)c->ny + 4 * (uint64_t)c->df_ny;
  uint64_t idx = (((uint64_t)draw * 3 + (uint64_t)m) * (uint64_t)c->nz + (uint64_t)k) * nye + (uint64_t)je;
  double u = (double)(splitmix64(c->df_seed, idx) >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(3.0) * (2.0 * u - 1.0);
}

static void df_coefs(int n, double* b) {
  int N = 2 * n;
  double s = 0.0;
  for (int l = -N; l <= N; ++l) {
    b[l + N] = exp(-acos(-1.0) * l * l / (2.0 * n * n));
    s += b[l + N] * b[l + N];
  }
  for (int l = -N; l <= N; ++l) b[l + N] /= sqrt(s);
}

int orc_df_plane(const orc_cfg* c, long long draw, double* psi) {
  int ny = c->ny, nz = c->nz, Ny = 2 * c->df_ny, Nz = 2 * c->df_nz;
  if (ny < 1 || nz < 1 || c->df_ny < 1 || c->df_nz < 1) return -1;
  double* by = malloc(sizeof(double) * (2 * Ny + 1));
  double* bz = malloc(sizeof(double) * (2 * Nz + 1));
  double* t = malloc(sizeof(double) * 3 * (size_t)nz * ny);
  df_coefs(c->df_ny, by);
  df_coefs(c->df_nz, bz);
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j) {
        double s = 0.0;
        for (int l = -Ny; l <= Ny; ++l) s += by[l + Ny] * df_random(c, draw, m, k, j + l + Ny);
        t[((size_t)m * nz + k) * ny + j] = s;
      }
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j) {
        double s = 0.0;
        for (int l = -Nz; l <= Nz; ++l) s += bz[l + Nz] * t[((size_t)m * nz + wrap(k + l, nz)) * ny + j];
        psi[((size_t)m * nz + k) * ny + j] = s;
      }
  free(by);
  free(bz);
  free(t);
  return 0;
}

int orc_df_init(const orc_cfg* c) {
  if (c->bc_xmin != ORC_BC_DF || !c->df_psi || !c->df_count) return -1;
  if (orc_df_plane(c, 0, c->df_psi)) return -1;
  *c->df_count = 1;
  return 0;
}

/* Step 3: blend a fresh filtered plane into the time-correlated one. */
static void df_advance(const orc_cfg* c, double dt) {
  size_t n = 3 * (size_t)c->nz * c->ny;
  double* psi = malloc(sizeof(double) * n);
  orc_df_plane(c, *c->df_count, psi);
  double pi = acos(-1.0);
  double e1 = exp(-pi * dt / (2.0 * c->df_tau)), e2 = sqrt(1.0 - exp(-pi * dt / c->df_tau));
  for (size_t q = 0; q < n; ++q) c->df_psi[q] = c->df_psi[q] * e1 + psi[q] * e2;
  *c->df_count += 1;
  free(psi);
}

/* Steps 4 and 5: the inflow ghost layers from the mean profiles and the fluctuation plane. */
static void fill_df(const grid_t* g, double* wg[5]) {
  const orc_cfg* c = g->c;
  int ny = g->ny, nz = g->nz;
  const double* P = c->df_prof;
  double cp = g->cv + c->r_gas;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      double U = P[j], V = P[ny + j], Tm = P[2 * ny + j];
      double R11 = P[3 * ny + j], R12 = P[4 * ny + j], R22 = P[5 * ny + j], R33 = P[6 * ny + j];
      double a11 = sqrt(R11);
      double a21 = a11 > 0.0 ? R12 / a11 : 0.0;
      double a22 = sqrt(fmax(R22 - a21 * a21, 0.0));
      double a33 = sqrt(R33);
      const double* ps = c->df_psi;
      double p0 = ps[((size_t)0 * nz + k) * ny + j], p1 = ps[((size_t)1 * nz + k) * ny + j],
             p2 = ps[((size_t)2 * nz + k) * ny + j];
      double up = a11 * p0, vp = a21 * p0 + a22 * p1, wp = a33 * p2;
      double T = Tm - U * up / cp;
      double q[5] = {c->ref[4] / (c->r_gas * T), U + up, V + vp, wp, c->ref[4]};
      double out[5];
      prim_to_cons(g, q, out);
      for (int l = 1; l <= G; ++l)
        for (int m = 0; m < 5; ++m) wg[m][gidx(g, -l, j, k)] = out[m];
    }
}

/* Fill the ghost layers of the five ghosted conserved arrays face by face. Only the faces are
 * filled (no edges or corners): every stencil of the method runs along one grid line. */
static void fill_ghosts_w(const grid_t* g, double* wg[5]) {
  const orc_cfg* c = g->c;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  /* periodic faces */
  for (int m = 0; m < 5; ++m) {
    double* f = wg[m];
    if (c->bc_xmin == ORC_BC_PERIODIC)
      for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
          for (int q = 1; q <= G; ++q) {
            f[gidx(g, -q, j, k)] = f[gidx(g, wrap(-q, nx), j, k)];
            f[gidx(g, nx - 1 + q, j, k)] = f[gidx(g, wrap(nx - 1 + q, nx), j, k)];
          }
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int q = 1; q <= G; ++q) {
          f[gidx(g, i, j, -q)] = f[gidx(g, i, j, wrap(-q, nz))];
          f[gidx(g, i, j, nz - 1 + q)] = f[gidx(g, i, j, wrap(nz - 1 + q, nz))];
        }
    if (c->bc_ymin == ORC_BC_PERIODIC)
      for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i)
          for (int q = 1; q <= G; ++q) {
            f[gidx(g, i, -q, k)] = f[gidx(g, i, wrap(-q, ny), k)];
            f[gidx(g, i, ny - 1 + q, k)] = f[gidx(g, i, wrap(ny - 1 + q, ny), k)];
          }
  }
  double in[5], out[5];
  /* x faces (outflow-type characteristic faces see the boundary state at the reference
   * pressure) */
  if (c->bc_xmin == ORC_BC_RECYCLE) fill_recycle(g, wg, recycle_scale_g(g, wg));
  if (c->bc_xmin == ORC_BC_DF) fill_df(g, wg);
  if (c->bc_xmin == ORC_BC_CHAR || c->bc_xmax == ORC_BC_CHAR)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int side = 0; side < 2; ++side) {
          if ((side == 0 ? c->bc_xmin : c->bc_xmax) != ORC_BC_CHAR) continue;
          int ib = side == 0 ? 0 : nx - 1;
          double qb[5], Tb;
          for (int m = 0; m < 5; ++m) in[m] = wg[m][gidx(g, ib, j, k)];
          cons_to_prim(g, in, qb, &Tb);
          qb[4] = c->ref[4];
          char_ghost(g, in, qb, 0, side == 0 ? -1 : 1, out);
          for (int q = 1; q <= G; ++q)
            for (int m = 0; m < 5; ++m) wg[m][gidx(g, side == 0 ? -q : nx - 1 + q, j, k)] = out[m];
        }
  /* y faces: walls mirror, characteristic faces from the boundary row */
  double qshock[5], x_foot = 0.0;
  if (c->shock) shock_state(g, qshock, &x_foot);
  for (int k = 0; k < nz; ++k)
    for (int i = 0; i < nx; ++i) {
      for (int q = 0; q < G; ++q) {
        if (c->bc_ymin == ORC_BC_WALL) { /* ghost j = -1-q mirrors j = q */
          for (int m = 0; m < 5; ++m) in[m] = wg[m][gidx(g, i, q, k)];
          wall_ghost(g, in, out);
          for (int m = 0; m < 5; ++m) wg[m][gidx(g, i, -1 - q, k)] = out[m];
        }
        if (c->bc_ymax == ORC_BC_WALL) { /* ghost j = ny+q mirrors j = ny-1-q */
          for (int m = 0; m < 5; ++m) in[m] = wg[m][gidx(g, i, ny - 1 - q, k)];
          wall_ghost(g, in, out);
          for (int m = 0; m < 5; ++m) wg[m][gidx(g, i, ny + q, k)] = out[m];
        }
      }
      if (c->bc_ymin == ORC_BC_CHAR) {
        for (int m = 0; m < 5; ++m) in[m] = wg[m][gidx(g, i, 0, k)];
        char_ghost(g, in, c->ref, 1, -1, out);
        for (int q = 1; q <= G; ++q)
          for (int m = 0; m < 5; ++m) wg[m][gidx(g, i, -q, k)] = out[m];
      }
      if (c->bc_ymax == ORC_BC_CHAR) {
        double xi = (i + 0.5) * g->dx;
        const double* qr = (c->shock && xi >= x_foot) ? qshock : c->ref;
        for (int m = 0; m < 5; ++m) in[m] = wg[m][gidx(g, i, ny - 1, k)];
        char_ghost(g, in, qr, 1, 1, out);
        for (int q = 1; q <= G; ++q)
          for (int m = 0; m < 5; ++m) wg[m][gidx(g, i, ny - 1 + q, k)] = out[m];
      }
    }
}

/* Ghost fill of a node scalar (sensor theta, node divergence): periodic copy, even mirror across
 * a wall, copy of the boundary node at characteristic and inflow faces. */
static void fill_ghosts_scalar(const grid_t* g, double* f) {
  const orc_cfg* c = g->c;
  int nx = g->nx, ny = g->ny, nz = g->nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int q = 1; q <= G; ++q) {
        int lo = c->bc_xmin == ORC_BC_PERIODIC ? wrap(-q, nx) : 0;
        int hi = c->bc_xmax == ORC_BC_PERIODIC ? wrap(nx - 1 + q, nx) : nx - 1;
        f[gidx(g, -q, j, k)] = f[gidx(g, lo, j, k)];
        f[gidx(g, nx - 1 + q, j, k)] = f[gidx(g, hi, j, k)];
      }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int q = 1; q <= G; ++q) {
        f[gidx(g, i, j, -q)] = f[gidx(g, i, j, wrap(-q, nz))];
        f[gidx(g, i, j, nz - 1 + q)] = f[gidx(g, i, j, wrap(nz - 1 + q, nz))];
      }
  for (int k = 0; k < nz; ++k)
    for (int i = 0; i < nx; ++i)
      for (int q = 0; q < G; ++q) {
        int lo, hi;
        if (c->bc_ymin == ORC_BC_PERIODIC) lo = wrap(-1 - q, ny);
        else if (c->bc_ymin == ORC_BC_WALL) lo = q;
        else lo = 0;
        if (c->bc_ymax == ORC_BC_PERIODIC) hi = wrap(ny + q, ny);
        else if (c->bc_ymax == ORC_BC_WALL) hi = ny - 1 - q;
        else hi = ny - 1;
        f[gidx(g, i, -1 - q, k)] = f[gidx(g, i, lo, k)];
        f[gidx(g, i, ny + q, k)] = f[gidx(g, i, hi, k)];
      }
}

static void load_interior(const grid_t* g, const double* w, double* wg[5]) {
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i)
          wg[m][gidx(g, i, j, k)] = w[(ptrdiff_t)m * g->nx * g->ny * g->nz + iidx(g, i, j, k)];
}

/* ---------------------------------------------------------------- primitives */

/* Primitive variables at every node from w = [rho, rho u, rho v, rho w, rho E]:
 * E = cv T + |u|^2/2, p = rho R T, H = E + p/rho (Section 2), c = sqrt(gamma p / rho). */
static void primitives(const grid_t* g, double* const wg[5], prims_t* P) {
  const orc_cfg* c = g->c;
#pragma omp parallel for schedule(static)
  for (ptrdiff_t n = 0; n < g->ng; ++n) {
    double rho = wg[0][n];
    double u = wg[1][n] / rho, v = wg[2][n] / rho, w = wg[3][n] / rho;
    double E = wg[4][n] / rho;
    double T = (E - 0.5 * (u * u + v * v + w * w)) / g->cv;
    double p = rho * c->r_gas * T;
    P->rho[n] = rho;
    P->u[n] = u; P->v[n] = v; P->w[n] = w;
    P->T[n] = T;
    P->p[n] = p;
    P->H[n] = E + p / rho;
    P->c[n] = sqrt(c->gamma * p / rho);
    P->mu[n] = (T == T) ? viscosity(c, T) : NAN;
  }
}

static void prims_alloc(const grid_t* g, prims_t* P) {
  P->rho = alloc_nan(g->ng); P->u = alloc_nan(g->ng); P->v = alloc_nan(g->ng);
  P->w = alloc_nan(g->ng); P->p = alloc_nan(g->ng); P->T = alloc_nan(g->ng);
  P->H = alloc_nan(g->ng); P->c = alloc_nan(g->ng); P->mu = alloc_nan(g->ng);
}

static void prims_free(prims_t* P) {
  free(P->rho); free(P->u); free(P->v); free(P->w); free(P->p);
  free(P->T); free(P->H); free(P->c); free(P->mu);
}

/* ---------------------------------------------------------------- derivatives */

static ptrdiff_t dir_stride(const grid_t* g, int dir) {
  return dir == 0 ? g->sx : (dir == 1 ? g->sy : g->sz);
}

/* First derivative of order 2L at interior node (i,j,k) along dir, in physical space:
 * sum_l a_l (f_{+l} - f_{-l}) / h, with h = dx, y_eta(j) deta, dz. */
static double d1(const grid_t* g, const double* f, int i, int j, int k, int dir) {
  ptrdiff_t n = gidx(g, i, j, k), st = dir_stride(g, dir);
  double s = 0.0;
  for (int l = 1; l <= g->c->L; ++l) s += g->a[l] * (f[n + l * st] - f[n - l * st]);
  if (dir == 0) return s / g->dx;
  if (dir == 1) return s / (g->deta * g->yeta[j]);
  return s / g->dz;
}

/* Second derivative of order 2L along dir in physical space. Along y (stretched):
 * d2f/dy2 = (f_etaeta - (y_etaeta / y_eta) f_eta) / y_eta^2. */
static double d2(const grid_t* g, const double* f, int i, int j, int k, int dir) {
  ptrdiff_t n = gidx(g, i, j, k), st = dir_stride(g, dir);
  double s2 = 0.0, s1 = 0.0;
  for (int l = 1; l <= g->c->L; ++l) {
    s2 += g->b[l] * ((f[n + l * st] + f[n - l * st]) - 2.0 * f[n]);
    s1 += g->a[l] * (f[n + l * st] - f[n - l * st]);
  }
  if (dir == 0) return s2 / (g->dx * g->dx);
  if (dir == 2) return s2 / (g->dz * g->dz);
  double fee = s2 / (g->deta * g->deta);
  double fe = s1 / g->deta;
  double ye = g->yeta[j];
  return (fee - (g->yetaeta[j] / ye) * fe) / (ye * ye);
}

/* ---------------------------------------------------------------- sensor */

/* Ducros sensor (Eq. sensor) at the interior nodes, theta = max(-div / sqrt(div^2 +
 * |curl u|^2 + (u0/L0)^2), 0); the node divergence is kept for the viscous terms. Both are
 * then ghost filled. */
static void sensor(const grid_t* g, const prims_t* P, double* theta, double* divg) {
  const orc_cfg* c = g->c;
  double eps = (c->u0 / c->l0) * (c->u0 / c->l0);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double ux = d1(g, P->u, i, j, k, 0), uy = d1(g, P->u, i, j, k, 1), uz = d1(g, P->u, i, j, k, 2);
        double vx = d1(g, P->v, i, j, k, 0), vy = d1(g, P->v, i, j, k, 1), vz = d1(g, P->v, i, j, k, 2);
        double wx = d1(g, P->w, i, j, k, 0), wy = d1(g, P->w, i, j, k, 1), wz = d1(g, P->w, i, j, k, 2);
        double div = ux + vy + wz;
        double o1 = wy - vz, o2 = uz - wx, o3 = vx - uy;
        double curl2 = o1 * o1 + o2 * o2 + o3 * o3;
        double th = -div / sqrt(div * div + curl2 + eps);
        ptrdiff_t n = gidx(g, i, j, k);
        theta[n] = th > 0.0 ? th : 0.0;
        divg[n] = div;
      }
  if (c->theta_fixed) /* prescribed switch input replaces the computed sensor */
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) theta[gidx(g, i, j, k)] = c->theta_fixed[iidx(g, i, j, k)];
  fill_ghosts_scalar(g, theta);
  fill_ghosts_scalar(g, divg);
}

/* Hybrid switch: WENO at the interface between nodes (n) and (n + st) iff the largest theta
 * over nodes n-L+1 .. n+L exceeds the threshold (or WENO is forced everywhere). */
static int interface_flag(const grid_t* g, const double* theta, ptrdiff_t n, ptrdiff_t st) {
  const orc_cfg* c = g->c;
  if (c->weno_mode == ORC_WENO_ALL) return 1;
  if (c->weno_mode == ORC_WENO_OFF) return 0;
  double tmax = 0.0;
  for (int q = -c->L + 1; q <= c->L; ++q)
    if (theta[n + q * st] > tmax) tmax = theta[n + q * st];
  return tmax > c->theta_thr;
}

/* ---------------------------------------------------------------- fluxes */

/* Three-point averaging operator (Eq. avg_operator). */
static double tilde(double Fa, double Fb, double Ga, double Gb, double Ha, double Hb) {
  return 0.125 * (Fa + Fb) * (Ga + Gb) * (Ha + Hb);
}

/* Energy-consistent central flux at the interface between node n and n+st (Eq. encflux):
 * f = 2 sum_l a_l sum_{m<l} (rho, u_d, phi)~_{n-m, l}, phi = 1, u, v, w, H; the pressure is
 * added to the momentum component along dir as sum_l a_l sum_{m<l} (p_{n-m} + p_{n-m+l}). */
static void central_flux(const grid_t* g, const prims_t* P, ptrdiff_t n, ptrdiff_t st, int dir,
                         double* f) {
  const double* ud = dir == 0 ? P->u : (dir == 1 ? P->v : P->w);
  const double* rho = P->rho;
  double acc[5] = {0, 0, 0, 0, 0}, accp = 0.0;
  for (int l = 1; l <= g->c->L; ++l) {
    double s[5] = {0, 0, 0, 0, 0}, sp = 0.0;
    for (int m = 0; m < l; ++m) {
      ptrdiff_t a = n - m * st, b = n + (l - m) * st;
      s[0] += tilde(rho[a], rho[b], ud[a], ud[b], 1.0, 1.0);
      s[1] += tilde(rho[a], rho[b], ud[a], ud[b], P->u[a], P->u[b]);
      s[2] += tilde(rho[a], rho[b], ud[a], ud[b], P->v[a], P->v[b]);
      s[3] += tilde(rho[a], rho[b], ud[a], ud[b], P->w[a], P->w[b]);
      s[4] += tilde(rho[a], rho[b], ud[a], ud[b], P->H[a], P->H[b]);
      sp += P->p[a] + P->p[b];
    }
    for (int q = 0; q < 5; ++q) acc[q] += g->a[l] * s[q];
    accp += g->a[l] * sp;
  }
  for (int q = 0; q < 5; ++q) f[q] = 2.0 * acc[q];
  f[1 + dir] += accp;
}

/* Left (rows) and right (columns) eigenvectors of the Euler flux Jacobian along dir, in
 * conserved variables, eigenvalues (u_n - c, u_n, u_n, u_n, u_n + c). Textbook form with
 * b1 = (gamma-1)/c^2, b2 = b1 |u|^2 / 2; the two shear waves carry the tangential
 * velocities in increasing index order. */
void orc_eigvecs(int dir, double gamma, double u, double v, double w, double H, double* Lm,
                 double* Rm) {
  double vel[3] = {u, v, w};
  double q2 = u * u + v * v + w * w;
  double c = sqrt((gamma - 1.0) * (H - 0.5 * q2));
  double un = vel[dir];
  double b1 = (gamma - 1.0) / (c * c);
  double b2 = 0.5 * q2 * b1;
  int t1 = dir == 0 ? 1 : 0;
  int t2 = dir == 2 ? 1 : 2;
  double nrm[3] = {0, 0, 0};
  nrm[dir] = 1.0;
  for (int q = 0; q < 25; ++q) Lm[q] = Rm[q] = 0.0;
  /* right eigenvectors: column r of Rm is Rm[row*5 + r] */
  Rm[0 * 5 + 0] = 1.0;
  Rm[0 * 5 + 1] = 1.0;
  Rm[0 * 5 + 4] = 1.0;
  for (int d = 0; d < 3; ++d) {
    Rm[(1 + d) * 5 + 0] = vel[d] - c * nrm[d];
    Rm[(1 + d) * 5 + 1] = vel[d];
    Rm[(1 + d) * 5 + 4] = vel[d] + c * nrm[d];
  }
  Rm[4 * 5 + 0] = H - un * c;
  Rm[4 * 5 + 1] = 0.5 * q2;
  Rm[4 * 5 + 4] = H + un * c;
  Rm[(1 + t1) * 5 + 2] = 1.0;
  Rm[4 * 5 + 2] = vel[t1];
  Rm[(1 + t2) * 5 + 3] = 1.0;
  Rm[4 * 5 + 3] = vel[t2];
  /* left eigenvectors: row l of Lm is Lm[l*5 + col] */
  Lm[0 * 5 + 0] = 0.5 * (b2 + un / c);
  Lm[4 * 5 + 0] = 0.5 * (b2 - un / c);
  for (int d = 0; d < 3; ++d) {
    Lm[0 * 5 + 1 + d] = 0.5 * (-b1 * vel[d] - nrm[d] / c);
    Lm[4 * 5 + 1 + d] = 0.5 * (-b1 * vel[d] + nrm[d] / c);
    Lm[1 * 5 + 1 + d] = b1 * vel[d];
  }
  Lm[0 * 5 + 4] = 0.5 * b1;
  Lm[4 * 5 + 4] = 0.5 * b1;
  Lm[1 * 5 + 0] = 1.0 - b2;
  Lm[1 * 5 + 4] = -b1;
  Lm[2 * 5 + 0] = -vel[t1];
  Lm[2 * 5 + 1 + t1] = 1.0;
  Lm[3 * 5 + 0] = -vel[t2];
  Lm[3 * 5 + 1 + t2] = 1.0;
}

/* WENO5 reconstruction of Jiang and Shu at i+1/2 from f_{i-2..i+2} (left-biased). */
double orc_weno5(const double* f, double eps) {
  double fm2 = f[0], fm1 = f[1], f0 = f[2], fp1 = f[3], fp2 = f[4];
  double b0 = 13.0 / 12.0 * (fm2 - 2.0 * fm1 + f0) * (fm2 - 2.0 * fm1 + f0) +
              0.25 * (fm2 - 4.0 * fm1 + 3.0 * f0) * (fm2 - 4.0 * fm1 + 3.0 * f0);
  double b1 = 13.0 / 12.0 * (fm1 - 2.0 * f0 + fp1) * (fm1 - 2.0 * f0 + fp1) +
              0.25 * (fm1 - fp1) * (fm1 - fp1);
  double b2 = 13.0 / 12.0 * (f0 - 2.0 * fp1 + fp2) * (f0 - 2.0 * fp1 + fp2) +
              0.25 * (3.0 * f0 - 4.0 * fp1 + fp2) * (3.0 * f0 - 4.0 * fp1 + fp2);
  double a0 = 0.1 / ((eps + b0) * (eps + b0));
  double a1 = 0.6 / ((eps + b1) * (eps + b1));
  double a2 = 0.3 / ((eps + b2) * (eps + b2));
  double s = a0 + a1 + a2;
  double q0 = (2.0 * fm2 - 7.0 * fm1 + 11.0 * f0) / 6.0;
  double q1 = (-fm1 + 5.0 * f0 + 2.0 * fp1) / 6.0;
  double q2 = (2.0 * f0 + 5.0 * fp1 - fp2) / 6.0;
  return (a0 / s) * q0 + (a1 / s) * q1 + (a2 / s) * q2;
}

/* Characteristic Lax-Friedrichs flux-vector splitting with WENO5 reconstruction at the
 * interface between node n and n+st (Section 2.1): Roe-averaged eigenvectors, projection of
 * w and of the physical flux at nodes n-2..n+3, local LF speeds (largest |eigenvalue| over the
 * stencil), WENO5 of the positive part from the left and of the negative part from the right,
 * and projection back. */
static void weno_flux(const grid_t* g, const prims_t* P, double* const wg[5], ptrdiff_t n,
                      ptrdiff_t st, int dir, double* f) {
  const orc_cfg* c = g->c;
  const double* ud = dir == 0 ? P->u : (dir == 1 ? P->v : P->w);
  ptrdiff_t nl = n, nr = n + st;
  double sl = sqrt(P->rho[nl]), sr = sqrt(P->rho[nr]);
  double ur = (sl * P->u[nl] + sr * P->u[nr]) / (sl + sr);
  double vr = (sl * P->v[nl] + sr * P->v[nr]) / (sl + sr);
  double wr = (sl * P->w[nl] + sr * P->w[nr]) / (sl + sr);
  double Hr = (sl * P->H[nl] + sr * P->H[nr]) / (sl + sr);
  double Lm[25], Rm[25];
  orc_eigvecs(dir, c->gamma, ur, vr, wr, Hr, Lm, Rm);

  double cw[5][6], cf[5][6], lam[5] = {0, 0, 0, 0, 0};
  for (int q = 0; q < 6; ++q) {
    ptrdiff_t nn = n + (q - 2) * st;
    double wv[5], F[5];
    for (int m = 0; m < 5; ++m) wv[m] = wg[m][nn];
    double rho = P->rho[nn], un = ud[nn];
    F[0] = rho * un;
    F[1] = rho * un * P->u[nn];
    F[2] = rho * un * P->v[nn];
    F[3] = rho * un * P->w[nn];
    F[4] = rho * un * P->H[nn];
    F[1 + dir] += P->p[nn];
    for (int k = 0; k < 5; ++k) {
      double sw = 0.0, sf = 0.0;
      for (int m = 0; m < 5; ++m) {
        sw += Lm[k * 5 + m] * wv[m];
        sf += Lm[k * 5 + m] * F[m];
      }
      cw[k][q] = sw;
      cf[k][q] = sf;
    }
    double ev[5] = {un - P->c[nn], un, un, un, un + P->c[nn]};
    for (int k = 0; k < 5; ++k)
      if (fabs(ev[k]) > lam[k]) lam[k] = fabs(ev[k]);
  }
  double gh[5];
  for (int k = 0; k < 5; ++k) {
    double gp[6], gm[6];
    for (int q = 0; q < 6; ++q) {
      gp[q] = 0.5 * (cf[k][q] + lam[k] * cw[k][q]);
      gm[q] = 0.5 * (cf[k][q] - lam[k] * cw[k][q]);
    }
    double sp[5] = {gp[0], gp[1], gp[2], gp[3], gp[4]};         /* nodes n-2 .. n+2 */
    double sm[5] = {gm[5], gm[4], gm[3], gm[2], gm[1]};         /* nodes n+3 .. n-1 */
    gh[k] = orc_weno5(sp, c->weno_eps) + orc_weno5(sm, c->weno_eps);
  }
  for (int m = 0; m < 5; ++m) {
    double s = 0.0;
    for (int k = 0; k < 5; ++k) s += Rm[m * 5 + k] * gh[k];
    f[m] = s;
  }
}

/* Convective part of R along one direction: interface fluxes along every interior line,
 * the wall rule, and the conservative difference (Eq. num_flux) with the metric. */
static void convective_dir(const grid_t* g, const prims_t* P, double* const wg[5],
                           const double* theta, int dir, double* R, unsigned char* flags) {
  int nd = dir == 0 ? g->nx : (dir == 1 ? g->ny : g->nz);
  int na = dir == 0 ? g->ny : g->nx; /* first transverse */
  int nb = dir == 2 ? g->ny : g->nz; /* second transverse */
  ptrdiff_t st = dir_stride(g, dir);
  ptrdiff_t Nint = (ptrdiff_t)g->nx * g->ny * g->nz;
  int wall_lo = dir == 1 && g->c->bc_ymin == ORC_BC_WALL;
  int wall_hi = dir == 1 && g->c->bc_ymax == ORC_BC_WALL;
#pragma omp parallel for schedule(static)
  for (int b = 0; b < nb; ++b) {
    double* fl = malloc(sizeof(double) * 5 * (size_t)(nd + 1));
    for (int a = 0; a < na; ++a) {
      for (int s = 0; s <= nd; ++s) {
        /* interface s lies between nodes s-1 and s along dir */
        int i, j, k;
        if (dir == 0) { i = s - 1; j = a; k = b; }
        else if (dir == 1) { i = a; j = s - 1; k = b; }
        else { i = a; j = b; k = s - 1; }
        ptrdiff_t n = gidx(g, i, j, k);
        int fw = interface_flag(g, theta, n, st);
        if (flags) {
          ptrdiff_t fi;
          if (dir == 0) fi = ((ptrdiff_t)k * g->ny + j) * (g->nx + 1) + s;
          else if (dir == 1) fi = ((ptrdiff_t)k * (g->ny + 1) + s) * g->nx + i;
          else fi = ((ptrdiff_t)s * g->ny + j) * g->nx + i;
          flags[fi] = (unsigned char)fw;
        }
        if (fw) weno_flux(g, P, wg, n, st, dir, fl + 5 * s);
        else central_flux(g, P, n, st, dir, fl + 5 * s);
        if ((wall_lo && s == 0) || (wall_hi && s == nd)) {
          /* staggered wall interface: no mass, x/z momentum or energy crosses the wall */
          fl[5 * s + 0] = 0.0;
          fl[5 * s + 1] = 0.0;
          fl[5 * s + 3] = 0.0;
          fl[5 * s + 4] = 0.0;
        }
      }
      for (int s = 0; s < nd; ++s) {
        int i, j, k;
        if (dir == 0) { i = s; j = a; k = b; }
        else if (dir == 1) { i = a; j = s; k = b; }
        else { i = a; j = b; k = s; }
        double h = dir == 0 ? g->dx : (dir == 1 ? g->deta * g->yeta[j] : g->dz);
        ptrdiff_t q = iidx(g, i, j, k);
        for (int m = 0; m < 5; ++m)
          R[m * Nint + q] -= (fl[5 * (s + 1) + m] - fl[5 * s + m]) / h;
      }
    }
    free(fl);
  }
}

/* ---------------------------------------------------------------- viscous terms */

/* Viscous terms in Laplacian form at an interior node (Section 2.1 and Eqs. sigma, heat_vec):
 *   V_i = mu lap(u_i) + mu/3 d_i(div) + d_j mu (d_j u_i + d_i u_j) - 2/3 div d_i mu,
 *   V_E = u_i V_i + sigma_ij d_j u_i + k lap(T) + d_j k d_j T,  k = cp mu / Pr,
 * with first derivatives D1 and second derivatives D2 of order 2L; d_i(div) is D1 of the
 * ghost-filled node divergence. */
static void viscous_node(const grid_t* g, const prims_t* P, const double* divg, int i, int j,
                         int k, double* out) {
  const orc_cfg* c = g->c;
  const double* vel[3] = {P->u, P->v, P->w};
  double du[3][3], dT[3], dmu[3], ddiv[3], lap[3], lapT = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) du[a][b] = d1(g, vel[a], i, j, k, b);
  for (int b = 0; b < 3; ++b) {
    dT[b] = d1(g, P->T, i, j, k, b);
    dmu[b] = d1(g, P->mu, i, j, k, b);
    ddiv[b] = d1(g, divg, i, j, k, b);
  }
  for (int a = 0; a < 3; ++a) {
    lap[a] = 0.0;
    for (int b = 0; b < 3; ++b) lap[a] += d2(g, vel[a], i, j, k, b);
  }
  for (int b = 0; b < 3; ++b) lapT += d2(g, P->T, i, j, k, b);
  ptrdiff_t n = gidx(g, i, j, k);
  double mu = P->mu[n];
  double div = du[0][0] + du[1][1] + du[2][2];
  double V[3];
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
    for (int b = 0; b < 3; ++b) s += dmu[b] * (du[a][b] + du[b][a]);
    V[a] = mu * lap[a] + mu * ddiv[a] / 3.0 + s - 2.0 / 3.0 * div * dmu[a];
  }
  double uvec[3] = {P->u[n], P->v[n], P->w[n]};
  double work = 0.0, diss = 0.0;
  for (int a = 0; a < 3; ++a) work += uvec[a] * V[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double sig = mu * (du[a][b] + du[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
      diss += sig * du[a][b];
    }
  double kc = g->cp * mu / c->prandtl;
  double heat = kc * lapT;
  for (int b = 0; b < 3; ++b) heat += g->cp / c->prandtl * dmu[b] * dT[b];
  out[0] = 0.0;
  out[1] = V[0];
  out[2] = V[1];
  out[3] = V[2];
  out[4] = work + diss + heat;
}

/* ---------------------------------------------------------------- right-hand side */

static int rhs_impl(const orc_cfg* c, const double* w, double* rhs, double* theta_out,
                    double* div_out, unsigned char* fx, unsigned char* fy, unsigned char* fz) {
  grid_t g;
  if (grid_init(&g, c)) return -1;
  ptrdiff_t N = (ptrdiff_t)g.nx * g.ny * g.nz;
  double* wg[5];
  for (int m = 0; m < 5; ++m) wg[m] = alloc_nan(g.ng);
  load_interior(&g, w, wg);
  fill_ghosts_w(&g, wg);
  prims_t P;
  prims_alloc(&g, &P);
  primitives(&g, wg, &P);
  double* theta = alloc_nan(g.ng);
  double* divg = alloc_nan(g.ng);
  sensor(&g, &P, theta, divg);

  double* R = rhs ? rhs : malloc(sizeof(double) * 5 * (size_t)N);
  memset(R, 0, sizeof(double) * 5 * (size_t)N);
  if (c->convective || fx || fy || fz) {
    double* Rc = c->convective ? R : calloc(5 * (size_t)N, sizeof(double));
    convective_dir(&g, &P, wg, theta, 0, Rc, fx);
    convective_dir(&g, &P, wg, theta, 1, Rc, fy);
    convective_dir(&g, &P, wg, theta, 2, Rc, fz);
    if (!c->convective) free(Rc);
  }
  if (c->viscous) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          double v[5];
          viscous_node(&g, &P, divg, i, j, k, v);
          ptrdiff_t q = iidx(&g, i, j, k);
          for (int m = 0; m < 5; ++m) R[m * N + q] += v[m];
        }
  }
  if (c->forcing) {
    /* constant mass flow: f makes the volume integral of the x-momentum residual vanish;
     * the power f u is added to the energy residual (Eqs. 1b, 1c). */
    double vol = 0.0, sru = 0.0;
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          double dv = g.dx * (g.yeta[j] * g.deta) * g.dz;
          vol += dv;
          sru += R[1 * N + iidx(&g, i, j, k)] * dv;
        }
    double f = -sru / vol;
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          ptrdiff_t q = iidx(&g, i, j, k);
          R[1 * N + q] += f;
          R[4 * N + q] += f * P.u[gidx(&g, i, j, k)];
        }
  }
  if (theta_out || div_out)
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          if (theta_out) theta_out[iidx(&g, i, j, k)] = theta[gidx(&g, i, j, k)];
          if (div_out) div_out[iidx(&g, i, j, k)] = divg[gidx(&g, i, j, k)];
        }
  if (!rhs) free(R);
  free(theta); free(divg);
  prims_free(&P);
  for (int m = 0; m < 5; ++m) free(wg[m]);
  grid_free(&g);
  return 0;
}

int orc_rhs(const orc_cfg* c, const double* w, double* rhs) {
  return rhs_impl(c, w, rhs, NULL, NULL, NULL, NULL, NULL);
}

int orc_sensor(const orc_cfg* c, const double* w, double* theta, double* div, unsigned char* fx,
               unsigned char* fy, unsigned char* fz) {
  orc_cfg cc = *c;
  cc.convective = 0; /* flags are still produced by walking the interfaces */
  cc.viscous = 0;
  cc.forcing = 0;
  return rhs_impl(&cc, w, NULL, theta, div, fx, fy, fz);
}

int orc_fill_ghosts(const orc_cfg* c, const double* w, double* out) {
  grid_t g;
  if (grid_init(&g, c)) return -1;
  double* wg[5];
  for (int m = 0; m < 5; ++m) {
    wg[m] = out + (ptrdiff_t)m * g.ng;
    for (ptrdiff_t q = 0; q < g.ng; ++q) wg[m][q] = NAN;
  }
  load_interior(&g, w, wg);
  fill_ghosts_w(&g, wg);
  grid_free(&g);
  return 0;
}

/* ---------------------------------------------------------------- time integration */

/* Eq. RK: w^(l+1) = w^(l) + alpha_l dt R^(l-1) + beta_l dt R^(l). The printed alpha_1 = +17/60
 * is read as -17/60 (Wray's scheme; first-order consistency requires sum alpha + sum beta = 1). */
void orc_rk_stage_update(int stage, double dt, double* w, const double* r_old, const double* r,
                         long n) {
  static const double alpha[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
  static const double beta[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
  for (long q = 0; q < n; ++q)
    w[q] = w[q] + alpha[stage] * dt * r_old[q] + beta[stage] * dt * r[q];
}

/* Convective CFL step: dt = cfl / max over nodes of sum_d (|u_d| + c) / h_d. */
double orc_cfl_dt(const orc_cfg* c, const double* w, double cfl) {
  grid_t g;
  if (grid_init(&g, c)) return -1.0;
  ptrdiff_t N = (ptrdiff_t)g.nx * g.ny * g.nz;
  double smax = 0.0;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        ptrdiff_t q = iidx(&g, i, j, k);
        double rho = w[q];
        double u = w[N + q] / rho, v = w[2 * N + q] / rho, ww = w[3 * N + q] / rho;
        double E = w[4 * N + q] / rho;
        double T = (E - 0.5 * (u * u + v * v + ww * ww)) / g.cv;
        double p = rho * c->r_gas * T;
        double cs = sqrt(c->gamma * p / rho);
        double s = (fabs(u) + cs) / g.dx + (fabs(v) + cs) / (g.yeta[j] * g.deta) +
                   (fabs(ww) + cs) / g.dz;
        if (!(s <= smax)) smax = s; /* a NaN propagates */
      }
  grid_free(&g);
  return cfl / smax;
}

int orc_rk_step(const orc_cfg* c, double* w, double dt, double cfl, double* dt_used) {
  long n = 5L * c->nx * c->ny * c->nz;
  if (dt <= 0.0) dt = orc_cfl_dt(c, w, cfl);
  if (dt_used) *dt_used = dt;
  if (c->bc_xmin == ORC_BC_DF) {
    grid_t g;
    if (grid_init(&g, c)) return -1;
    grid_free(&g);
    df_advance(c, dt);
  }
  double* r_old = calloc((size_t)n, sizeof(double));
  double* r = malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  for (int stage = 0; stage < 3 && rc == 0; ++stage) {
    rc = orc_rhs(c, w, r);
    orc_rk_stage_update(stage, dt, w, r_old, r, n);
    double* t = r_old;
    r_old = r;
    r = t;
  }
  free(r_old);
  free(r);
  return rc;
}

/* Per-sample statistics: the primitives of each interior node from w (E = cv T + |u|^2/2,
 * p = rho R T), the 24 products listed in the header, then plain means over the homogeneous
 * directions (x and z, or z only). */
int orc_stats(const orc_cfg* c, const double* w, int mode, double* out) {
  grid_t g;
  if ((mode != 0 && mode != 1) || grid_init(&g, c)) return -1;
  ptrdiff_t N = (ptrdiff_t)g.nx * g.ny * g.nz;
  int nrow = mode == 0 ? g.ny : g.ny * g.nx;
  for (ptrdiff_t q = 0; q < (ptrdiff_t)ORC_NSTAT * nrow; ++q) out[q] = 0.0;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        ptrdiff_t n = iidx(&g, i, j, k);
        double rho = w[n];
        double u = w[N + n] / rho, v = w[2 * N + n] / rho, ww = w[3 * N + n] / rho;
        double T = (w[4 * N + n] / rho - 0.5 * (u * u + v * v + ww * ww)) / g.cv;
        double p = rho * c->r_gas * T;
        double val[ORC_NSTAT] = {rho,          u,          v,           ww,
                                 p,            T,          rho * u,     rho * v,
                                 rho * ww,     rho * T,    rho * u * u, rho * v * v,
                                 rho * ww * ww, rho * u * v, rho * u * ww, rho * v * ww,
                                 u * u,        v * v,      ww * ww,     u * v,
                                 p * p,        T * T,      rho * rho,   viscosity(c, T)};
        int row = mode == 0 ? j : j * g.nx + i;
        for (int q = 0; q < ORC_NSTAT; ++q) out[(ptrdiff_t)q * nrow + row] += val[q];
      }
  double cnt = mode == 0 ? (double)g.nx * g.nz : (double)g.nz;
  for (ptrdiff_t q = 0; q < (ptrdiff_t)ORC_NSTAT * nrow; ++q) out[q] /= cnt;
  grid_free(&g);
  return 0;
}

/* Metric-weighted totals: sum over interior nodes of w_m dx (y_eta deta) dz. */
int orc_totals(const orc_cfg* c, const double* w, double out[5]) {
  grid_t g;
  if (grid_init(&g, c)) return -1;
  ptrdiff_t N = (ptrdiff_t)g.nx * g.ny * g.nz;
  for (int m = 0; m < 5; ++m) {
    double s = 0.0;
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i)
          s += w[m * N + iidx(&g, i, j, k)] * (g.dx * (g.yeta[j] * g.deta) * g.dz);
    out[m] = s;
  }
  grid_free(&g);
  return 0;
}
