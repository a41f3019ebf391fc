/*
 * FP64 CPU oracle for the compressible Navier-Stokes right-hand side and the
 * Wray low-storage RK3 update of STREAmS (arXiv 2004.02276, Section 2).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the plain, slow reference that the
 * CUDA path is checked against. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it. It shares no code, header,
 * table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Arrays passed in and out are interior-only, SoA, x fastest:
 *   w[m][k][j][i], m = 0..4 for (rho, rho u, rho v, rho w, rho E),
 *   i < nx, j < ny, k < nz.  Size 5*nx*ny*nz doubles.
 *
 * Interface flags (which interfaces use WENO) are returned per direction:
 *   x: [nz][ny][nx+1], y: [nz][ny+1][nx], z: [nz+1][ny][nx];
 *   entry s along the direction is the interface between nodes s-1 and s.
 */
#ifndef STRM_ORACLE_H
#define STRM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MAP_UNIFORM = 0, ORC_MAP_TANH = 1, ORC_MAP_TANH_ONESIDED = 2, ORC_MAP_ERF = 3,
       ORC_MAP_SINH_ONESIDED = 4 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_CHAR = 2, ORC_BC_RECYCLE = 3, ORC_BC_DF = 4 };
enum { ORC_WENO_OFF = 0, ORC_WENO_SENSOR = 1, ORC_WENO_ALL = 2 };
enum { ORC_VISC_POWER = 0, ORC_VISC_SUTHERLAND = 1 };

typedef struct {
  /* grid: nx*ny*nz interior nodes; y nodes at eta_j = (j+1/2)/ny */
  int nx, ny, nz;
  double lx, ly, lz;
  int y_map;            /* ORC_MAP_UNIFORM, ORC_MAP_TANH or ORC_MAP_ERF (both walls), or
                           ORC_MAP_TANH_ONESIDED or ORC_MAP_SINH_ONESIDED (wall at y = 0) */
  double beta;          /* stretching parameter of the map */
  /* face kinds (z is periodic): x faces PERIODIC, RECYCLE or DF (x-min only) or CHAR; y faces
   * PERIODIC, WALL or CHAR */
  int bc_xmin, bc_xmax, bc_ymin, bc_ymax;
  double ref[5];        /* reference primitives (rho, u, v, w, p) seen by characteristic faces */
  int shock;            /* 1: y-max characteristic ghosts downstream of the shock foot see the
                           post-shock state of an oblique shock of deflection shock_theta that
                           reaches the wall at x = shock_ximp */
  double shock_theta, shock_ximp;
  int i_recycle;        /* recycling plane (interior x index >= 2) */
  double delta_in;      /* inflow boundary-layer thickness (99 % of ref u) */
  /* digital-filter inflow (bc_xmin == ORC_BC_DF; Section 3.2): mean profiles and Reynolds
   * stresses per wall-normal node, df_prof[7][ny] = U, V, T, R11, R12, R22, R33; filter
   * half-widths n in grid points along y and z (support 2n on each side); integral time tau;
   * generator seed; the fluctuation plane df_psi[3][nz][ny] and the draw counter df_count,
   * both kept by the caller and updated by orc_df_init and orc_rk_step. The ghost pressure is
   * ref[4]. */
  const double* df_prof;
  double* df_psi;
  long long* df_count;
  int df_ny, df_nz;
  double df_tau;
  unsigned long long df_seed;
  /* gas: p = rho R T, E = cv T + |u|^2/2, k = cp mu / Pr */
  double gamma, prandtl, r_gas;
  int visc_law;         /* mu = mu_ref (T/t_ref)^visc_exp, or Sutherland with constant suth_s */
  double mu_ref, t_ref, visc_exp, suth_s;
  double t_wall;        /* isothermal wall temperature */
  int forcing;          /* constant mass flow rate forcing in x */
  /* scheme */
  int L;                /* central stencil half width (order 2L): 2 or 3 */
  int weno_mode;        /* ORC_WENO_OFF / SENSOR / ALL */
  double theta_thr;     /* sensor threshold */
  double weno_eps;      /* WENO epsilon */
  double u0, l0;        /* sensor velocity and length scales */
  int convective, viscous; /* term switches (both 1 for the full method) */
  /* nullable: a prescribed sensor value at the interior nodes ([nz][ny][nx]) that the hybrid
   * switch reads instead of the computed Ducros sensor (a test device: it fixes the
   * central/WENO decisions so that two runs can be compared without decision flips) */
  const double* theta_fixed;
} orc_cfg;

/* Full right-hand side R(w) (convective + viscous + forcing), interior only. */
int orc_rhs(const orc_cfg* c, const double* w, double* rhs);

/* One Wray RK3 step in place. dt > 0: fixed; dt <= 0: CFL step with number cfl.
 * The step used is written to *dt_used (nullable). */
int orc_rk_step(const orc_cfg* c, double* w, double dt, double cfl, double* dt_used);

/* One RK stage update w <- w + dt (alpha_l r_old + beta_l r), n values. */
void orc_rk_stage_update(int stage, double dt, double* w, const double* r_old,
                         const double* r, long n);

/* CFL time step for the state w. */
double orc_cfl_dt(const orc_cfg* c, const double* w, double cfl);

/* Volume-weighted totals of the five conserved fields. */
int orc_totals(const orc_cfg* c, const double* w, double out[5]);

/* Sensor, node divergence and interface flags (see layout above). Each output nullable. */
int orc_sensor(const orc_cfg* c, const double* w, double* theta, double* div,
               unsigned char* fx, unsigned char* fy, unsigned char* fz);

/* Ghost-filled conserved field, [5][nz+2G][ny+2G][nx+2G], G = 3. Corners stay NaN. */
int orc_fill_ghosts(const orc_cfg* c, const double* w, double* wg);

/* Wall-normal metrics at the nodes: y(eta_j), y_eta, y_etaeta (each ny). */
void orc_metrics(const orc_cfg* c, double* y, double* yeta, double* yetaeta);

/* Left/right eigenvectors of the flux Jacobian along direction dir (0,1,2) at the state
 * (u, v, w, H) with sound speed from H, row-major 5x5; Lm * Rm = I. */
void orc_eigvecs(int dir, double gamma, double u, double v, double w, double H,
                 double* Lm, double* Rm);

/* WENO5-JS reconstruction at i+1/2 from f[0..4] = f_{i-2..i+2}. */
double orc_weno5(const double* f, double eps);

/* Weak-branch oblique shock of deflection theta (radians) in a stream of Mach number mach:
 * writes the shock angle beta and the ratios p2/p1, rho2/rho1 and the post-shock Mach number.
 * Returns 0, or -1 if the deflection exceeds the attached-shock limit. */
int orc_oblique_shock(double gamma, double mach, double theta, double* beta, double* p_ratio,
                      double* rho_ratio, double* mach2);

/* Digital-filter inflow: draw the first fluctuation plane (draw 0) into df_psi and set
 * df_count = 1. Each orc_rk_step then blends in a new draw (see the source for the steps). */
int orc_df_init(const orc_cfg* c);

/* SplitMix64 output number k + 1 for the given seed (the generator of the inflow's random
 * numbers; exported for its test vector). */
unsigned long long orc_splitmix64(unsigned long long seed, unsigned long long k);

/* Filtered (not time-correlated) random plane of draw number `draw`, psi[3][nz][ny]. */
int orc_df_plane(const orc_cfg* c, long long draw, double* psi);

/* Threads of the OpenMP loops (n >= 1); returns the number in use afterwards. Timing only: the
 * results do not depend on it (every loop writes disjoint nodes in a fixed order per node). */
int orc_set_threads(int n);

/* Recycling rescale factor s = delta_r / delta_in for the state w (1 if no recycling face). */
double orc_recycle_scale(const orc_cfg* c, const double* w);

/* Statistics of one state (Section 3: Reynolds and Favre decompositions use averages over the
 * homogeneous directions and time; this is the spatial part for one sample). Quantities, in
 * this order (ORC_NSTAT of them):
 *   rho, u, v, w, p, T, rho u, rho v, rho w, rho T, rho uu, rho vv, rho ww, rho uv, rho uw,
 *   rho vw, uu, vv, ww, uv, p^2, T^2, rho^2, mu.
 * mode 0: averages over x and z, out[q][j] (ORC_NSTAT x ny);
 * mode 1: averages over z, out[q][j][i] (ORC_NSTAT x ny x nx). */
enum { ORC_NSTAT = 24 };
int orc_stats(const orc_cfg* c, const double* w, int mode, double* out);

/* Number of ghost layers used by the oracle. */
int orc_ghosts(void);

#ifdef __cplusplus
}
#endif
#endif
