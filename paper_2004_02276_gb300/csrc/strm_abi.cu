// C ABI of the library (declared in include/strm.h): context, workspace layout, stage
// sequencing on the caller's stream, and the CUDA graph replayed by strm_advance_n.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/strm.h"
#include "strm_dev.cuh"
#include "strm_launch.h"

using namespace strm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define STRM_CK(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(STRM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

#define STRM_CK_LAUNCH()                                                                   \
  do {                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) return fail(STRM_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Node fields held in FP64 and in FP32 (mixed precision only). FP64 precision: 12 fields, the
// 6 wave speeds u_d -+ c, the 3 momentum components and the 3 normal momentum fluxes; mixed
// precision: the 9 fields the FP64 characteristic projection and switch read and the same 6.
const int kN64All = 24, kN64Mixed = 15, kN32Mixed = 11, kN32Xdev = 3;

struct Layout {
  Dims d;
  bool mixed;
  size_t off_n64[kN64All], off_n32[kN32Mixed], off_xdev[kN32Xdev], off_xref;
  size_t off_fh[3];
  size_t off_R, off_grad, off_band, off_dbg, off_wl[3], off_cl[3], off_wcount, off_red, off_scal, off_metric, off_metric32;
  size_t total;
};

bool valid_grid(const strm_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->lx > 0 && g->ly > 0 && g->lz > 0 &&
         (g->y_map == STRM_MAP_UNIFORM ||
          ((g->y_map == STRM_MAP_TANH || g->y_map == STRM_MAP_TANH_ONESIDED || g->y_map == STRM_MAP_ERF ||
            g->y_map == STRM_MAP_SINH_ONESIDED) &&
           g->beta > 0));
}

bool valid_scheme(const strm_scheme* s) {
  return s && (s->L == 2 || s->L == 3) && s->weno_mode >= 0 && s->weno_mode <= 2 &&
         (s->precision == STRM_PREC_FP64 || s->precision == STRM_PREC_MIXED) && s->weno_eps > 0 &&
         s->l0 > 0;
}

Layout make_layout(const strm_grid* g, const strm_scheme* s) {
  Layout L{};
  L.mixed = s->precision == STRM_PREC_MIXED;
  Dims& d = L.d;
  d.nx = g->nx;
  d.ny = g->ny;
  d.nz = g->nz;
  d.px = ((g->nx + GX + G) + 3) / 4 * 4;
  d.py = g->ny + 2 * G;
  d.pz = g->nz + 2 * G;
  d.plane = (long long)d.px * d.py;
  d.ng = d.plane * d.pz;
  d.N = (long long)d.nx * d.ny * d.nz;
  d.nf[0] = (long long)(d.nx + 1) * d.ny * d.nz;
  d.nf[1] = (long long)d.nx * (d.ny + 1) * d.nz;
  d.nf[2] = (long long)d.nx * d.ny * (d.nz + 1);
  d.slab_ty = slab_rows_for(d.nx, d.ny, 32);
  // the z faces walk 8-row slabs: on the 2048 x 384 x 256 workload their classification list
  // then feeds the mixed z WENO kernel 8 % faster than with 32 rows (the assembly, which reads
  // y stencils across slab edges, stays fastest at 32)
  d.zslab_ty = slab_rows_for(d.nx, d.ny, 8);
  size_t off = 0;
  int n64 = L.mixed ? kN64Mixed : kN64All;
  for (int f = 0; f < n64; ++f) {
    L.off_n64[f] = off;
    off = align_up(off + sizeof(double) * (size_t)d.ng);
  }
  if (L.mixed) {
    for (int f = 0; f < kN32Mixed; ++f) {
      L.off_n32[f] = off;
      off = align_up(off + sizeof(float) * (size_t)d.ng);
    }
    // the x rows' deviations from their reference, and the references
    for (int f = 0; f < kN32Xdev; ++f) {
      L.off_xdev[f] = off;
      off = align_up(off + sizeof(float) * (size_t)d.ng);
    }
    L.off_xref = off;
    off = align_up(off + sizeof(float) * kN32Xdev * (size_t)d.ny * d.nz);
  }
  size_t fbytes = L.mixed ? sizeof(float) : sizeof(double);
  for (int dir = 0; dir < 3; ++dir) {
    L.off_fh[dir] = off;
    off = align_up(off + fbytes * 5 * (size_t)d.nf[dir]);
  }
  L.off_R = off;
  off = align_up(off + sizeof(double) * 5 * (size_t)d.N);
  // FP64: the velocity gradients of the sensor, reused by the viscous terms
  L.off_grad = off;
  if (!L.mixed) off = align_up(off + sizeof(double) * 9 * (size_t)d.N);
  // mixed: the list of nodes whose FP32 theta is near the switch threshold
  L.off_band = off;
  if (L.mixed) off = align_up(off + sizeof(int) * (size_t)d.N);
  for (int dir = 0; dir < 3; ++dir) {
    L.off_wl[dir] = off;
    off = align_up(off + sizeof(int) * (size_t)d.nf[dir]);
    L.off_cl[dir] = off;
    off = align_up(off + sizeof(int) * (size_t)d.nf[dir]);
  }
  L.off_wcount = off;
  off = align_up(off + 8 * sizeof(unsigned));
  L.off_dbg = off;  // error word of the bounds-checking (debug) build
  off = align_up(off + sizeof(unsigned));
  L.off_red = off;
  off = align_up(off + sizeof(double) * (5 * (size_t)reduce_blocks(d) + 64));
  L.off_scal = off;
  off = align_up(off + sizeof(double) * kScalCount);
  L.off_metric = off;
  off = align_up(off + sizeof(double) * 7 * (size_t)d.ny);  // 4 metrics, heights, c1/hy, recycle means
  L.off_metric32 = off;
  off = align_up(off + sizeof(float) * 3 * (size_t)d.ny);
  L.total = off;
  return L;
}

}  // namespace

int strm::record_error(int code, const std::string& msg) { return fail(code, msg); }

struct strm_ctx {
  strm_grid g;
  strm_phys p;
  strm_scheme s;
  Dims d;
  Consts C;
  Bufs B;
  cudaStream_t stream = nullptr;
  int weno_grid = 0;
  std::vector<double> metric_host;   // kept alive for the asynchronous uploads
  std::vector<float> metric_host32;
  double time_host[2] = {0.0, 0.0};
  // graph of one RK step, replayed by strm_advance_n
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double* g_w = nullptr;
  double* g_r = nullptr;
  double g_dt = 0.0, g_cfl = 0.0;
  long long graph_kernels = 0;
  // launch accounting and the optional per-kernel event timing
  long long launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> events;
  struct Rec {
    int cls, e0, e1;
  };
  std::vector<Rec> recs;
  double kms[STRM_K_COUNT] = {};
  long long klaunch[STRM_K_COUNT] = {};
  long long weno_faces[3] = {};
  // statistics accumulator (caller-owned buffer)
  double* st_acc = nullptr;  // [STRM_NSTAT][rows]
  double* st_scr = nullptr;  // x-z mode: [STRM_NSTAT][ny][nx] column sums
  int st_mode = 0;
  int st_every = 0;
  long long st_samples = 0;
  long long st_steps = 0;
  // digital-filter inflow (caller-owned buffer)
  DFParams df = {};
  std::vector<double> df_host;  // profiles and filter coefficients, kept for the async upload
  // overlap (strm_set_overlap): two side streams and the fork/join events of one right-hand side
  // prescribed switch input (strm_set_theta): caller-owned device array of N doubles, or null
  const double* theta_fixed = nullptr;
  int overlap = 0;  // STRM_OVERLAP_* bits
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

// Weak-branch oblique shock (Section 3.3): the deflection theta(beta) = atan(2 cot beta
// (M^2 sin^2 beta - 1) / (M^2 (gamma + cos 2 beta) + 2)) grows from 0 at the Mach angle to a
// maximum; the weak shock angle is the root below that maximum (found by bisection after a
// golden-section search for the maximum), followed by the normal-shock relations.
double deflection(double gamma, double M, double beta) {
  double sb = std::sin(beta);
  return std::atan(2.0 / std::tan(beta) * (M * M * sb * sb - 1.0) / (M * M * (gamma + std::cos(2.0 * beta)) + 2.0));
}

bool oblique_shock(double gamma, double M, double theta, double* beta, double* pr, double* rr, double* m2) {
  if (!(M > 1.0) || !(theta > 0.0)) return false;
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  double a = std::asin(1.0 / M), b = 0.5 * std::acos(-1.0);
  double x1 = b - g * (b - a), x2 = a + g * (b - a);
  for (int it = 0; it < 200; ++it) {
    if (deflection(gamma, M, x1) < deflection(gamma, M, x2)) {
      a = x1;
      x1 = x2;
      x2 = a + g * (b - a);
    } else {
      b = x2;
      x2 = x1;
      x1 = b - g * (b - a);
    }
  }
  double bmax = 0.5 * (a + b);
  if (theta > deflection(gamma, M, bmax)) return false;
  double lo = std::asin(1.0 / M), hi = bmax;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    (deflection(gamma, M, mid) < theta ? lo : hi) = mid;
  }
  double bs = 0.5 * (lo + hi), mn = M * std::sin(bs);
  *beta = bs;
  *pr = 1.0 + 2.0 * gamma / (gamma + 1.0) * (mn * mn - 1.0);
  *rr = (gamma + 1.0) * mn * mn / ((gamma - 1.0) * mn * mn + 2.0);
  double m2n2 = (mn * mn + 2.0 / (gamma - 1.0)) / (2.0 * gamma / (gamma - 1.0) * mn * mn - 1.0);
  *m2 = std::sqrt(m2n2) / std::sin(bs - theta);
  return true;
}

template <typename R>
void fill_coefs(Coefs<R>& K, const strm_phys& p, const strm_scheme& s, const strm_grid& g) {
  for (int l = 0; l < 4; ++l) K.a[l] = K.b[l] = R(0);
  // central coefficients of order 2L: first derivative a_l, second derivative b_l with
  // f'' ~ sum_l b_l (f_{+l} + f_{-l} - 2 f_0)/h^2 (Section 2.1)
  // b_0 = -2 sum_l b_l is the centre weight of the same stencil written as sum_l b_l f_l
  if (s.L == 3) {
    K.a[1] = R(3.0 / 4.0); K.a[2] = R(-3.0 / 20.0); K.a[3] = R(1.0 / 60.0);
    K.b[0] = R(-49.0 / 18.0); K.b[1] = R(3.0 / 2.0); K.b[2] = R(-3.0 / 20.0); K.b[3] = R(1.0 / 90.0);
  } else {
    K.a[1] = R(2.0 / 3.0); K.a[2] = R(-1.0 / 12.0);
    K.b[0] = R(-5.0 / 2.0); K.b[1] = R(4.0 / 3.0); K.b[2] = R(-1.0 / 12.0);
  }
  double dx = g.lx / g.nx, dz = g.lz / g.nz;
  for (int l = 0; l < 4; ++l) {
    K.ax[l] = R((double)K.a[l] / dx);
    K.az[l] = R((double)K.a[l] / dz);
    K.aq[l] = R(0.25 * (double)K.a[l]);
  }
  for (int r = 0; r < 4; ++r) {
    double t = 0.0;
    for (int l = r + 1; l <= s.L; ++l) t += (double)K.a[l];
    K.ap[r] = R(t);
  }
  for (int l = 0; l < 4; ++l) {
    K.bx[l] = R((double)K.b[l] / (dx * dx));
    K.bz[l] = R((double)K.b[l] / (dz * dz));
  }
  K.bxz0 = R((double)K.b[0] / (dx * dx) + (double)K.b[0] / (dz * dz));
  K.inv_dx = R(1.0 / dx);
  K.inv_dz = R(1.0 / dz);
  K.inv_dx2 = R((1.0 / dx) * (1.0 / dx));
  K.inv_dz2 = R((1.0 / dz) * (1.0 / dz));
  double cv = p.r_gas / (p.gamma - 1.0), cp = p.gamma * cv;
  K.cp_pr = R(cp / p.prandtl);
  K.sens_eps = R((s.u0 / s.l0) * (s.u0 / s.l0));
  K.theta_thr = R(s.theta_thr);
  K.weno_eps = R(s.weno_eps);
  K.gamma = R(p.gamma);
  K.gm1 = R(p.gamma - 1.0);
  K.r_gas = R(p.r_gas);
  K.cp = R(cp);
  K.t_wall = R(p.t_wall);
  K.mu_ref = R(p.mu_ref);
  K.inv_tref = R(1.0 / p.t_ref);
  K.visc_exp = R(p.visc_exp);
  K.exp_19_25 = p.visc_law == STRM_VISC_POWER && std::fabs(p.visc_exp - 0.76) < 1e-15 ? 1 : 0;
  K.suth_s = R(p.suth_s);
}

void set_consts(strm_ctx* x) {
  Consts& C = x->C;
  const strm_phys& p = x->p;
  const strm_scheme& s = x->s;
  C.gamma = p.gamma;
  C.gm1 = p.gamma - 1.0;
  C.r_gas = p.r_gas;
  C.inv_r = 1.0 / p.r_gas;
  C.cv = p.r_gas / (p.gamma - 1.0);
  C.inv_cv = 1.0 / C.cv;
  C.cp = p.gamma * C.cv;
  C.cp_pr = C.cp / p.prandtl;
  C.mu_ref = p.mu_ref;
  C.inv_tref = 1.0 / p.t_ref;
  C.visc_exp = p.visc_exp;
  C.suth_s = p.suth_s;
  C.t_wall = p.t_wall;
  C.visc_law = p.visc_law;
  C.forcing = p.forcing ? 1 : 0;
  C.L = s.L;
  C.weno_mode = s.weno_mode;
  C.convective = s.convective ? 1 : 0;
  C.viscous = s.viscous ? 1 : 0;
  C.mixed = s.precision == STRM_PREC_MIXED ? 1 : 0;
  C.p_shift = (double)(float)(p.r_gas * p.t_ref);
  fill_coefs(C.k64, p, s, x->g);
  fill_coefs(C.k32, p, s, x->g);
}

// Wall-normal metrics at the nodes eta_j = (j + 1/2)/ny of y = (ly/2) tanh(beta(2 eta - 1))/tanh(beta)
// (uniform: y = ly (eta - 1/2)): 1/(y_eta deta), its square, y_etaeta/(y_eta^3 deta) and the node
// volume dx (y_eta deta) dz.
void build_metrics(strm_ctx* x) {
  const strm_grid& g = x->g;
  int ny = g.ny;
  double deta = 1.0 / ny, dx = g.lx / g.nx, dz = g.lz / g.nz;
  x->metric_host.assign(6 * (size_t)ny, 0.0);
  double vt = 0.0;
  for (int j = 0; j < ny; ++j) {
    double eta = (j + 0.5) * deta, ye, yee, h;
    if (g.y_map == STRM_MAP_TANH_ONESIDED) {
      // y = ly (1 - tanh(beta (1 - eta)) / tanh(beta)), wall at y = 0
      double A = g.ly / std::tanh(g.beta);
      double th = std::tanh(g.beta * (1.0 - eta));
      double sech2 = 1.0 - th * th;
      ye = A * g.beta * sech2;
      yee = 2.0 * A * g.beta * g.beta * sech2 * th;
      h = g.ly - A * th;
    } else if (g.y_map == STRM_MAP_TANH) {
      double A = 0.5 * g.ly / std::tanh(g.beta);
      double th = std::tanh(g.beta * (2.0 * eta - 1.0));
      double sech2 = 1.0 - th * th;
      ye = 2.0 * g.beta * A * sech2;
      yee = -8.0 * g.beta * g.beta * A * sech2 * th;
      h = A * th + 0.5 * g.ly;
    } else if (g.y_map == STRM_MAP_ERF) {
      // y = (ly/2) erf(beta s) / erf(beta), s = 2 eta - 1: y_eta = (2 ly beta / (sqrt(pi)
      // erf(beta))) exp(-beta^2 s^2), y_etaeta = -4 beta^2 s y_eta
      double sv = 2.0 * eta - 1.0, E = std::erf(g.beta);
      ye = 2.0 * g.ly * g.beta / (std::sqrt(std::acos(-1.0)) * E) * std::exp(-g.beta * g.beta * sv * sv);
      yee = -4.0 * g.beta * g.beta * sv * ye;
      h = 0.5 * g.ly * std::erf(g.beta * sv) / E + 0.5 * g.ly;
    } else if (g.y_map == STRM_MAP_SINH_ONESIDED) {
      // y = ly sinh(beta eta) / sinh(beta): y_eta = ly beta cosh / sinh(beta), y_etaeta = beta^2 y
      double S = std::sinh(g.beta);
      h = g.ly * std::sinh(g.beta * eta) / S;
      ye = g.ly * g.beta * std::cosh(g.beta * eta) / S;
      yee = g.beta * g.beta * h;
    } else {
      ye = g.ly;
      yee = 0.0;
      h = g.ly * eta;
    }
    double ih = 1.0 / (ye * deta);
    x->metric_host[j] = ih;
    x->metric_host[ny + j] = ih * ih;
    x->metric_host[2 * ny + j] = yee / (ye * ye * ye * deta);
    x->metric_host[3 * ny + j] = dx * (ye * deta) * dz;
    x->metric_host[4 * ny + j] = h;  // height above the wall eta = 0
    x->metric_host[5 * ny + j] = yee / (ye * ye);  // c1y / inv_hy: y_etaeta/y_eta^2
    vt += x->metric_host[3 * ny + j];
  }
  x->metric_host32.resize(3 * (size_t)ny);
  for (int q = 0; q < 3 * ny; ++q) x->metric_host32[q] = (float)x->metric_host[q];
  x->C.vtot = vt * g.nx * g.nz;
}

const char* const kKernelNames[STRM_K_COUNT] = {
    "prims", "dt_finalize", "ghost_prims", "sensor", "ghost_sensor", "faces_x", "faces_y",
    "faces_z", "weno_x", "weno_y", "weno_z", "assemble", "force_finalize", "rk_update"};

int take_event(strm_ctx* x, size_t idx) {
  while (x->events.size() <= idx) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    x->events.push_back(e);
  }
  return (int)idx;
}

// Fold recorded event pairs into the per-kernel totals (synchronises the stream).
int fold_timing(strm_ctx* x) {
  if (x->recs.empty()) return STRM_OK;
  STRM_CK(cudaStreamSynchronize(x->stream));
  for (const auto& r : x->recs) {
    float ms = 0.f;
    STRM_CK(cudaEventElapsedTime(&ms, x->events[r.e0], x->events[r.e1]));
    x->kms[r.cls] += ms;
    x->klaunch[r.cls] += 1;
  }
  x->recs.clear();
  return STRM_OK;
}

// Launch accounting around one kernel launch; with timing on, an event pair brackets it.
struct LaunchScope {
  strm_ctx* x;
  cudaStream_t st;
  int cls, e0 = -1;
  int kernels = 1;  // kernels the scope launched (counted into x->launches)
  LaunchScope(strm_ctx* x_, cudaStream_t st_, int cls_) : x(x_), st(st_), cls(cls_) {
    if (x->timing) {
      if (x->recs.size() >= 2048) fold_timing(x);
      e0 = take_event(x, 2 * x->recs.size());
      if (e0 >= 0) cudaEventRecord(x->events[e0], st);
    }
  }
  ~LaunchScope() {
    x->launches += kernels;
    if (e0 >= 0) {
      int e1 = take_event(x, e0 + 1);
      if (e1 >= 0) {
        cudaEventRecord(x->events[e1], st);
        x->recs.push_back({cls, e0, e1});
      }
    }
  }
};

#define STRM_LAUNCH(cls, expr) \
  do {                         \
    LaunchScope ls_(x, st, cls); \
    expr;                      \
  } while (0)

// a scope that launches n kernels, n given by the expression
#define STRM_LAUNCH_N(cls, n_expr)   \
  do {                               \
    LaunchScope ls_(x, st, cls);     \
    ls_.kernels = (n_expr);          \
  } while (0)

// One right-hand-side evaluation into R (stream order). With dt_mode, stage-0 work also sets the
// step: dt_fixed > 0 is taken as is, otherwise the CFL step from the primitive pass.
int enqueue_rhs(strm_ctx* x, const double* w, double* R, bool dt_mode, double cfl, double dt_fixed,
                cudaStream_t st, const RkFuse& rk = RkFuse{nullptr, nullptr, 0}) {
  const Dims& d = x->d;
  const Consts& C = x->C;
  const Bufs& B = x->B;
  if ((C.bc[0] == kBcPeriodic) != (C.bc[1] == kBcPeriodic) || (C.bc[2] == kBcPeriodic) != (C.bc[3] == kBcPeriodic))
    return fail(STRM_EINVAL, "a periodic face needs a periodic opposite face");
  STRM_CK(cudaMemsetAsync(B.wcount, 0, 8 * sizeof(unsigned), st));
  STRM_LAUNCH(STRM_K_PRIMS, launch_prims(d, C, B, w, dt_mode && dt_fixed <= 0.0, st));
  if (dt_mode) STRM_LAUNCH(STRM_K_DT, launch_dt_finalize(d, B, cfl, dt_fixed, st));
  if (C.bc[0] == kBcRecycle) STRM_LAUNCH_N(STRM_K_GHOST_PRIMS, (launch_recycle(d, C, B, st), 2));
  // digital-filter inflow: a new plane once per step, after the step's dt is known
  if (dt_mode && C.bc[0] == kBcDigitalFilter)
    STRM_LAUNCH_N(STRM_K_GHOST_PRIMS, (launch_df_update(d, x->df, B, false, st), 2));
  // With overlap (not in timing mode, whose per-kernel events assume one stream): the ghost
  // fill runs on a side stream while the sensor covers the nodes whose stencils read no ghost;
  // the sensor's boundary shell follows the join. Later the x, y and z face stages, which
  // write separate flux arrays and lists, run as three concurrent branches.
  const int ovl = x->timing ? 0 : x->overlap;
  if ((ovl & STRM_OVERLAP_GHOST) && sensor_inner_nodes(d, C.L) > 0) {
    STRM_CK(cudaEventRecord(x->ev[0], st));
    STRM_CK(cudaStreamWaitEvent(x->side[0], x->ev[0], 0));
    STRM_LAUNCH(STRM_K_GHOST_PRIMS, launch_ghost_prims(d, C, B, x->side[0]));
    STRM_CK(cudaEventRecord(x->ev[1], x->side[0]));
    STRM_LAUNCH(STRM_K_SENSOR, launch_sensor(d, C, B, 1, st));
    STRM_CK(cudaStreamWaitEvent(st, x->ev[1], 0));
    STRM_LAUNCH(STRM_K_SENSOR, launch_sensor(d, C, B, 2, st));
  } else {
    STRM_LAUNCH(STRM_K_GHOST_PRIMS, launch_ghost_prims(d, C, B, st));
    STRM_LAUNCH(STRM_K_SENSOR, launch_sensor(d, C, B, 0, st));
  }
  if (C.mixed && C.weno_mode == 1 && !x->theta_fixed) STRM_LAUNCH(STRM_K_SENSOR, launch_band_theta(d, C, B, st));
  if (x->theta_fixed) STRM_LAUNCH(STRM_K_SENSOR, launch_theta_set(d, B, x->theta_fixed, st));
  STRM_LAUNCH(STRM_K_GHOST_SENSOR, launch_ghost_scalars(d, C, B, st));
  if (C.convective && (ovl & STRM_OVERLAP_FACES)) {
    STRM_CK(cudaEventRecord(x->ev[2], st));
    for (int b = 0; b < 2; ++b) STRM_CK(cudaStreamWaitEvent(x->side[b], x->ev[2], 0));
    for (int dir = 0; dir < 3; ++dir) {
      cudaStream_t sd = dir == 0 ? st : x->side[dir - 1];
      STRM_LAUNCH_N(STRM_K_FACES_X + dir, launch_faces_dir(d, C, B, dir, x->weno_grid * 2, sd));
      if (C.weno_mode != STRM_WENO_OFF)
        STRM_LAUNCH(STRM_K_WENO_X + dir, launch_weno_dir(d, C, B, dir, x->weno_grid, sd));
    }
    for (int b = 0; b < 2; ++b) {
      STRM_CK(cudaEventRecord(x->ev[3 + b], x->side[b]));
      STRM_CK(cudaStreamWaitEvent(st, x->ev[3 + b], 0));
    }
  } else if (C.convective) {
    for (int dir = 0; dir < 3; ++dir)
      STRM_LAUNCH_N(STRM_K_FACES_X + dir, launch_faces_dir(d, C, B, dir, x->weno_grid * 2, st));
    if (C.weno_mode != STRM_WENO_OFF) {
      for (int dir = 0; dir < 3; ++dir)
        STRM_LAUNCH(STRM_K_WENO_X + dir, launch_weno_dir(d, C, B, dir, x->weno_grid, st));
      if (x->timing) {  // pageable destination: the copy completes before the call returns
        unsigned c[4];
        STRM_CK(cudaMemcpyAsync(c, B.wcount, sizeof(c), cudaMemcpyDeviceToHost, st));
        STRM_CK(cudaStreamSynchronize(st));
        for (int dir = 0; dir < 3; ++dir) x->weno_faces[dir] += c[dir];
      }
    }
  }
  STRM_LAUNCH(STRM_K_ASSEMBLE, launch_assemble(d, C, B, R, rk, st));
  if (C.forcing) STRM_LAUNCH(STRM_K_FORCE, launch_force_finalize(d, C, B, st));
  STRM_CK_LAUNCH();
  return STRM_OK;
}

int enqueue_step(strm_ctx* x, double* w, double* r_old, double dt, double cfl, cudaStream_t st) {
  for (int stage = 0; stage < 3; ++stage) {
    if (!x->C.forcing) {  // no forcing to reduce first: the assembly applies the stage update
      int rc = enqueue_rhs(x, w, x->B.R, stage == 0, cfl, dt, st, RkFuse{w, r_old, stage});
      if (rc) return rc;
      continue;
    }
    int rc = enqueue_rhs(x, w, x->B.R, stage == 0, cfl, dt, st);
    if (rc) return rc;
    STRM_LAUNCH(STRM_K_RK_UPDATE,
                launch_rk_update(x->d, x->C, x->B, w, r_old, stage, st));
  }
  STRM_CK_LAUNCH();
  return STRM_OK;
}

int check_step_args(const strm_ctx* x, const double* w, const double* r_old, double dt, double cfl) {
  if (!x || !w || !r_old) return fail(STRM_EINVAL, "null context or buffer");
  if (w == r_old) return fail(STRM_EINVAL, "w and r_old must not alias");
  if (!(dt > 0.0) && !(cfl > 0.0)) return fail(STRM_EINVAL, "need dt > 0 or cfl > 0");
  return STRM_OK;
}

}  // namespace

extern "C" {

const char* strm_last_error(void) { return g_last_error.c_str(); }

size_t strm_workspace_bytes(const strm_grid* g, const strm_scheme* s) {
  if (!valid_grid(g) || !valid_scheme(s)) return 0;
  return make_layout(g, s).total;
}

int strm_init_grid(strm_ctx** out, const strm_grid* g, const strm_phys* p, const strm_scheme* s,
                   void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return fail(STRM_EINVAL, "ctx out-pointer is null");
  *out = nullptr;
  if (!valid_grid(g)) return fail(STRM_EINVAL, "invalid grid (sizes >= 1, lengths > 0, tanh needs beta > 0)");
  if (!valid_scheme(s)) return fail(STRM_EINVAL, "invalid scheme (L in {2,3}, weno_mode in 0..2, precision fp64 or mixed)");
  if (!p || !(p->gamma > 1.0) || !(p->r_gas > 0) || !(p->prandtl > 0) || !(p->mu_ref >= 0) ||
      !(p->t_ref > 0) || !(p->t_wall > 0) || p->visc_law < 0 || p->visc_law > 1)
    return fail(STRM_EINVAL, "invalid physical parameters");
  Layout L = make_layout(g, s);
  if (!workspace) return fail(STRM_EINVAL, "workspace is null");
  if (((uintptr_t)workspace & 255) != 0) return fail(STRM_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(STRM_ENOMEM, "workspace too small: need " + std::to_string(L.total) + " bytes");
  strm_ctx* x = new (std::nothrow) strm_ctx();
  if (!x) return fail(STRM_ENOMEM, "host allocation failed");
  x->g = *g;
  x->p = *p;
  x->s = *s;
  x->d = L.d;
  x->stream = (cudaStream_t)stream;
  set_consts(x);
  for (int f = 0; f < 4; ++f) x->C.bc[f] = kBcPeriodic;
  x->C.shock = 0;
  x->C.i_recycle = 0;
  x->C.delta_in = 1.0;
  x->C.dx = g->lx / g->nx;
  for (int m = 0; m < 5; ++m) x->C.ref[m] = x->C.shock_ref[m] = 0.0;
  x->C.x_foot = 0.0;
  x->C.df_p = 0.0;
  x->B.df_prof = nullptr;
  x->B.df_psi = nullptr;
  char* ws = (char*)workspace;
  Nodes<double>& N64 = x->B.n64;
  Nodes<float>& N32 = x->B.n32;
  N64 = Nodes<double>{};
  N32 = Nodes<float>{};
  if (L.mixed) {
    double** f64[9] = {&N64.rho, &N64.u, &N64.v, &N64.w, &N64.p, &N64.T, &N64.H, &N64.srho, &N64.theta};
    for (int f = 0; f < 9; ++f) *f64[f] = (double*)(ws + L.off_n64[f]);
    for (int dd = 0; dd < 3; ++dd) {
      x->B.mom[dd] = (double*)(ws + L.off_n64[9 + dd]);
      x->B.mflux[dd] = (double*)(ws + L.off_n64[12 + dd]);
    }
    float** f32[kN32Mixed] = {&N32.rho, &N32.u, &N32.v, &N32.w, &N32.p, &N32.T,
                              &N32.H,   &N32.c, &N32.mu, &N32.theta, &N32.div};
    for (int f = 0; f < kN32Mixed; ++f) *f32[f] = (float*)(ws + L.off_n32[f]);
    for (int f = 0; f < kN32Xdev; ++f) x->B.xdev[f] = (float*)(ws + L.off_xdev[f]);
    x->B.xref = (float*)(ws + L.off_xref);
  } else {
    for (int f = 0; f < kN32Xdev; ++f) x->B.xdev[f] = nullptr;
    x->B.xref = nullptr;
    double** f64[12] = {&N64.rho, &N64.u, &N64.v,  &N64.w,     &N64.p,   &N64.T,
                        &N64.H,   &N64.c, &N64.mu, &N64.theta, &N64.div, &N64.srho};
    for (int f = 0; f < 12; ++f) *f64[f] = (double*)(ws + L.off_n64[f]);
    for (int f = 0; f < 6; ++f) x->B.lam[f] = (double*)(ws + L.off_n64[12 + f]);
    for (int dd = 0; dd < 3; ++dd) {
      x->B.mom[dd] = (double*)(ws + L.off_n64[18 + dd]);
      x->B.mflux[dd] = (double*)(ws + L.off_n64[21 + dd]);
    }
  }
  for (int dir = 0; dir < 3; ++dir) {
    x->B.fh64[dir] = L.mixed ? nullptr : (double*)(ws + L.off_fh[dir]);
    x->B.fh32[dir] = L.mixed ? (float*)(ws + L.off_fh[dir]) : nullptr;
    x->B.wl[dir] = (int*)(ws + L.off_wl[dir]);
    x->B.cl[dir] = (int*)(ws + L.off_cl[dir]);
  }
  x->B.R = (double*)(ws + L.off_R);
  x->B.wcount = (unsigned*)(ws + L.off_wcount);
  x->B.red = (double*)(ws + L.off_red);
  x->B.scal = (double*)(ws + L.off_scal);
  double* met = (double*)(ws + L.off_metric);
  float* met32 = (float*)(ws + L.off_metric32);
  x->B.m64.inv_hy = met;
  x->B.m64.c2y = met + g->ny;
  x->B.m64.c1y = met + 2 * g->ny;
  x->B.vol = met + 3 * g->ny;
  x->B.hy = met + 4 * g->ny;
  x->B.c1h = met + 5 * g->ny;
  x->B.ubar = met + 6 * g->ny;
  x->B.grad = L.mixed ? nullptr : (double*)(ws + L.off_grad);
  x->B.band = L.mixed ? (int*)(ws + L.off_band) : nullptr;
  x->d.dbg = (unsigned*)(ws + L.off_dbg);
  x->B.m32.inv_hy = met32;
  x->B.m32.c2y = met32 + g->ny;
  x->B.m32.c1y = met32 + 2 * g->ny;
  build_metrics(x);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(met, x->metric_host.data(), sizeof(double) * 6 * g->ny,
                        cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(met32, x->metric_host32.data(), sizeof(float) * 3 * g->ny,
                        cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->B.scal, 0, sizeof(double) * kScalCount, x->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->B.wcount, 0, 8 * sizeof(unsigned), x->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->d.dbg, 0, sizeof(unsigned), x->stream);
  if (e != cudaSuccess) {
    delete x;
    return fail(STRM_ECUDA, std::string("init: ") + cudaGetErrorString(e));
  }
  x->weno_grid = sms * 8;
  *out = x;
  return STRM_OK;
}

int strm_set_bc(strm_ctx* x, int face, int kind, const double* params, int nparams) {
  if (!x) return fail(STRM_EINVAL, "null context");
  Consts& C = x->C;
  auto need = [&](int n) { return params && nparams == n; };
  auto set_ref = [&](double* dst) {
    for (int m = 0; m < 5; ++m) dst[m] = params[m];
    return params[0] > 0 && params[4] > 0;
  };
  switch (face) {
    case STRM_FACE_YMIN_YMAX:
      if (kind != STRM_BC_PERIODIC && kind != STRM_BC_WALL_ISOTHERMAL)
        return fail(STRM_EINVAL, "both y faces take periodic or wall");
      if (params || nparams) return fail(STRM_EINVAL, "periodic and wall faces take no params");
      if (kind == STRM_BC_WALL_ISOTHERMAL && x->g.ny < G) return fail(STRM_EINVAL, "walls need ny >= 3");
      C.bc[2] = C.bc[3] = kind == STRM_BC_PERIODIC ? kBcPeriodic : kBcWall;
      break;
    case STRM_FACE_XMIN:
    case STRM_FACE_XMAX:
    case STRM_FACE_YMIN:
    case STRM_FACE_YMAX: {
      int slot = face - STRM_FACE_XMIN;  // 0 xmin, 1 xmax, 2 ymin, 3 ymax
      bool xface = slot < 2;
      if (kind == STRM_BC_PERIODIC) {
        if (params || nparams) return fail(STRM_EINVAL, "periodic faces take no params");
        C.bc[slot] = kBcPeriodic;
      } else if (kind == STRM_BC_WALL_ISOTHERMAL) {
        if (xface) return fail(STRM_EINVAL, "walls are y faces");
        if (params || nparams) return fail(STRM_EINVAL, "wall faces take no params");
        if (x->g.ny < G) return fail(STRM_EINVAL, "walls need ny >= 3");
        C.bc[slot] = kBcWall;
      } else if (kind == STRM_BC_CHARACTERISTIC) {
        if (!need(5) || !set_ref(C.ref)) return fail(STRM_EINVAL, "characteristic faces take 5 params: rho u v w p (rho, p > 0)");
        C.bc[slot] = kBcChar;
        if (slot == 3) C.shock = 0;
      } else if (kind == STRM_BC_RECYCLE_INFLOW) {
        if (slot != 0) return fail(STRM_EINVAL, "recycling inflow is an x-min face");
        if (!need(7) || !set_ref(C.ref)) return fail(STRM_EINVAL, "recycling inflow takes 7 params: rho u v w p i_recycle delta_in");
        int ir = (int)params[5];
        if (ir != params[5] || ir < G - 1 || ir >= x->g.nx || !(params[6] > 0))
          return fail(STRM_EINVAL, "recycling plane must be an interior x index >= 2 and delta_in > 0");
        C.i_recycle = ir;
        C.delta_in = params[6];
        C.bc[0] = kBcRecycle;
      } else if (kind == STRM_BC_DF_INFLOW) {
        return fail(STRM_EINVAL, "digital-filter inflow faces are set with strm_set_inflow_df");
      } else if (kind == STRM_BC_SHOCK_TOP) {
        if (slot != 3) return fail(STRM_EINVAL, "the oblique-shock reference is a y-max face");
        if (!need(7) || !set_ref(C.ref)) return fail(STRM_EINVAL, "shock top takes 7 params: rho u v w p theta x_imp");
        double beta, pr, rr, m2;
        double c1 = std::sqrt(C.gamma * params[4] / params[0]);
        if (!oblique_shock(C.gamma, params[1] / c1, params[5], &beta, &pr, &rr, &m2))
          return fail(STRM_EINVAL, "deflection beyond the attached oblique-shock limit");
        // post-shock state: the stream deflected by theta toward the wall, shock foot on the top
        double V1 = params[1], un1 = V1 * std::sin(beta), ut = V1 * std::cos(beta), un2 = un1 / rr;
        C.shock_ref[0] = params[0] * rr;
        C.shock_ref[1] = ut * std::cos(beta) + un2 * std::sin(beta);
        C.shock_ref[2] = -ut * std::sin(beta) + un2 * std::cos(beta);
        C.shock_ref[3] = 0.0;
        C.shock_ref[4] = params[4] * pr;
        C.x_foot = params[6] - x->g.ly / std::tan(beta);
        C.shock = 1;
        C.bc[3] = kBcChar;
      } else {
        return fail(STRM_EINVAL, "unknown boundary kind");
      }
      break;
    }
    default:
      return fail(STRM_EINVAL, "unknown face");
  }
  if (x->gexec) {  // the captured graph holds the old constants
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  return STRM_OK;
}

int strm_compute_rhs(strm_ctx* x, const double* w, double* rhs) {
  if (!x || !w || !rhs) return fail(STRM_EINVAL, "null context or buffer");
  if (w == rhs) return fail(STRM_EINVAL, "w and rhs must not alias");
  int rc = enqueue_rhs(x, w, rhs, false, 0.0, 0.0, x->stream);
  if (rc) return rc;
  cudaStream_t st = x->stream;
  if (x->C.forcing) STRM_LAUNCH(STRM_K_FORCE, launch_apply_forcing(x->d, x->B, rhs, st));
  STRM_CK_LAUNCH();
  return STRM_OK;
}

namespace {

size_t stats_rows(const strm_ctx* x, int mode) {
  return mode == STRM_STATS_XZ ? (size_t)x->d.ny : (size_t)x->d.ny * x->d.nx;
}

int enqueue_stats(strm_ctx* x, const double* w) {
  launch_stats(x->d, x->C, w, x->st_acc, x->st_scr, x->st_mode, x->stream);
  x->launches += x->st_mode == STRM_STATS_XZ ? 2 : 1;
  STRM_CK_LAUNCH();
  ++x->st_samples;
  return STRM_OK;
}

// one step taken: sample if the automatic sampling is due
int after_step(strm_ctx* x, const double* w) {
  ++x->st_steps;
  if (x->st_acc && x->st_every > 0 && x->st_steps % x->st_every == 0) return enqueue_stats(x, w);
  return STRM_OK;
}

}  // namespace

int strm_rk_step(strm_ctx* x, double* w, double* r_old, double dt, double cfl) {
  int rc = check_step_args(x, w, r_old, dt, cfl);
  if (rc) return rc;
  rc = enqueue_step(x, w, r_old, dt, cfl, x->stream);
  if (rc) return rc;
  return after_step(x, w);
}

int strm_advance_n(strm_ctx* x, double* w, double* r_old, int nsteps, double dt, double cfl) {
  int rc = check_step_args(x, w, r_old, dt, cfl);
  if (rc) return rc;
  if (nsteps < 0) return fail(STRM_EINVAL, "nsteps < 0");
  if (nsteps == 0) return STRM_OK;
  if (x->timing) {  // event timing needs eager launches
    for (int n = 0; n < nsteps; ++n) {
      int erc = enqueue_step(x, w, r_old, dt, cfl, x->stream);
      if (!erc) erc = after_step(x, w);
      if (erc) return erc;
    }
    return STRM_OK;
  }
  if (!x->gexec || x->g_w != w || x->g_r != r_old || x->g_dt != dt || x->g_cfl != cfl) {
    if (x->gexec) {
      STRM_CK(cudaGraphExecDestroy(x->gexec));
      x->gexec = nullptr;
    }
    if (!x->cap) STRM_CK(cudaStreamCreateWithFlags(&x->cap, cudaStreamNonBlocking));
    // capture on a private stream; the graph itself is launched on the caller's stream
    STRM_CK(cudaStreamBeginCapture(x->cap, cudaStreamCaptureModeThreadLocal));
    long long before = x->launches;
    int erc = enqueue_step(x, w, r_old, dt, cfl, x->cap);
    x->graph_kernels = x->launches - before;
    x->launches = before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(x->cap, &graph);
    if (erc) {
      if (graph) cudaGraphDestroy(graph);
      return erc;
    }
    if (e != cudaSuccess) return fail(STRM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&x->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(STRM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    x->g_w = w;
    x->g_r = r_old;
    x->g_dt = dt;
    x->g_cfl = cfl;
  }
  for (int n = 0; n < nsteps; ++n) {
    STRM_CK(cudaGraphLaunch(x->gexec, x->stream));
    x->launches += x->graph_kernels;
    int src = after_step(x, w);
    if (src) return src;
  }
  return STRM_OK;
}

namespace {

// The device address of a page-locked host buffer of `bytes` bytes that is mapped into the
// device's address space, or null: both its first and its last element must map, at the same
// offset, and it must be 16-byte aligned. A pointer that is not mapped (pageable memory) leaves
// no error behind.
double* mapped_host(double* h, size_t bytes) {
  void* a = nullptr;
  void* b = nullptr;
  if ((uintptr_t)h & 15) return nullptr;
  if (cudaHostGetDevicePointer(&a, h, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&b, (char*)h + bytes - sizeof(double), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if ((char*)b - (char*)a != (ptrdiff_t)(bytes - sizeof(double)) || ((uintptr_t)a & 15)) return nullptr;
  return (double*)a;
}

bool is_device_memory(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

int strm_advance_n_host(strm_ctx* x, double* w_host, double* w, double* r_old, int nsteps, double dt,
                        double cfl) {
  if (!x || !w_host) return fail(STRM_EINVAL, "null context or host buffer");
  if (!w || !r_old || w == r_old) return fail(STRM_EINVAL, "null or aliased device state buffers");
  const size_t bytes = sizeof(double) * 5 * (size_t)x->d.N;
  const long long n = 5 * x->d.N;
  const int sms = x->weno_grid / 8;
  // a mapped page-locked buffer is copied by kernels through its device address, any other
  // host memory by the copy engines
  double* hd = is_device_memory(w) ? mapped_host(w_host, bytes) : nullptr;
  if (hd) {
    launch_copy_mapped(hd, w, n, sms, x->stream);
    x->launches += 1;
    STRM_CK(cudaGetLastError());
  } else {
    STRM_CK(cudaMemcpyAsync(w, w_host, bytes, cudaMemcpyHostToDevice, x->stream));
  }
  int rc = strm_advance_n(x, w, r_old, nsteps, dt, cfl);
  if (rc) return rc;
  if (hd) {
    launch_copy_mapped(w, hd, n, sms, x->stream);
    x->launches += 1;
    STRM_CK(cudaGetLastError());
  } else {
    STRM_CK(cudaMemcpyAsync(w_host, w, bytes, cudaMemcpyDeviceToHost, x->stream));
  }
  STRM_CK(cudaStreamSynchronize(x->stream));
  return STRM_OK;
}

namespace {

struct DFLayout {
  size_t prof, by, bz, t, psi, count, total;
};

bool df_layout(const strm_ctx* x, const strm_df* P, DFLayout* L) {
  if (!x || !P || P->ny_filter < 1 || P->nz_filter < 1 || !(P->tau > 0) || !(P->p_ref > 0)) return false;
  size_t ny = x->d.ny, plane = (size_t)x->d.nz * x->d.ny, off = 0;
  L->prof = off;
  off = align_up(off + sizeof(double) * 7 * ny);
  L->by = off;
  off = align_up(off + sizeof(double) * (4 * (size_t)P->ny_filter + 1));
  L->bz = off;
  off = align_up(off + sizeof(double) * (4 * (size_t)P->nz_filter + 1));
  L->t = off;
  off = align_up(off + sizeof(double) * 3 * plane);
  L->psi = off;
  off = align_up(off + sizeof(double) * 3 * plane);
  L->count = off;
  off = align_up(off + sizeof(unsigned long long));
  L->total = off;
  return true;
}

// filter coefficients b_l = exp(-pi l^2 / (2 n^2)), l = -2n..2n, scaled to unit sum of squares
void df_coefs(int n, double* b) {
  const double pi = std::acos(-1.0);
  double s = 0.0;
  for (int l = -2 * n; l <= 2 * n; ++l) {
    b[l + 2 * n] = std::exp(-pi * l * l / (2.0 * n * n));
    s += b[l + 2 * n] * b[l + 2 * n];
  }
  double r = 1.0 / std::sqrt(s);
  for (int l = 0; l <= 4 * n; ++l) b[l] *= r;
}

}  // namespace

size_t strm_inflow_df_bytes(const strm_ctx* x, const strm_df* P) {
  DFLayout L;
  return df_layout(x, P, &L) ? L.total : 0;
}

int strm_set_inflow_df(strm_ctx* x, const strm_df* P, const double* prof, void* buffer, size_t bytes) {
  if (!x) return fail(STRM_EINVAL, "null context");
  DFLayout L;
  if (!df_layout(x, P, &L)) return fail(STRM_EINVAL, "bad inflow parameters (filter widths >= 1, tau > 0, p_ref > 0)");
  if (!prof || !buffer) return fail(STRM_EINVAL, "null profiles or buffer");
  if (bytes < L.total) return fail(STRM_ENOMEM, "inflow buffer too small: need " + std::to_string(L.total));
  if ((uintptr_t)buffer & 7) return fail(STRM_EINVAL, "inflow buffer not 8-byte aligned");
  if (x->C.bc[1] == kBcPeriodic) return fail(STRM_EINVAL, "an inflow face needs a non-periodic x-max face");
  const int ny = x->d.ny;
  const int nby = 4 * P->ny_filter + 1, nbz = 4 * P->nz_filter + 1;
  // host copies: U, V, T and the Cholesky factors a11, a21, a22, a33 per j, then the filters
  x->df_host.assign(7 * (size_t)ny + nby + nbz, 0.0);
  double* h = x->df_host.data();
  for (int j = 0; j < ny; ++j) {
    double R11 = prof[3 * ny + j], R12 = prof[4 * ny + j], R22 = prof[5 * ny + j], R33 = prof[6 * ny + j];
    if (!(R11 >= 0) || !(R22 >= 0) || !(R33 >= 0) || !(prof[2 * ny + j] > 0))
      return fail(STRM_EINVAL, "inflow profiles: T > 0 and non-negative normal stresses required");
    double a11 = std::sqrt(R11), a21 = a11 > 0 ? R12 / a11 : 0.0;
    double r22 = R22 - a21 * a21;
    if (r22 < -1e-12 * (R22 + 1e-300)) return fail(STRM_EINVAL, "inflow Reynolds stresses not positive semi-definite");
    h[j] = prof[j];
    h[ny + j] = prof[ny + j];
    h[2 * ny + j] = prof[2 * ny + j];
    h[3 * ny + j] = a11;
    h[4 * ny + j] = a21;
    h[5 * ny + j] = std::sqrt(std::max(r22, 0.0));
    h[6 * ny + j] = std::sqrt(R33);
  }
  df_coefs(P->ny_filter, h + 7 * ny);
  df_coefs(P->nz_filter, h + 7 * ny + nby);
  char* b = (char*)buffer;
  DFParams& F = x->df;
  F.ny = P->ny_filter;
  F.nz = P->nz_filter;
  F.tau = P->tau;
  F.seed = P->seed;
  F.by = (const double*)(b + L.by);
  F.bz = (const double*)(b + L.bz);
  F.t = (double*)(b + L.t);
  F.psi = (double*)(b + L.psi);
  F.count = (unsigned long long*)(b + L.count);
  cudaStream_t st = x->stream;
  STRM_CK(cudaMemcpyAsync(b + L.prof, h, sizeof(double) * 7 * ny, cudaMemcpyHostToDevice, st));
  STRM_CK(cudaMemcpyAsync(b + L.by, h + 7 * ny, sizeof(double) * nby, cudaMemcpyHostToDevice, st));
  STRM_CK(cudaMemcpyAsync(b + L.bz, h + 7 * ny + nby, sizeof(double) * nbz, cudaMemcpyHostToDevice, st));
  STRM_CK(cudaMemsetAsync(F.count, 0, sizeof(unsigned long long), st));
  x->C.bc[0] = kBcDigitalFilter;
  x->C.df_p = P->p_ref;
  x->B.df_prof = (const double*)(b + L.prof);
  x->B.df_psi = F.psi;
  launch_df_update(x->d, F, x->B, true, st);
  x->launches += 2;
  STRM_CK_LAUNCH();
  if (x->gexec) {  // the captured graph holds the old constants
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  return STRM_OK;
}

size_t strm_stats_bytes(const strm_ctx* x, int mode) {
  if (!x || (mode != STRM_STATS_XZ && mode != STRM_STATS_Z)) return 0;
  size_t acc = align_up(sizeof(double) * STRM_NSTAT * stats_rows(x, mode));
  size_t scr = mode == STRM_STATS_XZ ? align_up(sizeof(double) * STRM_NSTAT * (size_t)x->d.nx * x->d.ny) : 0;
  return acc + scr;
}

int strm_stats_bind(strm_ctx* x, int mode, void* buffer, size_t bytes) {
  if (!x) return fail(STRM_EINVAL, "null context");
  x->st_samples = 0;
  x->st_steps = 0;
  if (!buffer) {
    x->st_acc = x->st_scr = nullptr;
    return STRM_OK;
  }
  size_t need = strm_stats_bytes(x, mode);
  if (!need) return fail(STRM_EINVAL, "unknown statistics mode");
  if (bytes < need) return fail(STRM_ENOMEM, "statistics buffer too small: need " + std::to_string(need));
  if ((uintptr_t)buffer & 7) return fail(STRM_EINVAL, "statistics buffer not 8-byte aligned");
  x->st_mode = mode;
  x->st_acc = (double*)buffer;
  x->st_scr = mode == STRM_STATS_XZ
                  ? (double*)((char*)buffer + align_up(sizeof(double) * STRM_NSTAT * stats_rows(x, mode)))
                  : nullptr;
  STRM_CK(cudaMemsetAsync(x->st_acc, 0, sizeof(double) * STRM_NSTAT * stats_rows(x, mode), x->stream));
  return STRM_OK;
}

int strm_stats_sample(strm_ctx* x, const double* w) {
  if (!x || !w) return fail(STRM_EINVAL, "null context or state");
  if (!x->st_acc) return fail(STRM_EINVAL, "no statistics buffer bound");
  return enqueue_stats(x, w);
}

int strm_stats_every(strm_ctx* x, int k) {
  if (!x) return fail(STRM_EINVAL, "null context");
  if (k < 0) return fail(STRM_EINVAL, "sampling interval < 0");
  x->st_every = k;
  x->st_steps = 0;
  return STRM_OK;
}

int strm_stats_read(strm_ctx* x, double* out_host, long long* nsamples_host) {
  if (!x || !out_host) return fail(STRM_EINVAL, "null context or output");
  if (!x->st_acc) return fail(STRM_EINVAL, "no statistics buffer bound");
  size_t n = STRM_NSTAT * stats_rows(x, x->st_mode);
  STRM_CK(cudaMemcpyAsync(out_host, x->st_acc, sizeof(double) * n, cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaStreamSynchronize(x->stream));
  double inv = x->st_samples > 0 ? 1.0 / (double)x->st_samples : 0.0;
  for (size_t q = 0; q < n; ++q) out_host[q] *= inv;
  if (nsamples_host) *nsamples_host = x->st_samples;
  return STRM_OK;
}

int strm_convert_f64_f32(const double* x, float* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(STRM_EINVAL, "bad conversion arguments");
  if (n == 0) return STRM_OK;
  launch_d2f(x, y, n, (cudaStream_t)stream);
  STRM_CK(cudaGetLastError());
  return STRM_OK;
}

int strm_convert_f32_f64(const float* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(STRM_EINVAL, "bad conversion arguments");
  if (n == 0) return STRM_OK;
  launch_f2d(x, y, n, (cudaStream_t)stream);
  STRM_CK(cudaGetLastError());
  return STRM_OK;
}

int strm_set_overlap(strm_ctx* x, int mode) {
  if (!x) return fail(STRM_EINVAL, "null context");
  if (mode & ~(STRM_OVERLAP_GHOST | STRM_OVERLAP_FACES)) return fail(STRM_EINVAL, "unknown overlap bits");
  if (mode && !x->side[0]) {
    for (int b = 0; b < 2; ++b) STRM_CK(cudaStreamCreateWithFlags(&x->side[b], cudaStreamNonBlocking));
    for (int e = 0; e < 5; ++e) STRM_CK(cudaEventCreateWithFlags(&x->ev[e], cudaEventDisableTiming));
  }
  x->overlap = mode;
  if (x->gexec) {  // the captured graph has the other launch structure
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  return STRM_OK;
}

int strm_set_theta(strm_ctx* x, const double* theta) {
  if (!x) return fail(STRM_EINVAL, "null context");
  if (theta && x->C.weno_mode != STRM_WENO_SENSOR)
    return fail(STRM_EINVAL, "a prescribed switch input needs the sensor mode (STRM_WENO_SENSOR)");
  x->theta_fixed = theta;
  if (x->gexec) {  // the captured graph has the other launch structure
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  return STRM_OK;
}

int strm_debug_build(void) { return kDebug ? 1 : 0; }

int strm_debug_flags(strm_ctx* x, unsigned* flags_host) {
  if (!x || !flags_host) return fail(STRM_EINVAL, "null context or output");
  STRM_CK(cudaMemcpyAsync(flags_host, x->d.dbg, sizeof(unsigned), cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaStreamSynchronize(x->stream));
  return STRM_OK;
}

int strm_conserved_totals(strm_ctx* x, const double* w, double out_host[5]) {
  if (!x || !w || !out_host) return fail(STRM_EINVAL, "null argument");
  launch_totals(x->d, x->B, w, x->stream);
  STRM_CK_LAUNCH();
  STRM_CK(cudaMemcpyAsync(out_host, x->B.scal + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaStreamSynchronize(x->stream));
  for (int m = 0; m < 5; ++m)
    if (!std::isfinite(out_host[m])) return fail(STRM_ENONFINITE, "non-finite conserved total");
  return STRM_OK;
}

int strm_get_time(strm_ctx* x, double* t_host, double* dt_host) {
  if (!x) return fail(STRM_EINVAL, "null context");
  double v[2];
  STRM_CK(cudaMemcpyAsync(&v[0], x->B.scal + kScalTime, sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaMemcpyAsync(&v[1], x->B.scal + kScalDt, sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaStreamSynchronize(x->stream));
  if (t_host) *t_host = v[0];
  if (dt_host) *dt_host = v[1];
  // a non-finite state makes the CFL maximum, hence dt and the time, non-finite
  if (!std::isfinite(v[0]) || !std::isfinite(v[1]))
    return fail(STRM_ENONFINITE, "non-finite time step: the state is not finite");
  return STRM_OK;
}

int strm_set_time(strm_ctx* x, double t) {
  if (!x) return fail(STRM_EINVAL, "null context");
  x->time_host[0] = t;
  x->time_host[1] = 0.0;
  STRM_CK(cudaMemcpyAsync(x->B.scal + kScalTime, &x->time_host[0], sizeof(double), cudaMemcpyHostToDevice, x->stream));
  STRM_CK(cudaMemcpyAsync(x->B.scal + kScalDt, &x->time_host[1], sizeof(double), cudaMemcpyHostToDevice, x->stream));
  return STRM_OK;
}

int strm_sensor(strm_ctx* x, const double* w, double* theta, double* div, unsigned char* fx,
                unsigned char* fy, unsigned char* fz) {
  if (!x || !w) return fail(STRM_EINVAL, "null context or state");
  STRM_CK(cudaMemsetAsync(x->B.wcount, 0, 8 * sizeof(unsigned), x->stream));
  launch_prims(x->d, x->C, x->B, w, false, x->stream);
  if (x->C.bc[0] == kBcRecycle) launch_recycle(x->d, x->C, x->B, x->stream);
  launch_ghost_prims(x->d, x->C, x->B, x->stream);
  launch_sensor(x->d, x->C, x->B, 0, x->stream);
  if (x->C.mixed && x->C.weno_mode == 1 && !x->theta_fixed) launch_band_theta(x->d, x->C, x->B, x->stream);
  if (x->theta_fixed) launch_theta_set(x->d, x->B, x->theta_fixed, x->stream);
  launch_ghost_scalars(x->d, x->C, x->B, x->stream);
  launch_export_sensor(x->d, x->C, x->B, theta, div, x->stream);
  unsigned char* fl[3] = {fx, fy, fz};
  for (int dir = 0; dir < 3; ++dir)
    if (fl[dir]) launch_flags(x->d, x->C, x->B, dir, fl[dir], x->stream);
  STRM_CK_LAUNCH();
  return STRM_OK;
}

int strm_weno_counts(strm_ctx* x, long long counts_host[3]) {
  if (!x || !counts_host) return fail(STRM_EINVAL, "null argument");
  unsigned c[4];
  STRM_CK(cudaMemcpyAsync(c, x->B.wcount, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, x->stream));
  STRM_CK(cudaStreamSynchronize(x->stream));
  for (int d = 0; d < 3; ++d) counts_host[d] = c[d];
  return STRM_OK;
}

const char* strm_kernel_name(int k) {
  return (k >= 0 && k < STRM_K_COUNT) ? kKernelNames[k] : "";
}

int strm_timing(strm_ctx* x, int enable) {
  if (!x) return fail(STRM_EINVAL, "null context");
  int rc = fold_timing(x);
  if (rc) return rc;
  for (int k = 0; k < STRM_K_COUNT; ++k) {
    x->kms[k] = 0.0;
    x->klaunch[k] = 0;
  }
  for (int d = 0; d < 3; ++d) x->weno_faces[d] = 0;
  x->timing = enable != 0;
  return STRM_OK;
}

int strm_timing_read(strm_ctx* x, double* ms_host, long long* launches_host, long long* weno_faces_host) {
  if (!x) return fail(STRM_EINVAL, "null context");
  int rc = fold_timing(x);
  if (rc) return rc;
  for (int k = 0; k < STRM_K_COUNT; ++k) {
    if (ms_host) ms_host[k] = x->kms[k];
    if (launches_host) launches_host[k] = x->klaunch[k];
  }
  if (weno_faces_host)
    for (int d = 0; d < 3; ++d) weno_faces_host[d] = x->weno_faces[d];
  return STRM_OK;
}

int strm_launch_count(strm_ctx* x, long long* launches_host) {
  if (!x || !launches_host) return fail(STRM_EINVAL, "null argument");
  *launches_host = x->launches;
  return STRM_OK;
}

}  // extern "C"

// Internal: the per-grid pieces of a context, for the batched ensemble.
void strm::ctx_parts(strm_ctx* x, Dims* d, Consts* C, Bufs* B, int* sms) {
  *d = x->d;
  *C = x->C;
  *B = x->B;
  *sms = x->weno_grid / 8;
}

bool strm::ctx_df(strm_ctx* x, DFParams* F) {
  if (x->C.bc[0] != kBcDigitalFilter) return false;
  *F = x->df;
  return true;
}

extern "C" {

void strm_destroy(strm_ctx* x) {
  if (!x) return;
  for (cudaEvent_t e : x->events) cudaEventDestroy(e);
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  if (x->cap) cudaStreamDestroy(x->cap);
  for (cudaStream_t sd : x->side)
    if (sd) cudaStreamDestroy(sd);
  for (cudaEvent_t e : x->ev)
    if (e) cudaEventDestroy(e);
  delete x;
}

}  // extern "C"
