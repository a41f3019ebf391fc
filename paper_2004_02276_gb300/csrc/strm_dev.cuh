// Device-side layout, constants and shared device functions of the sm_103a library.
//
// Layout in HBM
//   state w, residual R, RK register: SoA [5][nz][ny][nx] FP64 (interior only, caller-owned)
//   node fields (workspace): ghosted [nz+2G][ny+2G][px]; the interior node (i,j,k) sits at
//     ((k+G)*py + j+G)*px + i+GX; GX = 4 keeps interior rows 32-byte aligned, px is a multiple
//     of 4. FP64 precision keeps every node field in FP64. Mixed precision keeps the fields the
//     characteristic projection reads (rho, u, v, w, p, T, H, sqrt rho, and in both precisions
//     rho u_d and rho u_d^2 + p) in FP64 and FP32 copies of all fields for the FP32 kernels.
//   interface fluxes (workspace): x faces [5][nz][ny][nx+1], y faces [5][nz][ny+1][nx],
//     z faces [5][nz+1][ny][nx] (FP64, or FP32 in mixed precision); face s along a direction
//     lies between nodes s-1 and s.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

// Read-only loads of the bodies. A translation unit whose kernels read, after a grid-wide
// barrier, data that other blocks of the same launch wrote defines STRM_COHERENT_LOADS before
// including this header: the non-coherent read-only path (ld.global.nc) is only defined for
// data that no thread writes during the kernel, so there the loads are ordinary ones.
#ifdef STRM_COHERENT_LOADS
#define STRM_LDG(p) (*(p))
#define STRM_RO
#else
#define STRM_LDG(p) __ldg(p)
#define STRM_RO __restrict__
#endif

namespace strm {

constexpr int G = 3;   // ghost layers (central L <= 3, six-node WENO5 stencil)
constexpr int GX = 4;  // x offset of the interior in a ghosted row
constexpr int kRedBlock = 256;
// faces per thread of the y/z central-flux sweeps (body_central_sweep)
constexpr int kSweepSeg = 64;

struct Dims {
  int nx, ny, nz;
  int px, py, pz;     // ghosted extents (px padded)
  long long plane;    // px * py
  long long ng;       // px * py * pz
  long long N;        // nx * ny * nz
  long long nf[3];    // faces per direction
  int slab_ty;        // rows per slab of the slab traversal order (0: natural order), see slab_rows
  int zslab_ty;       // the same for the z-face kernels (zface_order)
  unsigned* dbg;      // debug builds: the context's error word (see kDebug)
};

// Slab heights the slab traversal order admits for an nx x ny grid: TY rows with ny % TY == 0
// and nx TY a multiple of 256 (a block's 256 elements then stay inside one slab-plane, so the
// element count of every block is unchanged and reductions keep their partitions' sizes).
constexpr bool slab_rows_allowed(int nx, int ny, int ty) {
  return ty > 0 && ny % ty == 0 && ((long long)nx * ty) % 256 == 0;
}

// The largest admitted slab height not above cap (32, 16 or 8), or 0 for the natural order.
constexpr int slab_rows_for(int nx, int ny, int cap) {
  for (int ty = 32; ty >= 8; ty >>= 1)
    if (ty <= cap && slab_rows_allowed(nx, ny, ty)) return ty;
  return 0;
}

// Ghosted node fields of one precision.
template <typename R>
struct Nodes {
  R *rho, *u, *v, *w, *p, *T, *H, *c, *mu, *srho, *theta, *div;
};

// Per-j wall-normal metrics: 1/(y_eta deta), 1/(y_eta deta)^2, y_etaeta/(y_eta^3 deta).
template <typename R>
struct Metric {
  const R *inv_hy, *c2y, *c1y;
};

// Scheme and gas coefficients in the arithmetic precision of a kernel.
template <typename R>
struct Coefs {
  R a[4], b[4];                      // central first/second-derivative coefficients, 1..L
  R ax[4], az[4];                    // a_l / dx and a_l / dz (first derivatives along x and z)
  R bx[4], bz[4];                    // b_l / dx^2 and b_l / dz^2, l = 0..L (second derivatives)
  R bxz0;                            // bx[0] + bz[0]
  R aq[4];                           // a_l / 4 (pair weights of the split central flux)
  R ap[4];                           // a_{r+1} + .. + a_L, r = 0..L-1 (its pressure part)
  R inv_dx, inv_dz, inv_dx2, inv_dz2;
  R cp_pr, sens_eps, theta_thr, weno_eps;
  R gamma, gm1, r_gas, cp, t_wall, mu_ref, inv_tref, visc_exp, suth_s;
  int exp_19_25;  // the power-law exponent is 0.76 = 19/25 (fast route, pow_19_25)
};

// Face kinds: x faces periodic, recycling inflow (x-min) or characteristic; y faces periodic,
// isothermal wall or characteristic (y-max optionally with the post-shock reference state
// downstream of the shock foot), digital-filter inflow (x-min); z periodic.
enum { kBcPeriodic = 0, kBcWall = 1, kBcChar = 2, kBcRecycle = 3, kBcDigitalFilter = 4 };

struct Consts {
  // gas (FP64)
  double gamma, gm1, r_gas, inv_r, cv, inv_cv, cp, cp_pr;
  double mu_ref, inv_tref, visc_exp, suth_s, t_wall;
  int visc_law, forcing;
  // boundaries: kinds of the x-min, x-max, y-min, y-max faces; reference primitives
  // (rho, u, v, w, p) of characteristic faces; oblique shock; recycling inflow
  int bc[4];
  double ref[5];
  int shock;
  double shock_ref[5], x_foot;
  int i_recycle;
  double delta_in, dx;
  double df_p;  // pressure of the digital-filter inflow ghosts
  // mixed precision: the FP32 pressure copy holds p - p_shift (p_shift = R t_ref rounded to
  // FP32, the reference pressure of the channel and boundary-layer units). A constant added to
  // the pressure of every face flux cancels exactly in the flux differences, so the FP32 copy
  // keeps the precision of the pressure's variations instead of its magnitude; the mixed WENO
  // faces subtract the same constant from their normal momentum flux.
  double p_shift;
  // scheme
  int L, weno_mode, convective, viscous, mixed;
  double vtot;  // total metric volume
  Coefs<double> k64;
  Coefs<float> k32;
};

struct Bufs {
  Nodes<double> n64;
  Nodes<float> n32;
  double* fh64[3];                              // interface fluxes (FP64 precision)
  float* fh32[3];                               // interface fluxes (mixed precision)
  double* R;                                    // residual, 5*N
  int* wl[3];                                   // compacted WENO face lists
  int* cl[3];                                   // compacted central face lists
  unsigned int* wcount;                         // [0..2] WENO list lengths, [4..6] central
  double* red;                                  // reduction partials
  double* scal;                                 // device scalars, see kScal*
  Metric<double> m64;
  Metric<float> m32;
  const double* vol;                            // node volume dx (y_eta deta) dz per j
  const double* hy;                             // node height above the wall eta = 0, per j
  const double* c1h;                            // y_etaeta / y_eta^2 per j (FP64)
  int* band;                                    // mixed: interior nodes whose FP32 theta is near
                                                //   the threshold (count in wcount[3])
  double* lam[6];                               // FP64: u - c, u + c, v - c, v + c, w - c, w + c
                                                //   at the nodes (ghosted), for the LF speeds
  double* mom[3];                               // rho u, rho v, rho w at the nodes (ghosted, FP64
                                                //   in both precisions), for the WENO projection
  double* mflux[3];                             // rho u_d^2 + p, d = x, y, z (the normal momentum
                                                //   flux; ghosted, FP64), for the WENO projection
  float* xdev[3];                               // mixed: rho, u, H less their x-row reference
                                                //   (ghosted; x rows only), for the x faces'
                                                //   central flux, see central_flux_xdev
  float* xref;                                  // mixed: [3][nz][ny] the reference of each x row
                                                //   (rho, u, H of its first node, FP32)
  double* grad;                                 // FP64: velocity gradients d_b u_a at the
                                                //   interior nodes, [3a + b][N], from the sensor
  double* ubar;                                 // spanwise-mean u at the recycling plane, per j
  // digital-filter inflow: per j U, V, T and the Cholesky factors a11, a21, a22, a33 of the
  // Reynolds stresses ([7][ny]), and the time-correlated fluctuation plane [3][nz][ny]
  const double* df_prof;
  const double* df_psi;
};

template <typename R> __device__ __forceinline__ const Nodes<R>& nodes(const Bufs& B);
template <> __device__ __forceinline__ const Nodes<double>& nodes<double>(const Bufs& B) { return B.n64; }
template <> __device__ __forceinline__ const Nodes<float>& nodes<float>(const Bufs& B) { return B.n32; }
template <typename R> __device__ __forceinline__ const Metric<R>& metric(const Bufs& B);
template <> __device__ __forceinline__ const Metric<double>& metric<double>(const Bufs& B) { return B.m64; }
template <> __device__ __forceinline__ const Metric<float>& metric<float>(const Bufs& B) { return B.m32; }
template <typename R> __device__ __forceinline__ R* face_flux(const Bufs& B, int dir);
template <> __device__ __forceinline__ double* face_flux<double>(const Bufs& B, int dir) { return B.fh64[dir]; }
template <> __device__ __forceinline__ float* face_flux<float>(const Bufs& B, int dir) { return B.fh32[dir]; }
template <typename R> __device__ __forceinline__ const Coefs<R>& coefs(const Consts& C);
template <> __device__ __forceinline__ const Coefs<double>& coefs<double>(const Consts& C) { return C.k64; }
template <> __device__ __forceinline__ const Coefs<float>& coefs<float>(const Consts& C) { return C.k32; }

// RK stage update fused into the assembly (flows without forcing): w <- w + dt (alpha R_old +
// beta R), R_old <- R, with dt from the device scalars; w == nullptr: no fusion.
struct RkFuse {
  double* w;
  double* r_old;
  int stage;  // RK stage 0..2
};

// Wray's low-storage RK3 (Eq. RK): w <- w + dt (alpha_s R_old + beta_s R). alpha_1 is printed
// +17/60 in the paper and read as -17/60 (first-order consistency: sum alpha + sum beta = 1).
__host__ __device__ constexpr double rk_alpha(int s) { return s == 0 ? 0.0 : (s == 1 ? -17.0 / 60.0 : -5.0 / 12.0); }
__host__ __device__ constexpr double rk_beta(int s) { return s == 0 ? 8.0 / 15.0 : (s == 1 ? 5.0 / 12.0 : 3.0 / 4.0); }

// device scalars: dt, time, forcing, CFL maximum, recycling scale, alpha_s dt (slots 5..7),
// the conserved totals (8..12), beta_s dt (13..15)
enum { kScalDt = 0, kScalTime = 1, kScalForce = 2, kScalCflMax = 3, kScalRecycle = 4, kScalAdt = 5,
       kScalBdt = 13, kScalCount = 16 };

__device__ __forceinline__ long long gidx(const Dims& d, int i, int j, int k) {
  return ((long long)(k + G) * d.py + (j + G)) * d.px + (i + GX);
}

// Debug builds (-DSTRM_DEBUG, the bounds-checking build): the kernels check the extreme nodes of
// every stencil, the ghost sources and the list entries they are about to use, OR a code into
// the context's error word when one lies outside its array, and skip that access instead of
// faulting (codes: kDbg*). Release builds compile the checks away.
#ifdef STRM_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif
enum : unsigned { kDbgGhost = 1u, kDbgNode = 2u, kDbgFace = 4u, kDbgList = 8u, kDbgInflow = 16u };

__device__ __forceinline__ bool node_in_box(const Dims& d, int i, int j, int k) {
  return i >= -G && i < d.nx + G && j >= -G && j < d.ny + G && k >= -G && k < d.nz + G;
}

// true when the nodes from -lo to +hi along dir around (i, j, k) are all in the ghosted box
// (always true in release builds); records `code` otherwise
__device__ __forceinline__ bool stencil_ok(const Dims& d, int i, int j, int k, int dir, int lo, int hi,
                                           unsigned code) {
  if constexpr (!kDebug) {
    return true;
  } else {
    int a0 = i - (dir == 0 ? lo : 0), a1 = j - (dir == 1 ? lo : 0), a2 = k - (dir == 2 ? lo : 0);
    int b0 = i + (dir == 0 ? hi : 0), b1 = j + (dir == 1 ? hi : 0), b2 = k + (dir == 2 ? hi : 0);
    bool ok = node_in_box(d, a0, a1, a2) && node_in_box(d, b0, b1, b2);
    if (!ok && d.dbg) atomicOr(d.dbg, code);
    return ok;
  }
}

// the same for a single index against an extent
__device__ __forceinline__ bool index_ok(const Dims& d, long long q, long long n, unsigned code) {
  if constexpr (!kDebug) {
    return true;
  } else {
    bool ok = q >= 0 && q < n;
    if (!ok && d.dbg) atomicOr(d.dbg, code);
    return ok;
  }
}

// Traversal order of the assembly and of the z-face kernels (classification and the sweeps over
// every z face). The t-th element is taken slab by slab: a slab is TY consecutive full rows
// (x fastest, so warps and DRAM see the same contiguous rows as in the natural order), the
// elements of one slab-plane come first, then the same slab one plane further in z, then the
// next slab. The z stencils (nodes k -+ 3, faces' nodes k-2 .. k+3) then re-read planes of the
// same slab that were read moments before, from L2, instead of planes millions of elements
// away in the natural order, which on the 2048 x 384 x 256 workload no longer fit in L2. The y
// stencil of the assembly reads 3 rows outside each slab (6/TY more rows). TY (Dims::slab_ty)
// is one of 32, 16, 8 admitted by slab_rows_allowed, by default the largest (slab_rows_for with
// cap 32); 0 keeps the natural order. An ensemble's autotuner may choose a smaller one.
__device__ __forceinline__ int slab_rows(const Dims& d) { return d.slab_ty; }

// Natural index (p ny + j) nx + i of the t-th element of nplanes planes in slab order
// (0 <= t < nx ny nplanes < 2^32, TY = slab_rows(d) > 0); 32-bit divisions.
__device__ __forceinline__ long long slab_order(const Dims& d, long long t, int nplanes, int TY) {
  const unsigned S = (unsigned)d.nx * (unsigned)TY;  // elements of one slab-plane
  const unsigned SP = S * (unsigned)nplanes;          // elements of one slab over all planes
  const unsigned u = (unsigned)t;
  const unsigned s = u / SP;
  const unsigned rem = u - s * SP;
  const unsigned p = rem / S;
  const unsigned r = rem - p * S;  // (j - s TY) nx + i
  return ((long long)p * d.ny + (long long)s * TY) * d.nx + r;
}

// The t-th interior node of the assembly (0 <= t < N) and the t-th z face of the z-face kernels
// (0 <= t < nf[2]).
__device__ __forceinline__ long long node_order(const Dims& d, long long t) {
  const int TY = slab_rows(d);
  return TY ? slab_order(d, t, d.nz, TY) : t;
}
__device__ __forceinline__ long long zface_order(const Dims& d, long long t) {
  const int TY = d.zslab_ty;
  return TY ? slab_order(d, t, d.nz + 1, TY) : t;
}

__device__ __forceinline__ long long dir_stride(const Dims& d, int dir) {
  return dir == 0 ? 1LL : (dir == 1 ? (long long)d.px : d.plane);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// x^e for x > 0 as exp(e log x): about half the FP64 operations of pow, within a few ulp of
// it for the temperatures of the flow (the error of the exponent argument is |e log x| ulp).
// x = 0 gives 0 and x < 0 gives NaN, as pow does.
__device__ __forceinline__ double rpow(double x, double e) { return exp(e * log(x)); }
__device__ __forceinline__ float rpow(float x, float e) { return powf(x, e); }

// defined below
__device__ __forceinline__ double rcp_nr(double x);
__device__ __forceinline__ float d2f(double x);
__device__ __forceinline__ double f2d(float x);

// t^(19/25) = t^0.76 (the power-law viscosity of the workloads) for t in [2^-6, 2^6], within
// about one ulp: an FP32 seed y0 = 2^(0.76 log2 t) (relative error a few 1e-7), then the exact
// relation y^25 = t^19 corrects it in one FP64 step, y = y0 (1 + delta)^(1/25) with
// delta = t^19 / y0^25 - 1, expanded to third order (|delta| < 3e-5, so the fourth-order term
// is below 1e-19). The powers take 12 multiplications by repeated squaring and 1/y0^25 an FP32
// estimate with one Newton step (relative error 2^-43, times |delta|): about 19 FP64 operations
// against about 45 for exp(e log t). Outside the range (or for NaN) it returns exp(e log t).
__device__ __forceinline__ double pow_19_25(double t) {
  const float tf = d2f(t);
  if (!(tf >= 0.015625f && tf <= 64.f)) return exp(0.76 * log(t));
  const double y0 = f2d(exp2f(0.76f * __log2f(tf)));
  const double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4, t16 = t8 * t8, t19 = (t16 * t2) * t;
  const double y2 = y0 * y0, y4 = y2 * y2, y8 = y4 * y4, y16 = y8 * y8, y25 = (y16 * y8) * y0;
  const double delta = (t19 - y25) * rcp_nr(y25);
  // (1 + d)^(1/25) = 1 + d/25 - (12/625) d^2 + (196/15625) d^3 + ...
  constexpr double c1 = 1.0 / 25.0, c2 = -12.0 / 625.0, c3 = 196.0 / 15625.0;
  return fma(y0 * delta, fma(fma(c3, delta, c2), delta, c1), y0);
}

// ---------------------------------------------------------------- FP64 bit patterns
// The two 32-bit halves of an FP64 value and back, as opaque register moves. Integer work on
// FP64 bit patterns goes through these: written as 64-bit integer operations on the bit
// pattern, a sign-bit mask is recognised by the compiler as |x| and issued on the FP64 pipe.
__device__ __forceinline__ void split64(double x, unsigned& lo, unsigned& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}
__device__ __forceinline__ double join64(unsigned lo, unsigned hi) {
  double x;
  asm("mov.b64 %0, {%1, %2};" : "=d"(x) : "r"(lo), "r"(hi));
  return x;
}

// ---------------------------------------------------------------- FP64 <-> FP32 conversions
// On GB300 (sm_103) the conversions between FP64 and FP32 issue on the FP64 pipe, which runs at 1/64
// of the FP32 rate. The mixed-precision kernels convert several values per stencil node, so
// they convert with 32-bit integer operations on the IEEE-754 bit patterns instead.
//
// binary64 -> binary32: round to nearest, ties away from zero (IEEE's ties-to-even differs only
// for values exactly halfway between two floats); magnitudes that round below the smallest
// normal float (2^-126) give a signed zero, those that round to 2^128 or above, infinities and
// NaNs give a signed infinity.
__device__ __forceinline__ float d2f(double x) {
  unsigned lo, hi;
  split64(x, lo, hi);
  const unsigned sign = hi & 0x80000000u;
  // magnitude plus half of the 29 dropped mantissa bits (the carry moves into the high word and,
  // past the mantissa, into the exponent as it should), rebiased from 1023 to 127 (896 << 20)
  const unsigned lo2 = lo + 0x10000000u;
  const int h = (int)((hi & 0x7fffffffu) + (lo2 < lo ? 1u : 0u) - (896u << 20));  // < 0 below 2^-127
  unsigned m = __funnelshift_r(lo2, (unsigned)h, 29);  // low 32 bits of (h:lo2) >> 29
  m = h >= (255 << 20) ? 0x7f800000u : m;
  m = h < (1 << 20) ? 0u : m;
  return __uint_as_float(m | sign);
}

// binary32 -> binary64, exact for normal floats; subnormals give a signed zero, infinities and
// NaNs stay infinities and NaNs.
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u, m = b & 0x7fffffffu;
  unsigned hi = (m >> 3) + (m >= 0x7f800000u ? (1792u << 20) : (896u << 20));
  unsigned lo = m << 29;
  if (m < 0x00800000u) hi = lo = 0u;
  return join64(lo, hi | sign);
}

__device__ __forceinline__ double to_f64(float x) { return f2d(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// 1/x and 1/sqrt(x) for positive normal x in the FP32 range, for the mixed-precision path: an
// FP32 estimate refined by one Newton-Raphson step in FP64. With an estimate of relative error
// d the step leaves d^2 (1/x) and about 1.5 d^2 (1/sqrt x): below 2^-43, far below the FP32
// rounding that every mixed-precision result gets.
__device__ __forceinline__ double rcp_nr(double x) {
  const double y = f2d(__frcp_rn(d2f(x)));
  return fma(y, fma(-x, y, 1.0), y);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = f2d(rsqrtf(d2f(x)));
  const double r = fma(-x * y, y, 1.0);  // 1 - x y^2
  return fma(0.5 * y, r, y);
}

// Viscosity law (Section 2): power law mu_ref (T/t_ref)^exp, or Sutherland.
template <typename R>
__device__ __forceinline__ R viscosity(const Coefs<R>& K, int law, R T) {
  R tr = T * K.inv_tref;
  if (law == 1) return K.mu_ref * (tr * sqrt(tr)) * (R(1) + K.suth_s) / (tr + K.suth_s);
  if constexpr (sizeof(R) == sizeof(double)) {
    if (K.exp_19_25) return K.mu_ref * pow_19_25(tr);
  }
  return K.mu_ref * rpow(tr, K.visc_exp);
}

// FP64 Laplacian numerator at node n on the stretched grid, without the y first-derivative term:
//   cc f_0 + sum_l [bx_l (f_{+l x} + f_{-l x}) + bz_l (f_{+l z} + f_{-l z})]
//          + c2 sum_l b_l (f_{+l y} + f_{-l y}),
// cc = bx_0 + bz_0 + c2 b_0 (b_0 = -2 sum_l b_l, the centre weight of the stencil written as
// sum_l b_l f_l): the three second differences share one centre term, applied once, and 1/dx^2,
// 1/dz^2 ride on the x and z weights; two operations per l and direction instead of three. In
// FP64 the cancellation of the large centre term costs ~1e-16 |f_0| / h^2, far below the
// truncation error; FP32 keeps the difference form. With grad, also the first-derivative sums
// along x, y, z (x and z already divided by dx and dz, y not yet by y_eta deta).
template <int L>
__device__ __forceinline__ double lap_c(const double* STRM_RO f, long long n, long long sy, long long sz,
                                        const Coefs<double>& K, double cc, double c2, double* grad = nullptr) {
  double s = cc * STRM_LDG(f + n), t = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const double xp = STRM_LDG(f + n + l), xm = STRM_LDG(f + n - l);
    const double yp = STRM_LDG(f + n + l * sy), ym = STRM_LDG(f + n - l * sy);
    const double zp = STRM_LDG(f + n + l * sz), zm = STRM_LDG(f + n - l * sz);
    s = fma(K.bx[l], xp + xm, s);
    s = fma(K.bz[l], zp + zm, s);
    t = fma(K.b[l], yp + ym, t);
    if (grad) {
      gx = fma(K.ax[l], xp - xm, gx);
      gy = fma(K.a[l], yp - ym, gy);
      gz = fma(K.az[l], zp - zm, gz);
    }
  }
  if (grad) {
    grad[0] = gx;
    grad[1] = gy;
    grad[2] = gz;
  }
  return fma(c2, t, s);
}

// sum_l a_l (f_{+l} - f_{-l}) along a line (first-derivative numerator of order 2L)
template <int L, typename R>
__device__ __forceinline__ R dsum(const R* STRM_RO f, long long n, long long st, const R* a) {
  R s = R(0);
#pragma unroll
  for (int l = 1; l <= L; ++l) s += a[l] * (STRM_LDG(f + n + l * st) - STRM_LDG(f + n - l * st));
  return s;
}

// First- and second-derivative numerators along one line, sharing the loads:
// s1 = sum_l a_l (f_{+l} - f_{-l}), s2 = sum_l b_l (f_{+l} + f_{-l} - 2 f_0).
template <int L, typename R>
__device__ __forceinline__ void dsum12(const R* STRM_RO f, long long n, long long st, const R* a,
                                       const R* b, R& s1, R& s2) {
  R f0 = STRM_LDG(f + n);
  s1 = R(0);
  s2 = R(0);
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    R fp = STRM_LDG(f + n + l * st), fm = STRM_LDG(f + n - l * st);
    s1 += a[l] * (fp - fm);
    s2 += b[l] * ((fp + fm) - R(2) * f0);
  }
}

// Ducros sensor at interior node (i,j,k) (Eq. sensor): theta = max(-div / sqrt(div^2 +
// |curl u|^2 + (u0/L0)^2), 0), first derivatives of order 2L in precision R; div is returned too.
template <int L, typename R>
__device__ __forceinline__ R theta_node(const Dims& d, const Consts& C, const Bufs& B, int i, int j,
                                        int k, R& div, R* g9 = nullptr) {
  const Nodes<R>& P = nodes<R>(B);
  const Coefs<R>& K = coefs<R>(C);
  long long n = gidx(d, i, j, k);
  long long sy = d.px, sz = d.plane;
  R hy = metric<R>(B).inv_hy[j];
  R ux = dsum<L>(P.u, n, 1, K.ax);
  R uy = dsum<L>(P.u, n, sy, K.a) * hy;
  R uz = dsum<L>(P.u, n, sz, K.az);
  R vx = dsum<L>(P.v, n, 1, K.ax);
  R vy = dsum<L>(P.v, n, sy, K.a) * hy;
  R vz = dsum<L>(P.v, n, sz, K.az);
  R wx = dsum<L>(P.w, n, 1, K.ax);
  R wy = dsum<L>(P.w, n, sy, K.a) * hy;
  R wz = dsum<L>(P.w, n, sz, K.az);
  div = ux + vy + wz;
  if (g9) {  // d_b u_a, a = u, v, w
    g9[0] = ux; g9[1] = uy; g9[2] = uz;
    g9[3] = vx; g9[4] = vy; g9[5] = vz;
    g9[6] = wx; g9[7] = wy; g9[8] = wz;
  }
  R o1 = wy - vz, o2 = uz - wx, o3 = vx - uy;
  R den = sqrt(div * div + (o1 * o1 + o2 * o2 + o3 * o3) + K.sens_eps);
  R th = -div / den;
  return th > R(0) ? th : R(0);
}

// Interior node whose theta a ghost node carries along a direction with face kinds lo/hi:
// periodic copy, even mirror across a wall, copy of the boundary node at other faces.
__device__ __forceinline__ int theta_source(int idx, int n, int lo, int hi) {
  if (idx >= 0 && idx < n) return idx;
  if (idx < 0) {
    if (lo == kBcPeriodic) return wrapi(idx, n);
    return lo == kBcWall ? -1 - idx : 0;
  }
  if (hi == kBcPeriodic) return wrapi(idx, n);
  return hi == kBcWall ? 2 * n - 1 - idx : n - 1;
}

// Hybrid switch decision for the face whose left node is (i,j,k) along dir: the largest theta
// over the window exceeds the threshold. The decision reads the FP64 theta field in both
// precisions (in mixed precision it holds FP64 theta at every node whose FP32 value is near
// the threshold). theta >= 0, so the maximum and the comparison are taken on the IEEE bit
// patterns on the integer pipe.
template <int L, typename R>
__device__ __forceinline__ bool face_decision(const Dims& d, const Consts& C, const Bufs& B, int i, int j,
                                              int k, int dir) {
  if (C.weno_mode == 2) return true;
  if (C.weno_mode == 0) return false;
  const double* th = B.n64.theta;
  long long n = gidx(d, i, j, k), st = dir_stride(d, dir), m = 0;
#pragma unroll
  for (int q = -L + 1; q <= L; ++q) {
    long long b = __double_as_longlong(STRM_LDG(th + n + q * st));
    m = b > m ? b : m;
  }
  return m > __double_as_longlong(C.k64.theta_thr);
}

// Block-wide sum (deterministic order) of a per-thread value; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// max that propagates NaN (a NaN anywhere must reach the CFL step and the totals)
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ float nanmaxf(float a, float b) { return (a > b || a != a) ? a : b; }

// FP32 block maximum (NaN-propagating) through a shared array of at least 32 floats.
__device__ __forceinline__ float block_max_f(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v = nanmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.f;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v = nanmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace strm
