// Device-side layout, constants and shared device functions of the sm_103a library.
//
// Layout in HBM
//   state w, residual R, RK register: SoA [5][nz][ny][nx] FP64 (interior only, caller-owned)
//   primitives and sensor fields: ghosted [nz+2G][ny+2G][px] FP64 (workspace); the interior
//     node (i,j,k) sits at ((k+G)*py + j+G)*px + i+GX; GX = 4 keeps interior rows 32-byte
//     aligned, px is a multiple of 4.
//   interface fluxes (workspace): x faces [5][nz][ny][nx+1], y faces [5][nz][ny+1][nx],
//     z faces [5][nz+1][ny][nx]; face s along a direction lies between nodes s-1 and s.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace strm {

constexpr int G = 3;   // ghost layers (central L <= 3, six-node WENO5 stencil)
constexpr int GX = 4;  // x offset of the interior in a ghosted row
constexpr int kRedBlock = 256;

struct Dims {
  int nx, ny, nz;
  int px, py, pz;     // ghosted extents (px padded)
  long long plane;    // px * py
  long long ng;       // px * py * pz
  long long N;        // nx * ny * nz
  long long nf[3];    // faces per direction
};

struct Consts {
  // gas
  double gamma, gm1, r_gas, inv_r, cv, inv_cv, cp, cp_pr;
  double mu_ref, inv_tref, visc_exp, suth_s, t_wall;
  int visc_law, wall_y, forcing;
  // scheme
  int L, weno_mode, convective, viscous;
  double a[4], b[4];
  double theta_thr, weno_eps, sens_eps;
  // uniform directions
  double inv_dx, inv_dz, inv_dx2, inv_dz2;
  double vtot;  // total metric volume
};

struct Bufs {
  double *rho, *u, *v, *w, *p, *T, *H, *c, *mu;  // ghosted primitives
  double *srho;                                 // ghosted sqrt(rho) (Roe weights)
  double *theta, *div;                          // ghosted sensor and node divergence
  double *fh[3];                                // interface fluxes
  double *R;                                    // residual, 5*N
  int *wl[3];                                   // compacted WENO face lists
  int *cl[3];                                   // compacted central face lists
  unsigned int *wcount;                         // [0..2] WENO list lengths, [4..6] central
  double *red;                                  // reduction partials
  double *scal;                                 // device scalars, see kScal*
  const double *inv_hy, *c2y, *c1y, *vol;       // per-j metrics: 1/(y_eta deta),
                                                // 1/(y_eta deta)^2, y_etaeta/(y_eta^3 deta), volume
};

// device scalars
enum { kScalDt = 0, kScalTime = 1, kScalForce = 2, kScalCflMax = 3, kScalCount = 16 };

__device__ __forceinline__ long long gidx(const Dims& d, int i, int j, int k) {
  return ((long long)(k + G) * d.py + (j + G)) * d.px + (i + GX);
}

__device__ __forceinline__ long long dir_stride(const Dims& d, int dir) {
  return dir == 0 ? 1LL : (dir == 1 ? (long long)d.px : d.plane);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Viscosity law (Section 2): power law mu_ref (T/t_ref)^exp, or Sutherland.
__device__ __forceinline__ double viscosity(const Consts& C, double T) {
  double tr = T * C.inv_tref;
  if (C.visc_law == 1) return C.mu_ref * pow(tr, 1.5) * (1.0 + C.suth_s) / (tr + C.suth_s);
  return C.mu_ref * pow(tr, C.visc_exp);
}

// sum_l a_l (f_{+l} - f_{-l}) along a line (first-derivative numerator of order 2L)
template <int L>
__device__ __forceinline__ double dsum(const double* __restrict__ f, long long n, long long st,
                                       const double* a) {
  double s = 0.0;
#pragma unroll
  for (int l = 1; l <= L; ++l) s += a[l] * (__ldg(f + n + l * st) - __ldg(f + n - l * st));
  return s;
}

// First- and second-derivative numerators along one line, sharing the loads:
// s1 = sum_l a_l (f_{+l} - f_{-l}), s2 = sum_l b_l (f_{+l} + f_{-l} - 2 f_0).
template <int L>
__device__ __forceinline__ void dsum12(const double* __restrict__ f, long long n, long long st,
                                       const double* a, const double* b, double& s1, double& s2) {
  double f0 = __ldg(f + n);
  s1 = 0.0;
  s2 = 0.0;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    double fp = __ldg(f + n + l * st), fm = __ldg(f + n - l * st);
    s1 += a[l] * (fp - fm);
    s2 += b[l] * ((fp + fm) - 2.0 * f0);
  }
}

// WENO switch at the face between nodes n and n+st: max theta over nodes n-L+1 .. n+L.
template <int L>
__device__ __forceinline__ bool face_flag(const Consts& C, const double* __restrict__ theta,
                                          long long n, long long st) {
  if (C.weno_mode == 2) return true;
  if (C.weno_mode == 0) return false;
  double tmax = 0.0;
#pragma unroll
  for (int q = -L + 1; q <= L; ++q) tmax = fmax(tmax, __ldg(theta + n + q * st));
  return tmax > C.theta_thr;
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
