// Node-wise kernels: primitives (+ CFL partial maxima), ghost fills of the primitives and of
// the sensor fields, the Ducros sensor, RK stage update, forcing, totals and flag export.
#include "strm_dev.cuh"
#include "strm_launch.h"

namespace strm {

// ---------------------------------------------------------------------------------- primitives

__device__ __forceinline__ void node_ijk(const Dims& d, long long q, int& i, int& j, int& k) {
  i = (int)(q % d.nx);
  long long r = q / d.nx;
  j = (int)(r % d.ny);
  k = (int)(r / d.ny);
}

// Primitive variables at the interior nodes from w = [rho, rho u, rho v, rho w, rho E]
// (Section 2: E = cv T + |u|^2/2, p = rho R T, H = E + p/rho), plus c, mu(T) and sqrt(rho).
// With want_cfl, each block also writes the largest sum_d (|u_d| + c)/h_d of its nodes.
__global__ void __launch_bounds__(256) k_prims(Dims d, Consts C, Bufs B, const double* __restrict__ w,
                                               int want_cfl) {
  __shared__ double sh[32];
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double spec = 0.0;
  if (q < d.N) {
    int i, j, k;
    node_ijk(d, q, i, j, k);
    const Nodes<double>& P = B.n64;
    double rho = w[q];
    double ir = 1.0 / rho;
    double u = w[d.N + q] * ir, v = w[2 * d.N + q] * ir, ww = w[3 * d.N + q] * ir;
    double E = w[4 * d.N + q] * ir;
    double T = (E - 0.5 * (u * u + v * v + ww * ww)) * C.inv_cv;
    double p = rho * C.r_gas * T;
    double c = sqrt(C.gamma * p * ir);
    long long n = gidx(d, i, j, k);
    P.rho[n] = rho;
    P.u[n] = u;
    P.v[n] = v;
    P.w[n] = ww;
    P.T[n] = T;
    P.p[n] = p;
    P.H[n] = E + p * ir;
    P.c[n] = c;
    P.mu[n] = viscosity(C.k64, C.visc_law, T);
    P.srho[n] = sqrt(rho);
    if (want_cfl)
      spec = (fabs(u) + c) * C.k64.inv_dx + (fabs(v) + c) * B.m64.inv_hy[j] + (fabs(ww) + c) * C.k64.inv_dz;
  }
  if (want_cfl) {
    double m = block_max(spec, sh);
    if (threadIdx.x == 0) B.red[blockIdx.x] = m;
  }
}

// Mixed precision: the fields the characteristic projection reads are formed in FP64 (rho, u,
// v, w, p, T, H, sqrt rho); FP32 copies of all fields feed the FP32 kernels, with c and mu(T)
// evaluated in FP32. The CFL partial is formed in FP64 from the FP64 velocities.
__global__ void __launch_bounds__(256) k_prims_mixed(Dims d, Consts C, Bufs B, const double* __restrict__ w,
                                                     int want_cfl) {
  __shared__ double sh[32];
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double spec = 0.0;
  if (q < d.N) {
    int i, j, k;
    node_ijk(d, q, i, j, k);
    const Nodes<double>& P = B.n64;
    const Nodes<float>& F = B.n32;
    double rho = w[q];
    double ir = 1.0 / rho;
    double u = w[d.N + q] * ir, v = w[2 * d.N + q] * ir, ww = w[3 * d.N + q] * ir;
    double E = w[4 * d.N + q] * ir;
    double T = (E - 0.5 * (u * u + v * v + ww * ww)) * C.inv_cv;
    double p = rho * C.r_gas * T;
    double H = E + p * ir;
    long long n = gidx(d, i, j, k);
    P.rho[n] = rho;
    P.u[n] = u;
    P.v[n] = v;
    P.w[n] = ww;
    P.T[n] = T;
    P.p[n] = p;
    P.H[n] = H;
    P.srho[n] = sqrt(rho);
    float rf = (float)rho, pf = (float)p, Tf = (float)T;
    float cf = sqrtf(C.k32.gamma * pf / rf);
    F.rho[n] = rf;
    F.u[n] = (float)u;
    F.v[n] = (float)v;
    F.w[n] = (float)ww;
    F.p[n] = pf;
    F.T[n] = Tf;
    F.H[n] = (float)H;
    F.c[n] = cf;
    F.mu[n] = viscosity(C.k32, C.visc_law, Tf);
    if (want_cfl) {
      double c = (double)cf;
      spec = (fabs(u) + c) * C.k64.inv_dx + (fabs(v) + c) * B.m64.inv_hy[j] + (fabs(ww) + c) * C.k64.inv_dz;
    }
  }
  if (want_cfl) {
    double m = block_max(spec, sh);
    if (threadIdx.x == 0) B.red[blockIdx.x] = m;
  }
}

// dt from the CFL partials (or the fixed step), and the simulated time.
__global__ void k_dt_finalize(Bufs B, int nparts, double cfl, double dt_fixed) {
  __shared__ double sh[32];
  double m = 0.0;
  if (dt_fixed <= 0.0)
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) m = nanmax(m, B.red[t]);
  m = block_max(m, sh);
  if (threadIdx.x == 0) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl / m;
    B.scal[kScalDt] = dt;
    B.scal[kScalCflMax] = m;
    B.scal[kScalTime] += dt;
  }
}

// ---------------------------------------------------------------------------------- ghost fills

// Thread layout of a face ghost fill: x faces (2G * ny * nz), then y faces (nx * 2G * nz), then
// z faces (nx * ny * 2G). Edges and corners are never read and stay untouched.
__device__ __forceinline__ bool ghost_target(const Dims& d, long long q, int& face, int& i, int& j,
                                             int& k, int& si, int& sj, int& sk, int& mirror) {
  long long nxf = 2LL * G * d.ny * d.nz, nyf = 2LL * G * d.nx * d.nz, nzf = 2LL * G * d.nx * d.ny;
  mirror = 0;
  if (q < nxf) {
    int g = (int)(q % (2 * G));
    long long r = q / (2 * G);
    j = (int)(r % d.ny);
    k = (int)(r / d.ny);
    i = g < G ? -1 - g : d.nx + (g - G);
    si = wrapi(i, d.nx);
    sj = j;
    sk = k;
    face = 0;
    return true;
  }
  q -= nxf;
  if (q < nyf) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    int g = (int)(r % (2 * G));
    k = (int)(r / (2 * G));
    j = g < G ? -1 - g : d.ny + (g - G);
    si = i;
    sk = k;
    face = 1;
    sj = wrapi(j, d.ny);
    mirror = g < G ? g : d.ny - 1 - (g - G);  // wall mirror: j=-1-q <-> q, j=ny+q <-> ny-1-q
    return true;
  }
  q -= nyf;
  if (q < nzf) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % d.ny);
    int g = (int)(r / d.ny);
    k = g < G ? -1 - g : d.nz + (g - G);
    si = i;
    sj = j;
    sk = wrapi(k, d.nz);
    face = 2;
    return true;
  }
  return false;
}

template <typename R>
__device__ __forceinline__ void copy_node(const Nodes<R>& P, long long dst, long long src, bool cmu) {
  P.rho[dst] = P.rho[src];
  P.u[dst] = P.u[src];
  P.v[dst] = P.v[src];
  P.w[dst] = P.w[src];
  P.p[dst] = P.p[src];
  P.T[dst] = P.T[src];
  P.H[dst] = P.H[src];
  if (cmu) {
    P.c[dst] = P.c[src];
    P.mu[dst] = P.mu[src];
  }
}

// Isothermal no-slip staggered wall: the ghost mirrors an interior node across the wall
// interface with reversed velocity, T_g = 2 T_w - T, p_g = p, rho_g = p_g/(R T_g).
struct WallGhost {
  double rho, u, v, w, p, T, H;
};

__device__ __forceinline__ WallGhost wall_state(const Consts& C, const Nodes<double>& P, long long src) {
  WallGhost g;
  g.u = -P.u[src];
  g.v = -P.v[src];
  g.w = -P.w[src];
  g.p = P.p[src];
  g.T = 2.0 * C.t_wall - P.T[src];
  g.rho = g.p / (C.r_gas * g.T);
  g.H = C.cp * g.T + 0.5 * (g.u * g.u + g.v * g.v + g.w * g.w);
  return g;
}

__device__ __forceinline__ void store_wall64(const Nodes<double>& P, long long dst, const WallGhost& g) {
  P.rho[dst] = g.rho;
  P.u[dst] = g.u;
  P.v[dst] = g.v;
  P.w[dst] = g.w;
  P.p[dst] = g.p;
  P.T[dst] = g.T;
  P.H[dst] = g.H;
  P.srho[dst] = sqrt(g.rho);
}

__global__ void __launch_bounds__(256) k_ghost_prims(Dims d, Consts C, Bufs B, long long nthreads) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, i, j, k, si, sj, sk, mirror;
  if (!ghost_target(d, q, face, i, j, k, si, sj, sk, mirror)) return;
  const Nodes<double>& P = B.n64;
  long long dst = gidx(d, i, j, k);
  if (face == 1 && C.wall_y) {
    WallGhost g = wall_state(C, P, gidx(d, i, mirror, k));
    store_wall64(P, dst, g);
    P.c[dst] = sqrt(C.gamma * g.p / g.rho);
    P.mu[dst] = viscosity(C.k64, C.visc_law, g.T);
  } else {
    long long src = gidx(d, si, sj, sk);
    copy_node(P, dst, src, true);
    P.srho[dst] = P.srho[src];
  }
}

// Mixed precision: FP64 fields by the same rules, FP32 copies from them (c, mu in FP32).
__global__ void __launch_bounds__(256) k_ghost_prims_mixed(Dims d, Consts C, Bufs B, long long nthreads) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, i, j, k, si, sj, sk, mirror;
  if (!ghost_target(d, q, face, i, j, k, si, sj, sk, mirror)) return;
  const Nodes<double>& P = B.n64;
  const Nodes<float>& F = B.n32;
  long long dst = gidx(d, i, j, k);
  if (face == 1 && C.wall_y) {
    WallGhost g = wall_state(C, P, gidx(d, i, mirror, k));
    store_wall64(P, dst, g);
    float rf = (float)g.rho, pf = (float)g.p, Tf = (float)g.T;
    F.rho[dst] = rf;
    F.u[dst] = (float)g.u;
    F.v[dst] = (float)g.v;
    F.w[dst] = (float)g.w;
    F.p[dst] = pf;
    F.T[dst] = Tf;
    F.H[dst] = (float)g.H;
    F.c[dst] = sqrtf(C.k32.gamma * pf / rf);
    F.mu[dst] = viscosity(C.k32, C.visc_law, Tf);
  } else {
    long long src = gidx(d, si, sj, sk);
    copy_node(P, dst, src, false);
    P.srho[dst] = P.srho[src];
    copy_node(F, dst, src, true);
  }
}

// theta and the node divergence: periodic copies, even mirror across a wall.
template <typename R>
__global__ void __launch_bounds__(256) k_ghost_scalars(Dims d, Consts C, Bufs B, long long nthreads) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, i, j, k, si, sj, sk, mirror;
  if (!ghost_target(d, q, face, i, j, k, si, sj, sk, mirror)) return;
  const Nodes<R>& P = nodes<R>(B);
  long long dst = gidx(d, i, j, k);
  long long src = (face == 1 && C.wall_y) ? gidx(d, i, mirror, k) : gidx(d, si, sj, sk);
  P.theta[dst] = P.theta[src];
  P.div[dst] = P.div[src];
}

// ---------------------------------------------------------------------------------- sensor

// Ducros sensor (Eq. sensor) at the interior nodes; the node divergence is kept for the
// viscous terms.
template <int L, typename R>
__global__ void __launch_bounds__(256) k_sensor(Dims d, Consts C, Bufs B) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  int i, j, k;
  node_ijk(d, q, i, j, k);
  const Nodes<R>& P = nodes<R>(B);
  R div;
  R th = theta_node<L, R>(d, C, B, i, j, k, div);
  long long n = gidx(d, i, j, k);
  P.theta[n] = th;
  P.div[n] = div;
}

// ---------------------------------------------------------------------------------- RK, forcing

// Forcing of the mass flow rate: f = -(sum_V vol R_rhou) / V_total from the assembly partials.
__global__ void k_force_finalize(Bufs B, int nparts, double inv_vtot) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += B.red[t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) B.scal[kScalForce] = -s * inv_vtot;
}

// Stage update of Eq. RK: w <- w + dt (alpha R_old + beta R), R includes the forcing terms
// R_rhou += f, R_rhoE += f u (Eqs. 1b, 1c); R_old <- R. One thread per node, five fields. FP64
// in both precisions.
__global__ void __launch_bounds__(256) k_rk_update(Dims d, Consts C, Bufs B, double* __restrict__ w,
                                                   double* __restrict__ r_old, double alpha,
                                                   double beta) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  double dt = B.scal[kScalDt];
  double f = C.forcing ? B.scal[kScalForce] : 0.0;
  double ad = alpha * dt, bd = beta * dt;
  double uq = 0.0;
  if (C.forcing) {
    int i, j, k;
    node_ijk(d, q, i, j, k);
    uq = B.n64.u[gidx(d, i, j, k)];
  }
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    long long e = m * d.N + q;
    double rr = B.R[e];
    if (m == 1) rr += f;
    if (m == 4) rr += f * uq;
    double wn = w[e] + bd * rr;
    if (alpha != 0.0) wn += ad * r_old[e];
    w[e] = wn;
    r_old[e] = rr;
  }
}

// Forcing terms added to an explicit residual (compute_rhs).
__global__ void __launch_bounds__(256) k_apply_forcing(Dims d, Bufs B, double* __restrict__ rhs) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  double f = B.scal[kScalForce];
  int i, j, k;
  node_ijk(d, q, i, j, k);
  double uq = B.n64.u[gidx(d, i, j, k)];
  rhs[d.N + q] += f;
  rhs[4 * d.N + q] += f * uq;
}

// ---------------------------------------------------------------------------------- totals

__global__ void __launch_bounds__(256) k_totals_partial(Dims d, Bufs B, const double* __restrict__ w) {
  __shared__ double sh[32];
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  double v = 0.0;
  if (q < d.N) {
    int j = (int)((q / d.nx) % d.ny);
    v = w[m * d.N + q] * B.vol[j];
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) B.red[(long long)m * gridDim.x + blockIdx.x] = v;
}

__global__ void k_totals_finalize(Bufs B, int nparts) {
  __shared__ double sh[32];
  int m = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += B.red[(long long)m * nparts + t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) B.scal[8 + m] = s;
}

// ---------------------------------------------------------------------------------- flags, copies

// WENO face flags in the export layout (x: [nz][ny][nx+1], y: [nz][ny+1][nx], z: [nz+1][ny][nx]).
template <int L, typename R>
__global__ void __launch_bounds__(256) k_flags(Dims d, Consts C, Bufs B, int dir, unsigned char* out) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.nf[dir]) return;
  int i, j, k;
  if (dir == 0) {
    int s = (int)(q % (d.nx + 1));
    long long r = q / (d.nx + 1);
    i = s - 1; j = (int)(r % d.ny); k = (int)(r / d.ny);
  } else if (dir == 1) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % (d.ny + 1)) - 1; k = (int)(r / (d.ny + 1));
  } else {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % d.ny); k = (int)(r / d.ny) - 1;
  }
  out[q] = face_decision<L, R>(d, C, B, i, j, k, dir) ? 1 : 0;
}

template <typename R>
__global__ void __launch_bounds__(256) k_export_interior(Dims d, const R* __restrict__ src,
                                                         double* __restrict__ dst) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  int i, j, k;
  node_ijk(d, q, i, j, k);
  dst[q] = (double)src[gidx(d, i, j, k)];
}

// ---------------------------------------------------------------------------------- launchers

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int reduce_blocks(const Dims& d) { return (int)blocks_for(d.N, kRedBlock); }

void launch_prims(const Dims& d, const Consts& C, const Bufs& B, const double* w, bool want_cfl,
                  cudaStream_t s) {
  if (C.mixed)
    k_prims_mixed<<<blocks_for(d.N, kRedBlock), kRedBlock, 0, s>>>(d, C, B, w, want_cfl ? 1 : 0);
  else
    k_prims<<<blocks_for(d.N, kRedBlock), kRedBlock, 0, s>>>(d, C, B, w, want_cfl ? 1 : 0);
}

void launch_dt_finalize(const Dims& d, const Bufs& B, double cfl, double dt_fixed, cudaStream_t s) {
  k_dt_finalize<<<1, 1024, 0, s>>>(B, reduce_blocks(d), cfl, dt_fixed);
}

static long long ghost_threads(const Dims& d) {
  return 2LL * G * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
}

void launch_ghost_prims(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  long long n = ghost_threads(d);
  if (C.mixed)
    k_ghost_prims_mixed<<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
  else
    k_ghost_prims<<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
}

void launch_sensor(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  unsigned nb = blocks_for(d.N, 256);
  if (C.mixed) {
    if (C.L == 3) k_sensor<3, float><<<nb, 256, 0, s>>>(d, C, B);
    else k_sensor<2, float><<<nb, 256, 0, s>>>(d, C, B);
  } else {
    if (C.L == 3) k_sensor<3, double><<<nb, 256, 0, s>>>(d, C, B);
    else k_sensor<2, double><<<nb, 256, 0, s>>>(d, C, B);
  }
}

void launch_ghost_scalars(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  long long n = ghost_threads(d);
  if (C.mixed)
    k_ghost_scalars<float><<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
  else
    k_ghost_scalars<double><<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
}

void launch_force_finalize(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  k_force_finalize<<<1, 1024, 0, s>>>(B, reduce_blocks(d), 1.0 / C.vtot);
}

void launch_rk_update(const Dims& d, const Consts& C, const Bufs& B, double* w, double* r_old,
                      double alpha, double beta, cudaStream_t s) {
  k_rk_update<<<blocks_for(d.N, 256), 256, 0, s>>>(d, C, B, w, r_old, alpha, beta);
}

void launch_apply_forcing(const Dims& d, const Bufs& B, double* rhs, cudaStream_t s) {
  k_apply_forcing<<<blocks_for(d.N, 256), 256, 0, s>>>(d, B, rhs);
}

void launch_totals(const Dims& d, const Bufs& B, const double* w, cudaStream_t s) {
  dim3 grid(blocks_for(d.N, kRedBlock), 5);
  k_totals_partial<<<grid, kRedBlock, 0, s>>>(d, B, w);
  k_totals_finalize<<<5, 1024, 0, s>>>(B, (int)grid.x);
}

void launch_flags(const Dims& d, const Consts& C, const Bufs& B, int dir, unsigned char* out,
                  cudaStream_t s) {
  unsigned nb = blocks_for(d.nf[dir], 256);
  if (C.mixed) {
    if (C.L == 3) k_flags<3, float><<<nb, 256, 0, s>>>(d, C, B, dir, out);
    else k_flags<2, float><<<nb, 256, 0, s>>>(d, C, B, dir, out);
  } else {
    if (C.L == 3) k_flags<3, double><<<nb, 256, 0, s>>>(d, C, B, dir, out);
    else k_flags<2, double><<<nb, 256, 0, s>>>(d, C, B, dir, out);
  }
}

void launch_export_sensor(const Dims& d, const Consts& C, const Bufs& B, double* theta, double* div,
                          cudaStream_t s) {
  unsigned nb = blocks_for(d.N, 256);
  if (C.mixed) {
    if (theta) k_export_interior<float><<<nb, 256, 0, s>>>(d, B.n32.theta, theta);
    if (div) k_export_interior<float><<<nb, 256, 0, s>>>(d, B.n32.div, div);
  } else {
    if (theta) k_export_interior<double><<<nb, 256, 0, s>>>(d, B.n64.theta, theta);
    if (div) k_export_interior<double><<<nb, 256, 0, s>>>(d, B.n64.div, div);
  }
}

}  // namespace strm
