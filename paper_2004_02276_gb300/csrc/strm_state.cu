// Node-wise kernels: primitives (+ CFL partial maxima), ghost fills of the primitives and of
// the sensor fields, the Ducros sensor, RK stage update, forcing, totals and flag export.
#include "strm_dev.cuh"
#include "strm_launch.h"

namespace strm {

// ---------------------------------------------------------------------------------- primitives

// Primitive variables at the interior nodes from w = [rho, rho u, rho v, rho w, rho E]
// (Section 2: E = cv T + |u|^2/2, p = rho R T, H = E + p/rho), plus c and mu(T). With
// want_cfl, each block also writes the largest sum_d (|u_d| + c)/h_d of its nodes.
__global__ void __launch_bounds__(256) k_prims(Dims d, Consts C, Bufs B, const double* __restrict__ w,
                                               int want_cfl) {
  __shared__ double sh[32];
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double spec = 0.0;
  if (q < d.N) {
    int i = (int)(q % d.nx);
    long long r = q / d.nx;
    int j = (int)(r % d.ny);
    int k = (int)(r / d.ny);
    double rho = w[q];
    double ir = 1.0 / rho;
    double u = w[d.N + q] * ir, v = w[2 * d.N + q] * ir, ww = w[3 * d.N + q] * ir;
    double E = w[4 * d.N + q] * ir;
    double T = (E - 0.5 * (u * u + v * v + ww * ww)) * C.inv_cv;
    double p = rho * C.r_gas * T;
    double c = sqrt(C.gamma * p * ir);
    long long n = gidx(d, i, j, k);
    B.rho[n] = rho;
    B.u[n] = u;
    B.v[n] = v;
    B.w[n] = ww;
    B.T[n] = T;
    B.p[n] = p;
    B.H[n] = E + p * ir;
    B.c[n] = c;
    B.mu[n] = viscosity(C, T);
    B.srho[n] = sqrt(rho);
    if (want_cfl)
      spec = (fabs(u) + c) * C.inv_dx + (fabs(v) + c) * B.inv_hy[j] + (fabs(ww) + c) * C.inv_dz;
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

__device__ __forceinline__ void copy_prims(const Bufs& B, long long dst, long long src) {
  B.rho[dst] = B.rho[src];
  B.u[dst] = B.u[src];
  B.v[dst] = B.v[src];
  B.w[dst] = B.w[src];
  B.p[dst] = B.p[src];
  B.T[dst] = B.T[src];
  B.H[dst] = B.H[src];
  B.c[dst] = B.c[src];
  B.mu[dst] = B.mu[src];
  B.srho[dst] = B.srho[src];
}

// Isothermal no-slip staggered wall: the ghost mirrors an interior node across the wall
// interface with reversed velocity, T_g = 2 T_w - T, p_g = p, rho_g = p_g/(R T_g).
__device__ __forceinline__ void wall_prims(const Consts& C, const Bufs& B, long long dst, long long src) {
  double u = -B.u[src], v = -B.v[src], w = -B.w[src];
  double p = B.p[src];
  double T = 2.0 * C.t_wall - B.T[src];
  double rho = p / (C.r_gas * T);
  B.rho[dst] = rho;
  B.u[dst] = u;
  B.v[dst] = v;
  B.w[dst] = w;
  B.p[dst] = p;
  B.T[dst] = T;
  B.H[dst] = C.cp * T + 0.5 * (u * u + v * v + w * w);
  B.c[dst] = sqrt(C.gamma * p / rho);
  B.mu[dst] = viscosity(C, T);
  B.srho[dst] = sqrt(rho);
}

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

__global__ void __launch_bounds__(256) k_ghost_prims(Dims d, Consts C, Bufs B, long long nthreads) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, i, j, k, si, sj, sk, mirror;
  if (!ghost_target(d, q, face, i, j, k, si, sj, sk, mirror)) return;
  long long dst = gidx(d, i, j, k);
  if (face == 1 && C.wall_y)
    wall_prims(C, B, dst, gidx(d, i, mirror, k));
  else
    copy_prims(B, dst, gidx(d, si, sj, sk));
}

// theta and the node divergence: periodic copies, even mirror across a wall.
__global__ void __launch_bounds__(256) k_ghost_scalars(Dims d, Consts C, Bufs B, long long nthreads) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, i, j, k, si, sj, sk, mirror;
  if (!ghost_target(d, q, face, i, j, k, si, sj, sk, mirror)) return;
  long long dst = gidx(d, i, j, k);
  long long src = (face == 1 && C.wall_y) ? gidx(d, i, mirror, k) : gidx(d, si, sj, sk);
  B.theta[dst] = B.theta[src];
  B.div[dst] = B.div[src];
}

// ---------------------------------------------------------------------------------- sensor

// Ducros sensor (Eq. sensor): theta = max(-div / sqrt(div^2 + |curl u|^2 + (u0/L0)^2), 0) with
// first derivatives of order 2L; the node divergence is kept for the viscous terms.
template <int L>
__global__ void __launch_bounds__(256) k_sensor(Dims d, Consts C, Bufs B) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  int i = (int)(q % d.nx);
  long long r = q / d.nx;
  int j = (int)(r % d.ny);
  int k = (int)(r / d.ny);
  long long n = gidx(d, i, j, k);
  long long sy = d.px, sz = d.plane;
  double hy = B.inv_hy[j];
  double ux = dsum<L>(B.u, n, 1, C.a) * C.inv_dx;
  double uy = dsum<L>(B.u, n, sy, C.a) * hy;
  double uz = dsum<L>(B.u, n, sz, C.a) * C.inv_dz;
  double vx = dsum<L>(B.v, n, 1, C.a) * C.inv_dx;
  double vy = dsum<L>(B.v, n, sy, C.a) * hy;
  double vz = dsum<L>(B.v, n, sz, C.a) * C.inv_dz;
  double wx = dsum<L>(B.w, n, 1, C.a) * C.inv_dx;
  double wy = dsum<L>(B.w, n, sy, C.a) * hy;
  double wz = dsum<L>(B.w, n, sz, C.a) * C.inv_dz;
  double div = ux + vy + wz;
  double o1 = wy - vz, o2 = uz - wx, o3 = vx - uy;
  double den = sqrt(div * div + (o1 * o1 + o2 * o2 + o3 * o3) + C.sens_eps);
  double th = -div / den;
  B.theta[n] = th > 0.0 ? th : 0.0;
  B.div[n] = div;
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
// R_rhou += f, R_rhoE += f u (Eqs. 1b, 1c); R_old <- R. One thread per node, five fields.
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
    int i = (int)(q % d.nx);
    long long r = q / d.nx;
    uq = B.u[gidx(d, i, (int)(r % d.ny), (int)(r / d.ny))];
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
  int i = (int)(q % d.nx);
  long long r = q / d.nx;
  double uq = B.u[gidx(d, i, (int)(r % d.ny), (int)(r / d.ny))];
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
template <int L>
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
  out[q] = face_flag<L>(C, B.theta, gidx(d, i, j, k), dir_stride(d, dir)) ? 1 : 0;
}

__global__ void __launch_bounds__(256) k_export_interior(Dims d, const double* __restrict__ src,
                                                         double* __restrict__ dst) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  int i = (int)(q % d.nx);
  long long r = q / d.nx;
  dst[q] = src[gidx(d, i, (int)(r % d.ny), (int)(r / d.ny))];
}

// ---------------------------------------------------------------------------------- launchers

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int reduce_blocks(const Dims& d) { return (int)blocks_for(d.N, kRedBlock); }

void launch_prims(const Dims& d, const Consts& C, const Bufs& B, const double* w, bool want_cfl,
                  cudaStream_t s) {
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
  k_ghost_prims<<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
}

void launch_sensor(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  if (C.L == 3)
    k_sensor<3><<<blocks_for(d.N, 256), 256, 0, s>>>(d, C, B);
  else
    k_sensor<2><<<blocks_for(d.N, 256), 256, 0, s>>>(d, C, B);
}

void launch_ghost_scalars(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  long long n = ghost_threads(d);
  k_ghost_scalars<<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
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
  if (C.L == 3)
    k_flags<3><<<blocks_for(d.nf[dir], 256), 256, 0, s>>>(d, C, B, dir, out);
  else
    k_flags<2><<<blocks_for(d.nf[dir], 256), 256, 0, s>>>(d, C, B, dir, out);
}

void launch_export_interior(const Dims& d, const double* src, double* dst, cudaStream_t s) {
  k_export_interior<<<blocks_for(d.N, 256), 256, 0, s>>>(d, src, dst);
}

}  // namespace strm
