// Convective interface fluxes (central energy-consistent, or characteristic LF-WENO5 at the
// faces the Ducros sensor flags) and the assembly of the residual with the viscous terms.
//
// Per direction: k_faces computes the central flux at every unflagged face and appends each
// flagged face to a compacted list (warp-aggregated atomics), so that k_weno runs the
// expensive characteristic reconstruction without warp divergence. k_assemble then forms
// R = -sum_d (f_{s+1} - f_s)/h_d + viscous terms per node and the forcing partial sums.
#include "strm_dev.cuh"
#include "strm_launch.h"

namespace strm {

// ------------------------------------------------------------------------------ face decoding

// Face q of direction DIR -> left node (i, j, k) (= node s-1 along DIR).
template <int DIR>
__device__ __forceinline__ void face_node(const Dims& d, long long q, int& i, int& j, int& k) {
  if (DIR == 0) {
    int s = (int)(q % (d.nx + 1));
    long long r = q / (d.nx + 1);
    i = s - 1;
    j = (int)(r % d.ny);
    k = (int)(r / d.ny);
  } else if (DIR == 1) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % (d.ny + 1)) - 1;
    k = (int)(r / (d.ny + 1));
  } else {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % d.ny);
    k = (int)(r / d.ny) - 1;
  }
}

// ------------------------------------------------------------------------------ central flux

// Energy-consistent split flux at the face between nodes n and n+st (Eqs. avg_operator,
// encflux): f_phi = 2 sum_l a_l sum_{m<l} (rho, u_n, phi)~_{n-m,l}. With
// qq = (rho_a + rho_b)(u_a + u_b)/4 this is sum_l a_l sum_m qq (phi_a + phi_b); the pressure
// enters the normal momentum as sum_l a_l sum_m (p_a + p_b).
template <int L, int DIR>
__device__ __forceinline__ void central_flux(const Consts& C, const Bufs& B, long long n, long long st,
                                             double* f) {
  const double* __restrict__ ud = DIR == 0 ? B.u : (DIR == 1 ? B.v : B.w);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0, ap = 0.0;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, sp = 0.0;
#pragma unroll
    for (int m = 0; m < l; ++m) {
      long long ia = n - m * st, ib = n + (l - m) * st;
      double qq = 0.25 * (__ldg(B.rho + ia) + __ldg(B.rho + ib)) * (__ldg(ud + ia) + __ldg(ud + ib));
      s0 += qq;
      s1 += qq * (__ldg(B.u + ia) + __ldg(B.u + ib));
      s2 += qq * (__ldg(B.v + ia) + __ldg(B.v + ib));
      s3 += qq * (__ldg(B.w + ia) + __ldg(B.w + ib));
      s4 += qq * (__ldg(B.H + ia) + __ldg(B.H + ib));
      sp += __ldg(B.p + ia) + __ldg(B.p + ib);
    }
    double al = C.a[l];
    a0 += al * s0;
    a1 += al * s1;
    a2 += al * s2;
    a3 += al * s3;
    a4 += al * s4;
    ap += al * sp;
  }
  f[0] = 2.0 * a0;
  f[1] = a1;
  f[2] = a2;
  f[3] = a3;
  f[4] = a4;
  f[1 + DIR] += ap;
}

// ------------------------------------------------------------------------------ WENO5

// Jiang-Shu WENO5 at i+1/2 from f_{i-2..i+2}, returned as numerator/denominator so that the
// caller divides once: value = num / den.
__device__ __forceinline__ void weno5_nd(double fm2, double fm1, double f0, double fp1, double fp2,
                                         double eps, double& num, double& den) {
  double t0 = fm2 - 2.0 * fm1 + f0, t1 = fm2 - 4.0 * fm1 + 3.0 * f0;
  double t2 = fm1 - 2.0 * f0 + fp1, t3 = fm1 - fp1;
  double t4 = f0 - 2.0 * fp1 + fp2, t5 = 3.0 * f0 - 4.0 * fp1 + fp2;
  double b0 = (13.0 / 12.0) * t0 * t0 + 0.25 * t1 * t1;
  double b1 = (13.0 / 12.0) * t2 * t2 + 0.25 * t3 * t3;
  double b2 = (13.0 / 12.0) * t4 * t4 + 0.25 * t5 * t5;
  double q0 = eps + b0, q1 = eps + b1, q2 = eps + b2;
  q0 *= q0;
  q1 *= q1;
  q2 *= q2;
  // alpha_k = d_k / q_k, scaled by q0 q1 q2 (the normalised weights are unchanged)
  double w0 = 0.1 * (q1 * q2), w1 = 0.6 * (q0 * q2), w2 = 0.3 * (q0 * q1);
  double c0 = 2.0 * fm2 - 7.0 * fm1 + 11.0 * f0;
  double c1 = -fm1 + 5.0 * f0 + 2.0 * fp1;
  double c2 = 2.0 * f0 + 5.0 * fp1 - fp2;
  num = w0 * c0 + w1 * c1 + w2 * c2;
  den = 6.0 * (w0 + w1 + w2);
}

// Characteristic Lax-Friedrichs flux-vector splitting with WENO5 (Section 2.1) at the face
// between nodes n and n+st: Roe average, projection of w and of the Euler flux at the six
// stencil nodes onto the left eigenvectors (written out through the two scalars A and B of
// the acoustic rows), local LF speeds (max |eigenvalue| over the stencil), WENO5 of the
// positive part from the left and of the negative part from the right, projection back.
template <int DIR>
__device__ __forceinline__ void weno_flux(const Consts& C, const Bufs& B, long long n, long long st,
                                          double* f) {
  constexpr int T1 = DIR == 0 ? 1 : 0;
  constexpr int T2 = DIR == 2 ? 1 : 2;
  const double* __restrict__ vel[3] = {B.u, B.v, B.w};
  // Roe average of nodes n and n + st
  double sl = sqrt(__ldg(B.rho + n)), sr = sqrt(__ldg(B.rho + n + st));
  double inv = 1.0 / (sl + sr);
  double wl = sl * inv, wr = sr * inv;
  double ua[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) ua[dd] = wl * __ldg(vel[dd] + n) + wr * __ldg(vel[dd] + n + st);
  double Ha = wl * __ldg(B.H + n) + wr * __ldg(B.H + n + st);
  double q2 = ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
  double ca = sqrt(C.gm1 * (Ha - 0.5 * q2));
  double ic = 1.0 / ca;
  double b1 = C.gm1 * ic * ic;
  double b2 = 0.5 * q2 * b1;
  double un_a = ua[DIR];

  // characteristic variables at the six stencil nodes
  double cw[5][6], cf[5][6];
  double lam0 = 0.0, lam1 = 0.0, lam4 = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    long long nn = n + (q - 2) * st;
    double rho = __ldg(B.rho + nn);
    double uu[3] = {__ldg(B.u + nn), __ldg(B.v + nn), __ldg(B.w + nn)};
    double H = __ldg(B.H + nn), p = __ldg(B.p + nn), cs = __ldg(B.c + nn);
    double un = uu[DIR];
    double run = rho * un;
    double udot = ua[0] * uu[0] + ua[1] * uu[1] + ua[2] * uu[2];
    double K = b2 + b1 * (H - udot);
    double b1p = b1 * p;
    double Aw = rho * K - b1p;
    double Af = run * K - b1p * un_a;
    double Bw = rho * (un_a - un) * ic;
    double Bf = (run * (un_a - un) - p) * ic;
    double d1 = uu[T1] - ua[T1], d2 = uu[T2] - ua[T2];
    cw[0][q] = 0.5 * (Aw + Bw);
    cf[0][q] = 0.5 * (Af + Bf);
    cw[1][q] = rho - Aw;
    cf[1][q] = run - Af;
    cw[2][q] = rho * d1;
    cf[2][q] = run * d1;
    cw[3][q] = rho * d2;
    cf[3][q] = run * d2;
    cw[4][q] = 0.5 * (Aw - Bw);
    cf[4][q] = 0.5 * (Af - Bf);
    lam0 = fmax(lam0, fabs(un - cs));
    lam1 = fmax(lam1, fabs(un));
    lam4 = fmax(lam4, fabs(un + cs));
  }
  double g[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double lam = k == 0 ? lam0 : (k == 4 ? lam4 : lam1);
    double gp[6], gm[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      gp[q] = 0.5 * (cf[k][q] + lam * cw[k][q]);
      gm[q] = 0.5 * (cf[k][q] - lam * cw[k][q]);
    }
    double np_, dp_, nm_, dm_;
    weno5_nd(gp[0], gp[1], gp[2], gp[3], gp[4], C.weno_eps, np_, dp_);
    weno5_nd(gm[5], gm[4], gm[3], gm[2], gm[1], C.weno_eps, nm_, dm_);
    g[k] = (np_ * dm_ + nm_ * dp_) / (dp_ * dm_);
  }
  // back to conserved variables with the right eigenvectors
  double gs = g[0] + g[1] + g[4];
  f[0] = gs;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) f[1 + dd] = gs * ua[dd];
  f[1 + DIR] += ca * (g[4] - g[0]);
  f[1 + T1] += g[2];
  f[1 + T2] += g[3];
  f[4] = Ha * (g[0] + g[4]) + un_a * ca * (g[4] - g[0]) + 0.5 * q2 * g[1] + ua[T1] * g[2] +
         ua[T2] * g[3];
}

// ------------------------------------------------------------------------------ face kernels

template <int L, int DIR>
__global__ void __launch_bounds__(256) k_faces(Dims d, Consts C, Bufs B) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.nf[DIR]) return;
  int i, j, k;
  face_node<DIR>(d, q, i, j, k);
  long long n = gidx(d, i, j, k);
  long long st = dir_stride(d, DIR);
  bool fl = face_flag<L>(C, B.theta, n, st);
  unsigned act = __activemask();
  unsigned m = __ballot_sync(act, fl);
  if (m) {
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(B.wcount + DIR, (unsigned)__popc(m));
    base = __shfl_sync(act, base, leader);
    if (fl) B.wl[DIR][base + __popc(m & ((1u << lane) - 1u))] = (int)q;
  }
  if (fl) return;
  double f[5];
  central_flux<L, DIR>(C, B, n, st, f);
  double* out = B.fh[DIR];
  long long nf = d.nf[DIR];
#pragma unroll
  for (int c = 0; c < 5; ++c) out[c * nf + q] = f[c];
}

template <int DIR>
__global__ void __launch_bounds__(128) k_weno(Dims d, Consts C, Bufs B) {
  unsigned cnt = *(volatile unsigned*)(B.wcount + DIR);
  long long nf = d.nf[DIR];
  long long st = dir_stride(d, DIR);
  double* out = B.fh[DIR];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x) {
    long long q = B.wl[DIR][t];
    int i, j, k;
    face_node<DIR>(d, q, i, j, k);
    double f[5];
    weno_flux<DIR>(C, B, gidx(d, i, j, k), st, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * nf + q] = f[c];
  }
}

// ------------------------------------------------------------------------------ assembly

// Viscous terms in Laplacian form at node n (Section 2.1 and Eqs. sigma, heat_vec):
//   V_i = mu lap u_i + mu/3 d_i(div) + d_j mu (d_j u_i + d_i u_j) - 2/3 div d_i mu,
//   V_E = u_i V_i + sigma_ij d_j u_i + k lap T + d_j k d_j T,  k = cp mu / Pr,
// first and second derivatives of order 2L; along y, d/dy = (1/y_eta) d/deta and
// d2/dy2 = (f_etaeta - (y_etaeta/y_eta) f_eta)/y_eta^2; d_i(div) from the ghost-filled div.
template <int L>
__device__ __forceinline__ void viscous_node(const Consts& C, const Bufs& B, const Dims& d, long long n,
                                             int j, double* V) {
  const long long sy = d.px, sz = d.plane;
  const double hy = __ldg(B.inv_hy + j), c2 = __ldg(B.c2y + j), c1 = __ldg(B.c1y + j);
  const double* __restrict__ fld[4] = {B.u, B.v, B.w, B.T};
  double du[3][3], lap[3], dT[3], lapT = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double s1, s2, d0, d1v, d2v, l0;
    dsum12<L>(fld[a], n, 1, C.a, C.b, s1, s2);
    d0 = s1 * C.inv_dx;
    l0 = s2 * C.inv_dx2;
    dsum12<L>(fld[a], n, sy, C.a, C.b, s1, s2);
    d1v = s1 * hy;
    l0 += s2 * c2 - s1 * c1;
    dsum12<L>(fld[a], n, sz, C.a, C.b, s1, s2);
    d2v = s1 * C.inv_dz;
    l0 += s2 * C.inv_dz2;
    if (a < 3) {
      du[a][0] = d0;
      du[a][1] = d1v;
      du[a][2] = d2v;
      lap[a] = l0;
    } else {
      dT[0] = d0;
      dT[1] = d1v;
      dT[2] = d2v;
      lapT = l0;
    }
  }
  double dmu[3], ddiv[3];
  dmu[0] = dsum<L>(B.mu, n, 1, C.a) * C.inv_dx;
  dmu[1] = dsum<L>(B.mu, n, sy, C.a) * hy;
  dmu[2] = dsum<L>(B.mu, n, sz, C.a) * C.inv_dz;
  ddiv[0] = dsum<L>(B.div, n, 1, C.a) * C.inv_dx;
  ddiv[1] = dsum<L>(B.div, n, sy, C.a) * hy;
  ddiv[2] = dsum<L>(B.div, n, sz, C.a) * C.inv_dz;
  const double mu = __ldg(B.mu + n);
  const double div = du[0][0] + du[1][1] + du[2][2];
  double Vm[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double s = dmu[0] * (du[a][0] + du[0][a]) + dmu[1] * (du[a][1] + du[1][a]) +
               dmu[2] * (du[a][2] + du[2][a]);
    Vm[a] = mu * lap[a] + mu * ddiv[a] * (1.0 / 3.0) + s - (2.0 / 3.0) * div * dmu[a];
  }
  const double uu[3] = {__ldg(B.u + n), __ldg(B.v + n), __ldg(B.w + n)};
  double work = uu[0] * Vm[0] + uu[1] * Vm[1] + uu[2] * Vm[2];
  // sigma_ij d_j u_i = mu [ sum_ij (d_j u_i + d_i u_j) d_j u_i - 2/3 div^2 ]
  double diss = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) diss += (du[a][b] + du[b][a]) * du[a][b];
  diss = mu * (diss - (2.0 / 3.0) * div * div);
  double heat = C.cp_pr * (mu * lapT + dmu[0] * dT[0] + dmu[1] * dT[1] + dmu[2] * dT[2]);
  V[0] = 0.0;
  V[1] = Vm[0];
  V[2] = Vm[1];
  V[3] = Vm[2];
  V[4] = work + diss + heat;
}

template <int L>
__global__ void __launch_bounds__(256) k_assemble(Dims d, Consts C, Bufs B, double* __restrict__ R) {
  __shared__ double sh[32];
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double fpart = 0.0;
  if (q < d.N) {
    int i = (int)(q % d.nx);
    long long r = q / d.nx;
    int j = (int)(r % d.ny);
    int k = (int)(r / d.ny);
    double res[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (C.convective) {
      long long qx = ((long long)k * d.ny + j) * (d.nx + 1) + i;
      long long qy = ((long long)k * (d.ny + 1) + j) * d.nx + i;
      long long qz = ((long long)k * d.ny + j) * d.nx + i;
      long long sxy = (long long)d.nx * d.ny;
      double hy = __ldg(B.inv_hy + j);
      bool wlo = C.wall_y && j == 0, whi = C.wall_y && j == d.ny - 1;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const double* fx = B.fh[0] + m * d.nf[0];
        const double* fy = B.fh[1] + m * d.nf[1];
        const double* fz = B.fh[2] + m * d.nf[2];
        double ylo = __ldg(fy + qy), yhi = __ldg(fy + qy + d.nx);
        // staggered wall interface: no mass, x/z momentum or energy crosses it
        if (m != 2) {
          if (wlo) ylo = 0.0;
          if (whi) yhi = 0.0;
        }
        res[m] = -((__ldg(fx + qx + 1) - __ldg(fx + qx)) * C.inv_dx + (yhi - ylo) * hy +
                   (__ldg(fz + qz + sxy) - __ldg(fz + qz)) * C.inv_dz);
      }
    }
    if (C.viscous) {
      double V[5];
      viscous_node<L>(C, B, d, gidx(d, i, j, k), j, V);
#pragma unroll
      for (int m = 1; m < 5; ++m) res[m] += V[m];
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) R[m * d.N + q] = res[m];
    fpart = res[1] * __ldg(B.vol + j);
  }
  if (C.forcing) {
    double s = block_sum(fpart, sh);
    if (threadIdx.x == 0) B.red[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------------------ launchers

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, cudaStream_t s) {
  unsigned nb = blocks_for(d.nf[dir], 256);
  if (C.L == 3) {
    if (dir == 0) k_faces<3, 0><<<nb, 256, 0, s>>>(d, C, B);
    else if (dir == 1) k_faces<3, 1><<<nb, 256, 0, s>>>(d, C, B);
    else k_faces<3, 2><<<nb, 256, 0, s>>>(d, C, B);
  } else {
    if (dir == 0) k_faces<2, 0><<<nb, 256, 0, s>>>(d, C, B);
    else if (dir == 1) k_faces<2, 1><<<nb, 256, 0, s>>>(d, C, B);
    else k_faces<2, 2><<<nb, 256, 0, s>>>(d, C, B);
  }
}

void launch_weno_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s) {
  if (dir == 0) k_weno<0><<<grid, 128, 0, s>>>(d, C, B);
  else if (dir == 1) k_weno<1><<<grid, 128, 0, s>>>(d, C, B);
  else k_weno<2><<<grid, 128, 0, s>>>(d, C, B);
}

void launch_assemble(const Dims& d, const Consts& C, const Bufs& B, double* R, cudaStream_t s) {
  if (C.L == 3)
    k_assemble<3><<<blocks_for(d.N, kRedBlock), kRedBlock, 0, s>>>(d, C, B, R);
  else
    k_assemble<2><<<blocks_for(d.N, kRedBlock), kRedBlock, 0, s>>>(d, C, B, R);
}

}  // namespace strm
