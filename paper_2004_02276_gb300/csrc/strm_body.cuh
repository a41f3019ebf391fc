// Device bodies of the hot-path kernels, shared by the single-grid kernels (strm_state.cu,
// strm_flux.cu) and the batched ensemble kernels (strm_batch.cu). Each body takes the grid, the
// constants and the buffers by reference and the block index it plays, so that a batched kernel
// can run the body of any instance of its table.
#pragma once

#include "strm_dev.cuh"

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
__device__ __forceinline__ void body_prims(const Dims& d, const Consts& C, const Bufs& B,
                                           const double* STRM_RO w, int want_cfl, int blk,
                                           double* sh) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  double spec = 0.0;
  if (q < d.N) {
    int i, j, k;
    node_ijk(d, q, i, j, k);
    const Nodes<double>& P = B.n64;
    double rho = w[q];
    double rs = rsqrt(rho);  // 1/rho and sqrt(rho) from one reciprocal square root
    double ir = rs * rs;
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
    B.lam[0][n] = u - c;
    B.lam[1][n] = u + c;
    B.lam[2][n] = v - c;
    B.lam[3][n] = v + c;
    B.lam[4][n] = ww - c;
    B.lam[5][n] = ww + c;
    P.mu[n] = viscosity(C.k64, C.visc_law, T);
    P.srho[n] = rho * rs;
    const double vel[3] = {u, v, ww};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const double m = w[(1 + dd) * d.N + q];
      B.mom[dd][n] = m;
      B.mflux[dd][n] = fma(m, vel[dd], p);
    }
    if (want_cfl)
      spec = (fabs(u) + c) * C.k64.inv_dx + (fabs(v) + c) * B.m64.inv_hy[j] + (fabs(ww) + c) * C.k64.inv_dz;
  }
  if (want_cfl) {
    double m = block_max(spec, sh);
    if (threadIdx.x == 0) B.red[blk] = m;
  }
}

// Reference state of the x row (j, k) for the deviation form of the mixed x faces' central
// flux: rho, u and H of the row's first node, from the conserved state, in FP32 with explicitly
// rounded operations (so that every thread of the row forms the same values). Any values
// constant along the row serve; these are close to the row's own. (v and w need none: the
// transverse velocities are small, so their FP32 copies already carry small absolute errors.)
__device__ __forceinline__ void xrow_ref(const Dims& d, const Consts& C, const double* w, int j, int k,
                                         float r[3]) {
  const long long q0 = ((long long)k * d.ny + j) * d.nx;
  const float rho = d2f(w[q0]);
  const float ir = __frcp_rn(rho);
  const float u = __fmul_rn(d2f(w[d.N + q0]), ir), v = __fmul_rn(d2f(w[2 * d.N + q0]), ir);
  const float ww = __fmul_rn(d2f(w[3 * d.N + q0]), ir), E = __fmul_rn(d2f(w[4 * d.N + q0]), ir);
  const float q2 = __fadd_rn(__fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v)), __fmul_rn(ww, ww));
  const float g = C.k32.gamma;
  r[0] = rho;
  r[1] = u;
  r[2] = __fsub_rn(__fmul_rn(g, E), __fmul_rn(__fmul_rn(0.5f, __fsub_rn(g, 1.f)), q2));  // E + p/rho
}

// Mixed precision: the fields the characteristic projection reads are formed in FP64 (rho, u,
// v, w, p, T, H, sqrt rho, rho u_d, rho u_d^2 + p); FP32 copies of all fields feed the FP32
// kernels, with c and mu(T) evaluated in FP32. The CFL partial is formed in FP32 (the FP64 pipe
// binds this kernel; the step needs no FP64 accuracy in this precision).
__device__ __forceinline__ void body_prims_mixed(const Dims& d, const Consts& C, const Bufs& B,
                                                 const double* STRM_RO w, int want_cfl, int blk,
                                                 double* sh) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  float spec = 0.f;
  if (q < d.N) {
    int i, j, k;
    node_ijk(d, q, i, j, k);
    const Nodes<double>& P = B.n64;
    const Nodes<float>& F = B.n32;
    double rho = w[q];
    double rs = rsqrt_nr(rho);
    double ir = rs * rs;
    const double m0 = w[d.N + q], m1 = w[2 * d.N + q], m2 = w[3 * d.N + q], rE = w[4 * d.N + q];
    double u = m0 * ir, v = m1 * ir, ww = m2 * ir;
    // p = (gamma - 1)(rho E - rho |u|^2 / 2) and H = (rho E + p)/rho: no FP64 temperature (the
    // FP32 copy comes from p and rho; ghost states form T from p and rho when they need it).
    // Explicit rounding: the same bits whichever kernel (single grid or batched) inlines this,
    // so that the FP32 CFL maxima and hence the step agree between them.
    const double ke2 = __fma_rn(m0, u, __fma_rn(m1, v, __dmul_rn(m2, ww)));
    double p = __dmul_rn(C.gm1, __fma_rn(-0.5, ke2, rE));
    double H = __dmul_rn(__dadd_rn(rE, p), ir);
    long long n = gidx(d, i, j, k);
    P.rho[n] = rho;
    P.u[n] = u;
    P.v[n] = v;
    P.w[n] = ww;
    P.p[n] = p;
    P.H[n] = H;
    P.srho[n] = rho * rs;
    const double vel[3] = {u, v, ww};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const double m = w[(1 + dd) * d.N + q];
      B.mom[dd][n] = m;
      B.mflux[dd][n] = fma(m, vel[dd], p);
    }
    float rf = d2f(rho), pf = d2f(p);
    float Tf = pf / (rf * C.k32.r_gas);
    float cf = sqrtf(C.k32.gamma * pf / rf);
    const float uf = d2f(u), vf = d2f(v), wf = d2f(ww);
    F.rho[n] = rf;
    F.u[n] = uf;
    F.v[n] = vf;
    F.w[n] = wf;
    F.p[n] = d2f(p - C.p_shift);  // shifted copy (see Consts::p_shift); c uses the full pf
    F.T[n] = Tf;
    F.H[n] = d2f(H);
    F.c[n] = cf;
    F.mu[n] = viscosity(C.k32, C.visc_law, Tf);
    // x-row deviations rho - rho_0, u - u_0, H - H_0 (FP64 differences, then FP32): the x faces'
    // central flux works on these, so its FP32 rounding scales with the row's variations
    float r[3];
    xrow_ref(d, C, w, j, k, r);
    const double xv[3] = {rho, u, H};
#pragma unroll
    for (int m = 0; m < 3; ++m) B.xdev[m][n] = d2f(xv[m] - f2d(r[m]));
    if (i == 0) {
      const long long rs = (long long)d.ny * d.nz, row = (long long)k * d.ny + j;
#pragma unroll
      for (int m = 0; m < 3; ++m) B.xref[m * rs + row] = r[m];
    }
    if (want_cfl)  // FP32 spectral radius: the step needs no more than FP32 accuracy here
      spec = (fabsf(uf) + cf) * C.k32.inv_dx + (fabsf(vf) + cf) * B.m32.inv_hy[j] + (fabsf(wf) + cf) * C.k32.inv_dz;
  }
  if (want_cfl) {
    float m = block_max_f(spec, reinterpret_cast<float*>(sh));
    if (threadIdx.x == 0) B.red[blk] = f2d(m);
  }
}

// dt from the CFL partials (or the fixed step), and the simulated time.
__device__ __forceinline__ void body_dt_finalize(const Bufs& B, int nparts, double cfl, double dt_fixed,
                                                 double* sh) {
  double m = 0.0;
  if (dt_fixed <= 0.0)
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) m = nanmax(m, B.red[t]);
  m = block_max(m, sh);
  if (threadIdx.x == 0) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl / m;
    B.scal[kScalDt] = dt;
    B.scal[kScalCflMax] = m;
    B.scal[kScalTime] += dt;
    // the stage weights of this step, once, instead of two FP64 products in every thread of
    // every stage update
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      B.scal[kScalAdt + s] = rk_alpha(s) * dt;
      B.scal[kScalBdt + s] = rk_beta(s) * dt;
    }
  }
}

// ---------------------------------------------------------------------------------- ghost fills

// Thread layout of a face ghost fill: x faces (2G * ny * nz), then y faces (nx * 2G * nz), then
// z faces (nx * ny * 2G). The ghost node is (i, j, k); side is 0 for the min face, 1 for the max
// face; layer 0..G-1 counts away from the boundary. Edges and corners are never read.
__device__ __forceinline__ bool ghost_target(const Dims& d, long long q, int& face, int& side, int& layer,
                                             int& i, int& j, int& k) {
  long long nxf = 2LL * G * d.ny * d.nz, nyf = 2LL * G * d.nx * d.nz, nzf = 2LL * G * d.nx * d.ny;
  if (q < nxf) {
    int g = (int)(q % (2 * G));
    long long r = q / (2 * G);
    j = (int)(r % d.ny);
    k = (int)(r / d.ny);
    side = g < G ? 0 : 1;
    layer = g < G ? g : g - G;
    i = side == 0 ? -1 - layer : d.nx + layer;
    face = 0;
    return true;
  }
  q -= nxf;
  if (q < nyf) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    int g = (int)(r % (2 * G));
    k = (int)(r / (2 * G));
    side = g < G ? 0 : 1;
    layer = g < G ? g : g - G;
    j = side == 0 ? -1 - layer : d.ny + layer;
    face = 1;
    return true;
  }
  q -= nyf;
  if (q < nzf) {
    i = (int)(q % d.nx);
    long long r = q / d.nx;
    j = (int)(r % d.ny);
    int g = (int)(r / d.ny);
    side = g < G ? 0 : 1;
    layer = g < G ? g : g - G;
    k = side == 0 ? -1 - layer : d.nz + layer;
    face = 2;
    return true;
  }
  return false;
}

// Primitive state of a node (FP64).
struct PState {
  double rho, u, v, w, p, T;
};

// Mixed precision stores no FP64 temperature: T = p / (rho R) for the nodes a ghost state reads.
__device__ __forceinline__ PState load_pstate(const Consts& C, const Nodes<double>& P, long long n) {
  const double rho = P.rho[n], p = P.p[n];
  return PState{rho, P.u[n], P.v[n], P.w[n], p, C.mixed ? p / (rho * C.r_gas) : P.T[n]};
}

__device__ __forceinline__ PState pstate_from_prims(const Consts& C, const double* q) {
  // (rho, u, v, w, p) -> with T = p / (rho R)
  return PState{q[0], q[1], q[2], q[3], q[4], q[4] / (q[0] * C.r_gas)};
}

// Write a ghost state: FP64 fields (all of them in FP64 precision; the projection's in mixed
// precision) and, in mixed precision, the FP32 copies with c and mu(T) in FP32.
__device__ __forceinline__ void store_pstate(const Consts& C, const Bufs& B, long long dst, const PState& g) {
  const Nodes<double>& P = B.n64;
  P.rho[dst] = g.rho;
  P.u[dst] = g.u;
  P.v[dst] = g.v;
  P.w[dst] = g.w;
  P.p[dst] = g.p;
  P.T[dst] = g.T;
  // explicit rounding: the same bits whichever kernel (single grid or batched) inlines this
  double q2 = __fma_rn(g.u, g.u, __fma_rn(g.v, g.v, __dmul_rn(g.w, g.w)));
  double H = __fma_rn(C.cp, g.T, __dmul_rn(0.5, q2));
  P.H[dst] = H;
  P.srho[dst] = sqrt(g.rho);
  const double gm[3] = {__dmul_rn(g.rho, g.u), __dmul_rn(g.rho, g.v), __dmul_rn(g.rho, g.w)};
  const double gv[3] = {g.u, g.v, g.w};
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    B.mom[dd][dst] = gm[dd];
    B.mflux[dd][dst] = __fma_rn(gm[dd], gv[dd], g.p);
  }
  if (!C.mixed) {
    double c = sqrt(C.gamma * g.p / g.rho);
    P.c[dst] = c;
    B.lam[0][dst] = g.u - c;
    B.lam[1][dst] = g.u + c;
    B.lam[2][dst] = g.v - c;
    B.lam[3][dst] = g.v + c;
    B.lam[4][dst] = g.w - c;
    B.lam[5][dst] = g.w + c;
    P.mu[dst] = viscosity(C.k64, C.visc_law, g.T);
  } else {
    const Nodes<float>& F = B.n32;
    float rf = d2f(g.rho), pf = d2f(g.p), Tf = d2f(g.T);
    F.rho[dst] = rf;
    F.u[dst] = d2f(g.u);
    F.v[dst] = d2f(g.v);
    F.w[dst] = d2f(g.w);
    F.p[dst] = d2f(__dadd_rn(g.p, -C.p_shift));  // shifted copy (see Consts::p_shift)
    F.T[dst] = Tf;
    F.H[dst] = d2f(H);
    F.c[dst] = sqrtf(C.k32.gamma * pf / rf);
    F.mu[dst] = viscosity(C.k32, C.visc_law, Tf);
  }
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

__device__ __forceinline__ void copy_ghost(const Consts& C, const Bufs& B, long long dst, long long src) {
  copy_node(B.n64, dst, src, !C.mixed);
  B.n64.srho[dst] = B.n64.srho[src];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    B.mom[dd][dst] = B.mom[dd][src];
    B.mflux[dd][dst] = B.mflux[dd][src];
  }
  if (C.mixed) {
    copy_node(B.n32, dst, src, true);
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f) B.lam[f][dst] = B.lam[f][src];
  }
}

// Isothermal no-slip staggered wall: the ghost mirrors an interior node across the wall
// interface with reversed velocity, T_g = 2 T_w - T, p_g = p, rho_g = p_g/(R T_g).
__device__ __forceinline__ PState wall_pstate(const Consts& C, const PState& s) {
  PState g;
  g.u = -s.u;
  g.v = -s.v;
  g.w = -s.w;
  g.p = s.p;
  g.T = 2.0 * C.t_wall - s.T;
  g.rho = g.p / (C.r_gas * g.T);
  return g;
}

// Non-reflecting characteristic ghost (Section 3.2, characteristic decomposition normal to the
// boundary): eigenvectors of the Euler flux along dir at the boundary node b; a characteristic
// variable whose speed points out of the domain (outward = +1 at a max face, -1 at a min face)
// is extrapolated from b at zeroth order, the others come from the reference state r. The left
// eigenvector rows are applied through the acoustic scalars A = b2 x0 + b1 (x4 - u.m),
// Bn = (u_n x0 - m_n)/c and the shear rows; the right eigenvectors map back.
__device__ __forceinline__ PState char_pstate(const Consts& C, const PState& b, const PState& r, int dir,
                                              int outward) {
  const double ub[3] = {b.u, b.v, b.w};
  const int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
  double q2 = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
  double H = C.cp * b.T + 0.5 * q2;
  double c = sqrt(C.gamma * b.p / b.rho);
  double ic = 1.0 / c;
  double b1 = C.gm1 * ic * ic, b2 = 0.5 * q2 * b1;
  double un = ub[dir];
  // conserved states of b and r
  double xb[5] = {b.rho, b.rho * b.u, b.rho * b.v, b.rho * b.w, b.rho * (C.cv * b.T + 0.5 * q2)};
  double xr[5] = {r.rho, r.rho * r.u, r.rho * r.v, r.rho * r.w,
                  r.rho * (C.cv * r.T + 0.5 * (r.u * r.u + r.v * r.v + r.w * r.w))};
  double Wb[5], Wr[5];
  const double* xs[2] = {xb, xr};
  double* Ws[2] = {Wb, Wr};
  for (int s = 0; s < 2; ++s) {
    const double* x = xs[s];
    double um = ub[0] * x[1] + ub[1] * x[2] + ub[2] * x[3];
    double A = b2 * x[0] + b1 * (x[4] - um);
    double Bn = (un * x[0] - x[1 + dir]) * ic;
    Ws[s][0] = 0.5 * (A + Bn);
    Ws[s][1] = x[0] - A;
    Ws[s][2] = x[1 + t1] - ub[t1] * x[0];
    Ws[s][3] = x[1 + t2] - ub[t2] * x[0];
    Ws[s][4] = 0.5 * (A - Bn);
  }
  const double lam[5] = {un - c, un, un, un, un + c};
  double W[5];
  for (int k = 0; k < 5; ++k) W[k] = (outward * lam[k] > 0.0) ? Wb[k] : Wr[k];
  double gs = W[0] + W[1] + W[4];
  double x[5];
  x[0] = gs;
  for (int dd = 0; dd < 3; ++dd) x[1 + dd] = gs * ub[dd];
  x[1 + dir] += c * (W[4] - W[0]);
  x[1 + t1] += W[2];
  x[1 + t2] += W[3];
  x[4] = H * (W[0] + W[4]) + un * c * (W[4] - W[0]) + 0.5 * q2 * W[1] + ub[t1] * W[2] + ub[t2] * W[3];
  PState g;
  g.rho = x[0];
  double ir = 1.0 / g.rho;
  g.u = x[1] * ir;
  g.v = x[2] * ir;
  g.w = x[3] * ir;
  g.T = (x[4] * ir - 0.5 * (g.u * g.u + g.v * g.v + g.w * g.w)) * C.inv_cv;
  g.p = g.rho * C.r_gas * g.T;
  return g;
}

// Rescaled recycling inflow (reading): ghost plane i = -1-layer takes interior plane
// i_recycle - layer with the wall-normal coordinate stretched by s = delta_r / delta_in: the
// value at height h is the recycled plane's value at height s h, u, v, w, T, p interpolated
// linearly between nodes (below the first node between the wall state u = v = w = 0, T = T_w,
// p = p_0 and the first node; above the last node, the last node's value); rho = p / (R T).
__device__ __forceinline__ PState recycle_pstate(const Dims& d, const Consts& C, const Bufs& B, int layer,
                                                 int j, int k) {
  const Nodes<double>& P = B.n64;
  double s = B.scal[kScalRecycle];
  double ht = s * STRM_LDG(B.hy + j);
  int is = C.i_recycle - layer;
  // first node jb with h[jb] >= ht
  int lo = 0, hi = d.ny;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (STRM_LDG(B.hy + mid) < ht) lo = mid + 1;
    else hi = mid;
  }
  int jb = lo;
  PState a, bb;
  double alpha;
  if (jb == d.ny) {
    bb = load_pstate(C, P, gidx(d, is, d.ny - 1, k));
    a = bb;
    alpha = 1.0;
  } else {
    bb = load_pstate(C, P, gidx(d, is, jb, k));
    double ha, hb = STRM_LDG(B.hy + jb);
    if (jb == 0) {
      a = PState{0.0, 0.0, 0.0, 0.0, bb.p, C.t_wall};
      ha = 0.0;
    } else {
      a = load_pstate(C, P, gidx(d, is, jb - 1, k));
      ha = STRM_LDG(B.hy + jb - 1);
    }
    alpha = (ht - ha) / (hb - ha);
  }
  // linear interpolation with explicit rounding (no contraction left to the compiler)
  double am = __dadd_rn(1.0, -alpha);
  auto lerp = [&](double fa, double fb) { return __fma_rn(alpha, fb, __dmul_rn(am, fa)); };
  PState g;
  g.T = lerp(a.T, bb.T);
  g.u = lerp(a.u, bb.u);
  g.v = lerp(a.v, bb.v);
  g.w = lerp(a.w, bb.w);
  g.p = lerp(a.p, bb.p);
  g.rho = g.p / (C.r_gas * g.T);
  return g;
}

// Digital-filter inflow ghost (every layer of the x-min face): mean profile plus the velocity
// fluctuations a Psi (Cholesky factor of the Reynolds stresses times the filtered plane), the
// temperature from the strong Reynolds analogy cp T' + U u' = 0, and the inflow pressure.
__device__ __forceinline__ PState df_pstate(const Dims& d, const Consts& C, const Bufs& B, int j, int k) {
  const double* P = B.df_prof;
  const int ny = d.ny;
  double U = STRM_LDG(P + j), V = STRM_LDG(P + ny + j), Tm = STRM_LDG(P + 2 * ny + j);
  double a11 = STRM_LDG(P + 3 * ny + j), a21 = STRM_LDG(P + 4 * ny + j), a22 = STRM_LDG(P + 5 * ny + j),
         a33 = STRM_LDG(P + 6 * ny + j);
  long long plane = (long long)d.nz * ny, at = (long long)k * ny + j;
  double p0 = STRM_LDG(B.df_psi + at), p1 = STRM_LDG(B.df_psi + plane + at), p2 = STRM_LDG(B.df_psi + 2 * plane + at);
  double up = a11 * p0, vp = fma(a21, p0, a22 * p1), wp = a33 * p2;
  PState g;
  g.u = U + up;
  g.v = V + vp;
  g.w = wp;
  g.T = Tm - U * up / C.cp;
  g.p = C.df_p;
  g.rho = g.p / (C.r_gas * g.T);
  return g;
}

// Ghost node primitives by face kind (both precisions).
__device__ __forceinline__ void body_ghost_prims(const Dims& d, const Consts& C, const Bufs& B,
                                                 long long nthreads, int blk) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, side, layer, i, j, k;
  if (!ghost_target(d, q, face, side, layer, i, j, k)) return;
  if (!stencil_ok(d, i, j, k, 0, 0, 0, kDbgGhost)) return;
  const Nodes<double>& P = B.n64;
  long long dst = gidx(d, i, j, k);
  int kind = face == 2 ? kBcPeriodic : C.bc[2 * face + side];
  if (kind == kBcPeriodic) {
    int si = face == 0 ? wrapi(i, d.nx) : i, sj = face == 1 ? wrapi(j, d.ny) : j;
    int sk = face == 2 ? wrapi(k, d.nz) : k;
    if (!stencil_ok(d, si, sj, sk, 0, 0, 0, kDbgGhost)) return;
    const long long src = gidx(d, si, sj, sk);
    copy_ghost(C, B, dst, src);
    if (C.mixed && face == 0)  // the source node lies in the same x row: same reference
#pragma unroll
      for (int m = 0; m < 3; ++m) B.xdev[m][dst] = B.xdev[m][src];
    return;
  }
  if constexpr (kDebug) {  // the interior source node of the face kinds below
    int si = face == 0 ? (side == 0 ? 0 : d.nx - 1) : i, sj = face == 1 ? (side == 0 ? 0 : d.ny - 1) : j;
    if (kind == kBcRecycle) si = C.i_recycle - layer;
    if (!stencil_ok(d, si, sj, k, 0, 0, 0, kDbgGhost) || si < 0 || si >= d.nx) return;
    if (kind == kBcDigitalFilter && !index_ok(d, (long long)k * d.ny + j, (long long)d.nz * d.ny, kDbgInflow)) return;
  }
  PState g;
  if (kind == kBcWall) {
    int jm = side == 0 ? layer : d.ny - 1 - layer;  // j=-1-l <-> l, j=ny+l <-> ny-1-l
    g = wall_pstate(C, load_pstate(C, P, gidx(d, i, jm, k)));
  } else if (kind == kBcRecycle) {
    g = recycle_pstate(d, C, B, layer, j, k);
  } else if (kind == kBcDigitalFilter) {
    g = df_pstate(d, C, B, j, k);
  } else {  // characteristic
    int ib = face == 0 ? (side == 0 ? 0 : d.nx - 1) : i;
    int jb = face == 1 ? (side == 0 ? 0 : d.ny - 1) : j;
    PState bs = load_pstate(C, P, gidx(d, ib, jb, k));
    PState rs;
    if (face == 0) {
      // outflow-type face: the boundary state at the reference pressure (a subsonic outflow
      // only prescribes the far-field pressure; the plane crosses the boundary layer)
      rs = bs;
      rs.p = C.ref[4];
      rs.T = rs.p / (rs.rho * C.r_gas);
    } else {
      bool post = C.shock && side == 1 && (i + 0.5) * C.dx >= C.x_foot;
      rs = pstate_from_prims(C, post ? C.shock_ref : C.ref);
    }
    g = char_pstate(C, bs, rs, face, side == 0 ? -1 : 1);
  }
  store_pstate(C, B, dst, g);
  if (C.mixed && face == 0) {  // x-row deviations of the ghost state (reference from k_prims)
    const long long rs = (long long)d.ny * d.nz, row = (long long)k * d.ny + j;
    const double xv[3] = {g.rho, g.u, P.H[dst]};
#pragma unroll
    for (int m = 0; m < 3; ++m) B.xdev[m][dst] = d2f(xv[m] - f2d(B.xref[m * rs + row]));
  }
}

// theta and the node divergence: periodic copies, even mirror across a wall, copy of the
// boundary node at characteristic and inflow faces.
template <typename R>
__device__ __forceinline__ void body_ghost_scalars(const Dims& d, const Consts& C, const Bufs& B,
                                                   long long nthreads, int blk) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  if (q >= nthreads) return;
  int face, side, layer, i, j, k;
  if (!ghost_target(d, q, face, side, layer, i, j, k)) return;
  const Nodes<R>& P = nodes<R>(B);
  int si = theta_source(i, d.nx, C.bc[0], C.bc[1]);
  int sj = theta_source(j, d.ny, C.bc[2], C.bc[3]);
  int sk = theta_source(k, d.nz, kBcPeriodic, kBcPeriodic);
  if (!stencil_ok(d, i, j, k, 0, 0, 0, kDbgGhost) || !stencil_ok(d, si, sj, sk, 0, 0, 0, kDbgGhost)) return;
  long long dst = gidx(d, i, j, k), src = gidx(d, si, sj, sk);
  P.theta[dst] = P.theta[src];
  if (!std::is_same<R, double>::value) B.n64.theta[dst] = B.n64.theta[src];  // mixed: switch field
  P.div[dst] = P.div[src];
}

// Spanwise mean of u at the recycling plane, one block per row j (fixed reduction order).
__device__ __forceinline__ void body_recycle_mean(const Dims& d, const Consts& C, const Bufs& B, int j,
                                                  double* sh) {
  double s = 0.0;
  for (int k = threadIdx.x; k < d.nz; k += blockDim.x) s += B.n64.u[gidx(d, C.i_recycle, j, k)];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) B.ubar[j] = s / d.nz;
}

// delta_r: the height where the spanwise-mean u first reaches 0.99 of the reference u (linear
// interpolation from the wall, where u = 0); s = delta_r / delta_in, 1 if never reached.
__device__ __forceinline__ void body_recycle_scale(const Dims& d, const Consts& C, const Bufs& B) {
  double target = 0.99 * C.ref[1], pu = 0.0, ph = 0.0, s = 1.0;
  for (int j = 0; j < d.ny; ++j) {
    double ub = B.ubar[j], h = B.hy[j];
    if (ub >= target) {
      double dr = ph + (target - pu) * (h - ph) / (ub - pu);
      s = dr / C.delta_in;
      break;
    }
    pu = ub;
    ph = h;
  }
  B.scal[kScalRecycle] = s;
}

// ---------------------------------------------------------------------------------- sensor

// Ducros sensor (Eq. sensor) at the interior nodes; the node divergence is kept for the
// viscous terms.
// Block-aggregated append of q to one compacted list (every thread of the block calls it).
__device__ __forceinline__ void block_append1(bool mine, int q, int* list, unsigned* count) {
  __shared__ unsigned s_w[32], s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  unsigned m = __ballot_sync(0xffffffffu, mine);
  if (lane == 0) s_w[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < nwarp; ++w) {
      unsigned c = s_w[w];
      s_w[w] = t;
      t += c;
    }
    s_base = t ? atomicAdd(count, t) : 0u;
  }
  __syncthreads();
  if (mine) list[s_base + s_w[warp] + __popc(m & ((1u << lane) - 1u))] = q;
}

// Node of sensor thread t for a part of the grid: region 0 all interior nodes; region 1 the
// nodes at least L from every face of the box (the inner box), whose stencils read no ghost
// node, so they can run while the ghost layers are being filled; region 2 the others (the
// shell), enumerated as the L planes at each z end, then the L rows at each y end of the
// remaining planes, then the L nodes at each x end of the remaining rows. Region 1 and 2 are
// used only when the inner box is not empty.
__device__ __forceinline__ bool sensor_node(const Dims& d, int region, int L, long long t, long long& q) {
  const long long nx = d.nx, ny = d.ny, nz = d.nz;
  const long long bx = nx - 2 * L, by = ny - 2 * L, bz = nz - 2 * L;
  long long i, j, k;
  if (region == 0) {
    q = t;
    return t < d.N;
  }
  if (region == 1) {
    if (t >= bx * by * bz) return false;
    i = t % bx;
    const long long r = t / bx;
    j = r % by;
    k = r / by;
    q = ((k + L) * ny + (j + L)) * nx + (i + L);
    return true;
  }
  const long long zn = 2 * L * nx * ny, yn = bz * 2 * L * nx, xn = bz * by * 2 * L;
  if (t < zn) {  // z-end planes
    const long long p = t / (nx * ny), r = t % (nx * ny);
    k = p < L ? p : nz - 2 * L + p;
    j = r / nx;
    i = r % nx;
  } else if (t < zn + yn) {  // y-end rows of the inner planes
    const long long u = t - zn, row = u / nx;
    i = u % nx;
    k = L + row / (2 * L);
    const long long jr = row % (2 * L);
    j = jr < L ? jr : ny - 2 * L + jr;
  } else if (t < zn + yn + xn) {  // x-end nodes of the inner rows
    const long long u = t - zn - yn, ir = u % (2 * L), row = u / (2 * L);
    i = ir < L ? ir : nx - 2 * L + ir;
    j = L + row % by;
    k = L + row / by;
  } else {
    return false;
  }
  q = (k * ny + j) * nx + i;
  return true;
}

template <int L, typename R>
__device__ __forceinline__ void body_sensor(const Dims& d, const Consts& C, const Bufs& B, int blk,
                                            int region = 0) {
  long long q = 0;  // set by sensor_node for the threads that own a node
  const bool mine = sensor_node(d, region, L, (long long)blk * blockDim.x + threadIdx.x, q);
  if constexpr (!std::is_same<R, double>::value) {
    // mixed precision: FP32 theta; the switch decides on an FP64 theta field, which holds the
    // FP32 value, except at the nodes whose FP32 theta falls within 0.2 % of the threshold
    // (far wider than its FP32 error): those are listed here and get the FP64 theta from the
    // FP64 velocities (body_band_theta), so the decisions are the ones FP64 takes on this state
    bool valid = mine, band = false;
    if (valid) {
      int i, j, k;
      node_ijk(d, q, i, j, k);
      const Nodes<R>& P = nodes<R>(B);
      R div;
      if (!stencil_ok(d, i, j, k, 0, L, L, kDbgNode) || !stencil_ok(d, i, j, k, 1, L, L, kDbgNode) ||
          !stencil_ok(d, i, j, k, 2, L, L, kDbgNode))
        i = j = k = 0;  // (debug builds) keep the block's barrier: compute at a safe node
      R th = theta_node<L, R>(d, C, B, i, j, k, div);
      long long n = gidx(d, i, j, k);
      P.theta[n] = th;
      P.div[n] = div;
      B.n64.theta[n] = f2d(th);
      const R thr = coefs<R>(C).theta_thr;
      band = C.weno_mode == 1 && fabs(th - thr) <= R(0.002) * thr;
    }
    block_append1(band, (int)q, B.band, B.wcount + 3);
    return;
  }
  if (!mine) return;
  int i, j, k;
  node_ijk(d, q, i, j, k);
  if (!stencil_ok(d, i, j, k, 0, L, L, kDbgNode) || !stencil_ok(d, i, j, k, 1, L, L, kDbgNode) ||
      !stencil_ok(d, i, j, k, 2, L, L, kDbgNode))
    return;
  const Nodes<R>& P = nodes<R>(B);
  R div;
  if constexpr (std::is_same<R, double>::value) {
    // FP64: the velocity gradients are kept for the viscous terms
    double g9[9];
    double th = theta_node<L, double>(d, C, B, i, j, k, div, g9);
#pragma unroll
    for (int c = 0; c < 9; ++c) B.grad[c * d.N + q] = g9[c];
    long long n = gidx(d, i, j, k);
    P.theta[n] = th;
    P.div[n] = div;
  } else {
    R th = theta_node<L, R>(d, C, B, i, j, k, div);
    long long n = gidx(d, i, j, k);
    P.theta[n] = th;
    P.div[n] = div;
  }
}

// Mixed precision: the FP64 theta at the listed near-threshold nodes (grid-stride loop).
template <int L>
__device__ __forceinline__ void body_band_theta(const Dims& d, const Consts& C, const Bufs& B, long long t0,
                                                long long tstride) {
  long long cnt = B.wcount[3];
  for (long long t = t0; t < cnt; t += tstride) {
    long long q = B.band[t];
    if (!index_ok(d, q, d.N, kDbgList)) continue;
    int i, j, k;
    node_ijk(d, q, i, j, k);
    double dv;
    B.n64.theta[gidx(d, i, j, k)] = theta_node<L, double>(d, C, B, i, j, k, dv);
  }
}

// ---------------------------------------------------------------------------------- RK, forcing

// Forcing of the mass flow rate: f = -(sum_V vol R_rhou) / V_total from the assembly partials.
__device__ __forceinline__ void body_force_finalize(const Bufs& B, int nparts, double inv_vtot, double* sh) {
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += B.red[t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) B.scal[kScalForce] = -s * inv_vtot;
}

// Stage update of Eq. RK: w <- w + dt (alpha R_old + beta R), R includes the forcing terms
// R_rhou += f, R_rhoE += f u (Eqs. 1b, 1c); R_old <- R. One thread per node, five fields. FP64
// in both precisions.
__device__ __forceinline__ void body_rk_update(const Dims& d, const Consts& C, const Bufs& B,
                                               double* STRM_RO w, double* STRM_RO r_old,
                                               int stage, int blk) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  double f = C.forcing ? B.scal[kScalForce] : 0.0;
  const double ad = B.scal[kScalAdt + stage], bd = B.scal[kScalBdt + stage];
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
    if (stage != 0) wn += ad * r_old[e];  // alpha_0 = 0
    w[e] = wn;
    r_old[e] = rr;
  }
}

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
// encflux): f_phi = 2 sum_l a_l sum_{m<l} (rho, u_n, phi)~_{n-m,l}. With the pair weight
// q = a_l (rho_a + rho_b)(u_a + u_b)/4 this is sum_{l,m} q (phi_a + phi_b) (the 1/4 is carried in
// the coefficients a_l/4, and f_rho = 2 sum q); the pressure enters the normal momentum as
// sum_l a_l sum_m (p_a + p_b) = sum_r ap_r (p_{n-r} + p_{n+1+r}), ap_r = a_{r+1} + .. + a_L,
// r = 0..L-1, since the pressure sum is linear. R is the arithmetic precision; in mixed
// precision the FP32 pressure copy is p - p_shift, so the face flux is short of the constant
// p_shift, as every mixed face flux is (the constant cancels in the flux differences).
template <int L, int DIR, typename R>
__device__ __forceinline__ void central_flux(const Consts& C, const Bufs& B, long long n, long long st,
                                             R* f) {
  const Nodes<R>& P = nodes<R>(B);
  const R* aq = coefs<R>(C).aq;  // a_l / 4
  const R* apc = coefs<R>(C).ap;  // a_{r+1} + .. + a_L
  const R* STRM_RO ud = DIR == 0 ? P.u : (DIR == 1 ? P.v : P.w);
  R a0 = R(0), a1 = R(0), a2 = R(0), a3 = R(0), a4 = R(0), ap = R(0);
#pragma unroll
  for (int r = 0; r < L; ++r) ap = fma(apc[r], STRM_LDG(P.p + n - r * st) + STRM_LDG(P.p + n + (r + 1) * st), ap);
#pragma unroll
  for (int l = 1; l <= L; ++l) {
#pragma unroll
    for (int m = 0; m < l; ++m) {
      long long ia = n - m * st, ib = n + (l - m) * st;
      R q = (aq[l] * (STRM_LDG(P.rho + ia) + STRM_LDG(P.rho + ib))) * (STRM_LDG(ud + ia) + STRM_LDG(ud + ib));
      a0 += q;
      a1 = fma(q, STRM_LDG(P.u + ia) + STRM_LDG(P.u + ib), a1);
      a2 = fma(q, STRM_LDG(P.v + ia) + STRM_LDG(P.v + ib), a2);
      a3 = fma(q, STRM_LDG(P.w + ia) + STRM_LDG(P.w + ib), a3);
      a4 = fma(q, STRM_LDG(P.H + ia) + STRM_LDG(P.H + ib), a4);
    }
  }
  f[0] = R(2) * a0;
  f[1] = a1;
  f[2] = a2;
  f[3] = a3;
  f[4] = a4;
  f[1 + DIR] += ap;
}

// Mixed precision, x faces: the same split flux from the x-row deviations. With the row's
// reference (rho_0, u_0, H_0; v_0 = w_0 = 0) and the pair sums S_rho = rho'_a + rho'_b, S_u, S_H
// of the deviations, (rho_a + rho_b) = 2 rho_0 + S_rho and so on, each pair's terms split into the
// constant a_l rho_0 u_0 (1, 2 u_0, 2 H_0) and the rest,
//   q' = a_l/4 [S_u (2 rho_0 + S_rho) + 2 u_0 S_rho],
//   f_rho gets 2 q',  f_phi gets K_l S_phi + q' (2 phi_0 + S_phi),  K_l = a_l rho_0 u_0,
// (phi = u, H; for v and w, whose reference is 0, (K_l + q') S_phi with the full FP32 sums), all
// in FP32. The constant parts add up to (rho_0 u_0)(1, u_0, 0, 0, H_0) (consistency,
// 8 sum_l l a_l/4 = 1): the same for every face of the row, so they cancel in the flux
// differences and are left out; the row's WENO faces subtract them too (xrow_flux_const). The
// FP32 rounding then scales with the deviations instead of the values (the x momentum flux
// rho u^2 + p is of order one). The pressure part is as in central_flux.
template <int L>
__device__ __forceinline__ void central_flux_xdev(const Dims& d, const Consts& C, const Bufs& B, long long n,
                                                  int j, int k, float* f) {
  const Nodes<float>& P = B.n32;
  const float* aq = C.k32.aq;
  const float* apc = C.k32.ap;
  const long long rs = (long long)d.ny * d.nz, row = (long long)k * d.ny + j;
  const float r0 = B.xref[row], u0 = B.xref[rs + row], H0 = B.xref[2 * rs + row];
  const float* STRM_RO Dr = B.xdev[0];
  const float* STRM_RO Du = B.xdev[1];
  const float* STRM_RO DH = B.xdev[2];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, ap = 0.f;
#pragma unroll
  for (int r = 0; r < L; ++r) ap = fmaf(apc[r], STRM_LDG(P.p + n - r) + STRM_LDG(P.p + n + r + 1), ap);
  const float r2 = 2.f * r0, u2 = 2.f * u0, H2 = 2.f * H0;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const float Kl = (4.f * aq[l]) * (r0 * u0);
#pragma unroll
    for (int m = 0; m < l; ++m) {
      const long long ia = n - m, ib = n + l - m;
      const float Sr = STRM_LDG(Dr + ia) + STRM_LDG(Dr + ib), Su = STRM_LDG(Du + ia) + STRM_LDG(Du + ib);
      const float SH = STRM_LDG(DH + ia) + STRM_LDG(DH + ib);
      const float Sv = STRM_LDG(P.v + ia) + STRM_LDG(P.v + ib), Sw = STRM_LDG(P.w + ia) + STRM_LDG(P.w + ib);
      const float qp = aq[l] * fmaf(Su, r2 + Sr, u2 * Sr);
      const float qf = Kl + qp;
      a0 += qp;
      a1 = fmaf(Kl, Su, fmaf(qp, u2 + Su, a1));
      a2 = fmaf(qf, Sv, a2);
      a3 = fmaf(qf, Sw, a3);
      a4 = fmaf(Kl, SH, fmaf(qp, H2 + SH, a4));
    }
  }
  f[0] = 2.f * a0;
  f[1] = a1 + ap;
  f[2] = a2;
  f[3] = a3;
  f[4] = a4;
}

// The constant the deviation-form x flux leaves out, (rho_0 u_0) c (1, u_0, 0, 0, H_0) with
// c = 8 sum_l l a_l/4 in the FP32 coefficients, taken off the x WENO faces of mixed precision
// so that every face of the row carries the same offset.
__device__ __forceinline__ void xrow_flux_const(const Dims& d, const Consts& C, const Bufs& B, int j, int k,
                                                float* c5) {
  const long long rs = (long long)d.ny * d.nz, row = (long long)k * d.ny + j;
  float s = 0.f;
  for (int l = 1; l <= C.L; ++l) s = fmaf((float)l, C.k32.aq[l], s);
  const float c0 = (8.f * s) * (B.xref[row] * B.xref[rs + row]);
  c5[0] = c0;
  c5[1] = c0 * B.xref[rs + row];
  c5[2] = 0.f;
  c5[3] = 0.f;
  c5[4] = c0 * B.xref[2 * rs + row];
}

// ------------------------------------------------------------------------------ WENO5

// Jiang-Shu WENO5 at i+1/2 from f_{i-2..i+2} = (f0..f4), written in first differences a..d of
// the stencil. Each smoothness indicator is a quadratic form in two differences; completing the
// square gives
//   12 beta_0 = 16 [(a - 11b/8)^2 + (39/64) b^2],   12 beta_1 = 16 [(b - 5c/8)^2 + (39/64) c^2],
//   12 beta_2 = 16 [(d - 11c/8)^2 + (39/64) c^2],
// so q_k = (3/4) beta_k + eps3 (eps3 = (3/4) eps keeps the weights) takes ten operations, the
// (39/64) c^2 term being shared by q_1 and q_2. The weights d_k/(eps+beta_k)^2 are multiplied
// through by 10 (4/3)^2 q_0^2 q_1^2 q_2^2: (w0, 6 v1, 3 v2). With the candidates
//   p_0 = f2 + (5b - 2a)/6,  p_1 = f2 + (b + 2c)/6,  p_2 = f2 + (4c - d)/6,
// the result is f2 - num/(3 den), num = w0 e0 + v1 e1 + v2 e2 with e0 = a - 5b/2 = -3 (p_0 - f2),
// e1 = -3b - 6c = -18 (p_1 - f2), e2 = 3d/2 - 6c = -9 (p_2 - f2), and den = w0 + 6 v1 + 3 v2.
__device__ __forceinline__ void weno5_nd(double f0, double f1, double f2, double f3, double f4,
                                         double eps3, double& num, double& den) {
  double a = f1 - f0, b = f2 - f1, c = f3 - f2, d = f4 - f3;
  double u0 = fma(-1.375, b, a), u1 = fma(-0.625, c, b), u2 = fma(-1.375, c, d);
  double kb = 0.609375 * b, kc = 0.609375 * c;
  double q0 = fma(u0, u0, fma(kb, b, eps3));
  double qc = fma(kc, c, eps3);
  double q1 = fma(u1, u1, qc), q2 = fma(u2, u2, qc);
  double Q0 = q0 * q0, Q1 = q1 * q1, Q2 = q2 * q2;
  double w0 = Q1 * Q2, v1 = Q0 * Q2, v2 = Q0 * Q1;
  double c6 = 6.0 * c;
  double e0 = fma(-2.5, b, a);
  double e1 = fma(-3.0, b, -c6);
  double e2 = fma(1.5, d, -c6);
  num = fma(v2, e2, fma(v1, e1, w0 * e0));
  den = fma(3.0, v2, fma(6.0, v1, w0));
}

// Characteristic Lax-Friedrichs flux-vector splitting with WENO5 (Section 2.1) at the face
// between nodes n and n+st: Roe average, local LF speeds (largest |eigenvalue| of each field over
// the six stencil nodes), projection of w and of the Euler flux at the stencil nodes onto the
// left eigenvectors (written out through the acoustic-row scalars A, B and the shear rows),
// WENO5 of the positive part from the left and of the negative part from the right, and
// projection back with the right eigenvectors.
//
// The split values of field k are carried scaled by s_k (4 for the acoustic fields, 2 for the
// others) to drop the 1/2 and 1/4 factors of the projection and of the splitting; WENO5 is then
// run with eps scaled by s_k^2, which leaves its weights unchanged, and the result is divided
// by s_k. The acoustic difference row is formed as c B (no division by c per node) and the 1/c
// enters the sums A +- B as an FMA.
//
// FP64 is the binding pipe on this path, so the maxima of the LF speeds |x| are taken on their
// IEEE bit patterns (with the sign bit cleared, monotone in |x|) on the integer pipe, as
// (high word, low word) pairs.
struct AbsMax {
  unsigned hi = 0u, lo = 0u;
  __device__ __forceinline__ void add(double x) {
    unsigned l, h;
    split64(x, l, h);
    h &= 0x7fffffffu;
    const bool gt = h > hi || (h == hi && l > lo);
    hi = gt ? h : hi;
    lo = gt ? l : lo;
  }
  __device__ __forceinline__ double value() const { return join64(lo, hi); }
};

// Reciprocals of five positive doubles with one division (prefix-product method): each value
// is first brought to [1, 2) by replacing its exponent field (integer operations on the high
// word), the five mantissas are inverted together, and each reciprocal gets its exponent back
// by an integer subtraction on its exponent field. That is valid for positive normal inputs
// below 2^1022 (biased exponent field 1 .. 2044: the reciprocals stay normal). Any other input
// (zero, subnormal, 2^1022 or more, infinity, NaN, negative) sends the five through plain
// correctly rounded divisions instead, so the result is 1/y in every case; the range test is
// integer work and the fallback is not taken for the states of the method.
__device__ __forceinline__ void recip5(const double* y, double* r) {
  double m[5];
  int e[5];
  bool in_range = true;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    unsigned lo, hi;
    split64(y[k], lo, hi);
    const unsigned field = hi >> 20;  // sign and biased exponent
    in_range = in_range && field >= 1u && field <= 2044u;
    e[k] = (int)(field & 0x7ffu) - 1023;
    m[k] = join64(lo, (hi & 0x000fffffu) | 0x3ff00000u);
  }
  if (!in_range) {
#pragma unroll
    for (int k = 0; k < 5; ++k) r[k] = 1.0 / y[k];
    return;
  }
  double p1 = m[0] * m[1], p2 = p1 * m[2], p3 = p2 * m[3], p4 = p3 * m[4];
  double inv = 1.0 / p4;
  double i4 = inv * p3;
  inv *= m[4];
  double i3 = inv * p2;
  inv *= m[3];
  double i2 = inv * p1;
  inv *= m[2];
  double i1 = inv * m[0], i0 = inv * m[1];
  const double im[5] = {i0, i1, i2, i3, i4};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    unsigned lo, hi;
    split64(im[k], lo, hi);
    r[k] = join64(lo, hi - ((unsigned)e[k] << 20));
  }
}

template <int DIR>
__device__ __forceinline__ void weno_flux(const Consts& C, const Bufs& B, long long n, long long st,
                                          double* f) {
  constexpr int T1 = DIR == 0 ? 1 : 0;
  constexpr int T2 = DIR == 2 ? 1 : 2;
  const Nodes<double>& P = B.n64;
  const double* STRM_RO vel[3] = {P.u, P.v, P.w};
  const double* STRM_RO un_p = vel[DIR];
  // Roe average of nodes n and n + st
  double sl = STRM_LDG(P.srho + n), sr = STRM_LDG(P.srho + n + st);
  double inv = 1.0 / (sl + sr);
  double wl = sl * inv, wr = sr * inv;
  double ua[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) ua[dd] = wl * STRM_LDG(vel[dd] + n) + wr * STRM_LDG(vel[dd] + n + st);
  double Ha = wl * STRM_LDG(P.H + n) + wr * STRM_LDG(P.H + n + st);
  double q2 = ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
  double c2a = C.gm1 * (Ha - 0.5 * q2);
  double ic = rsqrt(c2a);
  double ca = c2a * ic;
  double b1 = C.gm1 * ic * ic;
  double b2 = (0.5 * q2) * b1;
  double un_a = ua[DIR];

  // local Lax-Friedrichs speeds over the stencil nodes n-2 .. n+3
  AbsMax m0, m1, m4;
  const double* STRM_RO lm = B.lam[2 * DIR];      // u_n - c at the nodes
  const double* STRM_RO lp = B.lam[2 * DIR + 1];  // u_n + c
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    long long nn = n + (q - 2) * st;
    m0.add(STRM_LDG(lm + nn));
    m1.add(STRM_LDG(un_p + nn));
    m4.add(STRM_LDG(lp + nn));
  }
  const double lam0 = m0.value(), lam1 = m1.value(), lam4 = m4.value();

  // scaled split characteristic values s_k (L F +- lam_k L w)/2 at the stencil nodes
  double gp[5][6], gm[5][6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    long long nn = n + (q - 2) * st;
    double rho = STRM_LDG(P.rho + nn);
    double uu[3] = {STRM_LDG(P.u + nn), STRM_LDG(P.v + nn), STRM_LDG(P.w + nn)};
    double H = STRM_LDG(P.H + nn), p = STRM_LDG(P.p + nn);
    double run = STRM_LDG(B.mom[DIR] + nn);  // rho u_n, the conserved momentum
    double hu = fma(-ua[2], uu[2], fma(-ua[1], uu[1], fma(-ua[0], uu[0], H)));  // H - ua.u
    double K = fma(b1, hu, b2);
    double b1p = b1 * p;
    double Aw = fma(rho, K, -b1p);  // acoustic rows: (l0 + l4) w = A_w, c (l0 - l4) w = cB_w
    double Af = fma(run, K, -b1p * un_a);
    // c B rows: rho (ua_n - u_n) and rho u_n (ua_n - u_n) - p = rho u_n ua_n - (rho u_n^2 + p)
    double cBw = fma(rho, un_a, -run);
    double cBf = fma(run, un_a, -STRM_LDG(B.mflux[DIR] + nn));
    double Sw = fma(ic, cBw, Aw), Sf = fma(ic, cBf, Af), Dw = fma(-ic, cBw, Aw), Df = fma(-ic, cBf, Af);
    gp[0][q] = fma(lam0, Sw, Sf);
    gm[0][q] = fma(-lam0, Sw, Sf);
    gp[4][q] = fma(lam4, Dw, Df);
    gm[4][q] = fma(-lam4, Dw, Df);
    double r1 = fma(lam1, rho, run), r2 = fma(-lam1, rho, run);
    gp[1][q] = r1 - fma(lam1, Aw, Af);
    gm[1][q] = r2 - fma(-lam1, Aw, Af);
    double d1 = uu[T1] - ua[T1], d2 = uu[T2] - ua[T2];
    gp[2][q] = d1 * r1;
    gm[2][q] = d1 * r2;
    gp[3][q] = d2 * r1;
    gm[3][q] = d2 * r2;
  }
  // per field: the + and - reconstructions over one common denominator, the five
  // denominators inverted together
  double num[5], den[5], rden[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const bool acoustic = (k == 0 || k == 4);
    const double eps3 = (acoustic ? 12.0 : 3.0) * C.k64.weno_eps;  // (3/4) s_k^2 eps
    double np_, dp_, nm_, dm_;
    weno5_nd(gp[k][0], gp[k][1], gp[k][2], gp[k][3], gp[k][4], eps3, np_, dp_);
    weno5_nd(gm[k][5], gm[k][4], gm[k][3], gm[k][2], gm[k][1], eps3, nm_, dm_);
    num[k] = fma(np_, dm_, nm_ * dp_);
    den[k] = dp_ * dm_;
  }
  recip5(den, rden);
  double g[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const double s = (k == 0 || k == 4) ? 0.25 : 0.5;
    g[k] = fma(s * (-1.0 / 3.0), num[k] * rden[k], s * (gp[k][2] + gm[k][3]));
  }
  // back to conserved variables with the right eigenvectors
  double s04 = g[0] + g[4], cd40 = ca * (g[4] - g[0]);
  double gs = s04 + g[1];
  f[0] = gs;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) f[1 + dd] = gs * ua[dd];
  f[1 + DIR] += cd40;
  f[1 + T1] += g[2];
  f[1 + T2] += g[3];
  f[4] = Ha * s04 + un_a * cd40 + 0.5 * q2 * g[1] + ua[T1] * g[2] + ua[T2] * g[3];
}

// FP32 WENO5 (mixed precision), same first-difference form; the nonlinear weights are formed
// as 10 d_k/(eps+beta_k)^2 directly (products of (eps+beta)^2 could overflow FP32).
__device__ __forceinline__ float weno5_f(float f0, float f1, float f2, float f3, float f4, float eps4) {
  float a = f1 - f0, b = f2 - f1, c = f3 - f2, d = f4 - f3;
  float t0 = b - a, t1 = fmaf(3.f, b, -a);
  float t2 = c - b, t3 = b + c;
  float t4 = d - c, t5 = fmaf(-3.f, c, d);
  float q0 = eps4 + fmaf((13.f / 3.f) * t0, t0, t1 * t1);
  float q1 = eps4 + fmaf((13.f / 3.f) * t2, t2, t3 * t3);
  float q2 = eps4 + fmaf((13.f / 3.f) * t4, t4, t5 * t5);
  float w0 = 1.f / (q0 * q0), w1 = 6.f / (q1 * q1), w2 = 3.f / (q2 * q2);
  float e0 = fmaf(-2.f, a, 5.f * b), e1 = fmaf(2.f, c, b), e2 = fmaf(4.f, c, -d);
  return f2 + fmaf(w2, e2, fmaf(w1, e1, w0 * e0)) / (6.f * (w0 + w1 + w2));
}

// Mixed-precision characteristic WENO flux. The projection into characteristic variables is
// done in FP64: Roe state, eigen-scalars and, per stencil node, the acoustic-row scalars
// A and B of w and of the Euler flux (where cancellation happens). The LF split, WENO5 and the
// projection back to conserved variables run in FP32; the result is an FP32 face flux.
// The FP64 pipe bounds this kernel, so its FP64 -> FP32 roundings run on the integer pipe (d2f)
// and the Roe state's reciprocal and inverse sound speed come from FP32 estimates refined by a
// Newton step in FP64 (rcp_nr, rsqrt_nr; relative error below 2^-43).
template <int DIR>
__device__ __forceinline__ void weno_flux_mixed(const Consts& C, const Bufs& B, long long n, long long st,
                                                float* f) {
  constexpr int T1 = DIR == 0 ? 1 : 0;
  constexpr int T2 = DIR == 2 ? 1 : 2;
  const Nodes<double>& P = B.n64;
  const Nodes<float>& F = B.n32;
  const double* STRM_RO vel[3] = {P.u, P.v, P.w};
  const float* STRM_RO velf[3] = {F.u, F.v, F.w};
  // FP64 Roe average of nodes n and n + st and the eigen-scalars
  double sl = STRM_LDG(P.srho + n), sr = STRM_LDG(P.srho + n + st);
  double inv = rcp_nr(sl + sr);
  double wl = sl * inv, wr = sr * inv;
  double ua[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) ua[dd] = wl * STRM_LDG(vel[dd] + n) + wr * STRM_LDG(vel[dd] + n + st);
  double Ha = wl * STRM_LDG(P.H + n) + wr * STRM_LDG(P.H + n + st);
  double q2 = ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
  double c2a = C.gm1 * (Ha - 0.5 * q2);
  double ic = rsqrt_nr(c2a);
  double b1 = C.gm1 * ic * ic;
  double b2 = 0.5 * q2 * b1;
  double un_a = ua[DIR];
  const float uaf[3] = {d2f(ua[0]), d2f(ua[1]), d2f(ua[2])};
  // FP32 local LF speeds
  float lam0 = 0.f, lam1 = 0.f, lam4 = 0.f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    long long nn = n + (q - 2) * st;
    float un = STRM_LDG(velf[DIR] + nn), cs = STRM_LDG(F.c + nn);
    lam0 = fmaxf(lam0, fabsf(un - cs));
    lam1 = fmaxf(lam1, fabsf(un));
    lam4 = fmaxf(lam4, fabsf(un + cs));
  }
  float gp[5][6], gm[5][6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    long long nn = n + (q - 2) * st;
    double rho = STRM_LDG(P.rho + nn);
    double uu[3] = {STRM_LDG(P.u + nn), STRM_LDG(P.v + nn), STRM_LDG(P.w + nn)};
    double H = STRM_LDG(P.H + nn), p = STRM_LDG(P.p + nn);
    double run = STRM_LDG(B.mom[DIR] + nn);  // rho u_n, the conserved momentum
    double hu = fma(-ua[2], uu[2], fma(-ua[1], uu[1], fma(-ua[0], uu[0], H)));  // H - ua.u
    double K = fma(b1, hu, b2);
    double b1p = b1 * p;
    double Aw = fma(rho, K, -b1p);
    double Af = fma(run, K, -b1p * un_a);
    double cBw = fma(rho, un_a, -run), cBf = fma(run, un_a, -STRM_LDG(B.mflux[DIR] + nn));
    float Sw = d2f(fma(ic, cBw, Aw)), Sf = d2f(fma(ic, cBf, Af)), Dw = d2f(fma(-ic, cBw, Aw)),
          Df = d2f(fma(-ic, cBf, Af));
    float Awf = d2f(Aw), Aff = d2f(Af);
    float rhof = STRM_LDG(F.rho + nn), unf = STRM_LDG(velf[DIR] + nn);
    float runf = rhof * unf;
    gp[0][q] = fmaf(lam0, Sw, Sf);
    gm[0][q] = fmaf(-lam0, Sw, Sf);
    gp[4][q] = fmaf(lam4, Dw, Df);
    gm[4][q] = fmaf(-lam4, Dw, Df);
    float r1 = fmaf(lam1, rhof, runf), r2 = fmaf(-lam1, rhof, runf);
    gp[1][q] = r1 - fmaf(lam1, Awf, Aff);
    gm[1][q] = r2 - fmaf(-lam1, Awf, Aff);
    float d1 = STRM_LDG(velf[T1] + nn) - uaf[T1], d2 = STRM_LDG(velf[T2] + nn) - uaf[T2];
    gp[2][q] = d1 * r1;
    gm[2][q] = d1 * r2;
    gp[3][q] = d2 * r1;
    gm[3][q] = d2 * r2;
  }
  const float eps = C.k32.weno_eps;
  float g[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const bool acoustic = (k == 0 || k == 4);
    const float eps4 = (acoustic ? 64.f : 16.f) * eps;  // 4 s_k^2 eps
    float v = weno5_f(gp[k][0], gp[k][1], gp[k][2], gp[k][3], gp[k][4], eps4) +
              weno5_f(gm[k][5], gm[k][4], gm[k][3], gm[k][2], gm[k][1], eps4);
    g[k] = (acoustic ? 0.25f : 0.5f) * v;
  }
  const float icf = d2f(ic), c2f = d2f(c2a);
  const float caf = c2f * icf, Haf = d2f(Ha), q2f = d2f(q2), unaf = uaf[DIR];
  float gs = g[0] + g[1] + g[4];
  f[0] = gs;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) f[1 + dd] = gs * uaf[dd];
  f[1 + DIR] += caf * (g[4] - g[0]);
  f[1 + T1] += g[2];
  f[1 + T2] += g[3];
  f[4] = Haf * (g[0] + g[4]) + unaf * caf * (g[4] - g[0]) + 0.5f * q2f * g[1] + uaf[T1] * g[2] +
         uaf[T2] * g[3];
  // the central faces carry the pressure less p_shift (their FP32 pressure copy is shifted);
  // the same constant comes off here, so that every face flux has the same offset, which
  // cancels in the flux differences
  f[1 + DIR] -= (float)C.p_shift;
}

// ------------------------------------------------------------------------------ face kernels

// Block-aggregated append of face q to one of two compacted lists (a when to_a, else b): per-warp
// counts by ballot, one atomic per list and block, in-block offsets from a prefix over the
// warps. Every thread of the block calls it (valid = false for threads past the end).
__device__ __forceinline__ void block_append2(bool valid, bool to_a, int q, int* list_a, unsigned* count_a,
                                              int* list_b, unsigned* count_b) {
  __shared__ unsigned s_a[32], s_b[32], s_base[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  unsigned ma = __ballot_sync(0xffffffffu, valid && to_a);
  unsigned mb = __ballot_sync(0xffffffffu, valid && !to_a);
  if (lane == 0) {
    s_a[warp] = __popc(ma);
    s_b[warp] = __popc(mb);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ta = 0, tb = 0;
    for (int w = 0; w < nwarp; ++w) {  // exclusive prefix over the warps
      unsigned a = s_a[w], b = s_b[w];
      s_a[w] = ta;
      s_b[w] = tb;
      ta += a;
      tb += b;
    }
    s_base[0] = ta ? atomicAdd(count_a, ta) : 0u;
    s_base[1] = tb ? atomicAdd(count_b, tb) : 0u;
  }
  __syncthreads();
  if (valid) {
    unsigned below = (1u << lane) - 1u;
    if (to_a) list_a[s_base[0] + s_a[warp] + __popc(ma & below)] = q;
    else list_b[s_base[1] + s_b[warp] + __popc(mb & below)] = q;
  }
}

// Hybrid switch, sensor mode: split the faces of one direction into a WENO list and a central
// list, so that each flux kernel runs without warp divergence whatever the flagged fraction.
template <int L, int DIR, typename R>
__device__ __forceinline__ void body_classify(const Dims& d, const Consts& C, const Bufs& B, int blk) {
  long long q = (long long)blk * blockDim.x + threadIdx.x;
  bool valid = q < d.nf[DIR], fl = false;
  if (DIR == 2 && valid) q = zface_order(d, q);
  if (valid) {
    int i, j, k;
    face_node<DIR>(d, q, i, j, k);
    if (stencil_ok(d, i, j, k, DIR, L - 1, L, kDbgFace)) fl = face_decision<L, R>(d, C, B, i, j, k, DIR);
  }
  block_append2(valid, fl, (int)q, B.wl[DIR], B.wcount + DIR, B.cl[DIR], B.wcount + 4 + DIR);
}

// Central flux at every face of one direction (WENO off) or at the faces of the central list.
template <int L, int DIR, typename R>
__device__ __forceinline__ void body_central(const Dims& d, const Consts& C, const Bufs& B, int use_list,
                                             long long t0, long long tstride) {
  long long cnt = use_list ? (long long)B.wcount[4 + DIR] : d.nf[DIR];
  long long nf = d.nf[DIR];
  long long st = dir_stride(d, DIR);
  R* out = face_flux<R>(B, DIR);
  for (long long t = t0; t < cnt; t += tstride) {
    long long q = use_list ? (long long)B.cl[DIR][t] : (DIR == 2 ? zface_order(d, t) : t);
    if (!index_ok(d, q, nf, kDbgList)) continue;
    int i, j, k;
    face_node<DIR>(d, q, i, j, k);
    if (!stencil_ok(d, i, j, k, DIR, L - 1, L, kDbgFace)) continue;
    R f[5];
    if constexpr (DIR == 0 && sizeof(R) == sizeof(float)) central_flux_xdev<L>(d, C, B, gidx(d, i, j, k), j, k, f);
    else central_flux<L, DIR, R>(C, B, gidx(d, i, j, k), st, f);
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * nf + q] = f[c];
  }
}

// Central flux at every face of direction DIR = 1 (y) or 2 (z) by sweeps along DIR that reuse
// the split flux's pair terms. The flux at face s (between nodes s-1 and s) is the sum over
// l = 1..L of the L pairs (a, a + l), s - l <= a <= s - 1 (Eq. encflux), each pair contributing
// q (1, phi_a + phi_b) with q = (a_l/4)(rho_a + rho_b)(u_a + u_b) along DIR. Pair (a, a + l)
// serves the l faces it spans, so a thread that walks consecutive faces computes at each face
// only the L pairs starting at node s - 1 and keeps the others in registers, and loads one new
// node per face instead of 2L (the same products, summed in another order than body_central;
// the pressure part is as in central_flux). Thread t takes segment seg of the column (i, c):
// i = t mod nx, then c (z for y sweeps, y for z sweeps), then seg, so a warp walks 32
// consecutive x and reads coalesced rows; each segment first computes the L - 1 pair
// generations before its first face. Faces past the last one of the column are not computed.
template <int L, int DIR, typename R>
__device__ __forceinline__ void body_central_sweep(const Dims& d, const Consts& C, const Bufs& B, long long t) {
  static_assert(DIR == 1 || DIR == 2, "sweeps run along y or z");
  constexpr int SEG = kSweepSeg;
  const int ncol = DIR == 1 ? d.nz : d.ny;   // columns per x
  const int nfa = (DIR == 1 ? d.ny : d.nz) + 1;  // faces along the sweep
  const long long nseg = (nfa + SEG - 1) / SEG;
  if (t >= (long long)d.nx * ncol * nseg) return;
  const int i = (int)(t % d.nx);
  const long long r = t / d.nx;
  const int c = (int)(r % ncol);
  const int s0 = (int)(r / ncol) * SEG;
  const int s1 = min(s0 + SEG, nfa);  // faces s0 .. s1 - 1
  // nodes read: s0 - L .. s1 - 2 + L along DIR (ghosts included)
  {
    const int jj = DIR == 1 ? s0 - L : c, kk = DIR == 1 ? c : s0 - L;
    if (!stencil_ok(d, i, jj, kk, DIR, 0, s1 - s0 + 2 * L - 2, kDbgFace)) return;
  }
  const Nodes<R>& P = nodes<R>(B);
  const Coefs<R>& K = coefs<R>(C);
  const R* STRM_RO ud = DIR == 1 ? P.v : P.w;
  const long long st = dir_stride(d, DIR);
  // node (i, j, k) with the sweep coordinate at -0; n(s) = base + s * st
  const long long base = DIR == 1 ? gidx(d, i, 0, c) : gidx(d, i, c, 0);
  const long long nf = d.nf[DIR];
  R* out = face_flux<R>(B, DIR);
  // node window: nodes s-1 .. s-1+L at face s (rho, u_d, u, v, w, H) and the pressure at
  // nodes s-L .. s+L-1
  R wr[L + 1], wu[L + 1], wv[L + 1], ww[L + 1], wh[L + 1], pw[2 * L];
  const int sb = s0 - L + 1;  // first (warm-up) face of the walk
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    const long long n = base + (long long)(sb - 1 + m) * st;
    wr[m] = STRM_LDG(P.rho + n);
    wu[m] = STRM_LDG(P.u + n);
    wv[m] = STRM_LDG(P.v + n);
    ww[m] = STRM_LDG(P.w + n);
    wh[m] = STRM_LDG(P.H + n);
  }
#pragma unroll
  for (int m = 0; m < 2 * L; ++m) {
    const int sn = sb - L + m;  // node index along the sweep; below -G it is never used
    pw[m] = sn >= -G ? STRM_LDG(P.p + base + (long long)sn * st) : R(0);
  }
  // pair history: hq[l][g] (and hu, hv, hw, hh) holds the terms of the pair of length l that
  // starts at node s-2-g (g = 0 .. l-2: the l-1 generations before this face); filled by the
  // warm-up faces before the first face written
  R hq[L + 1][L], hu[L + 1][L], hv[L + 1][L], hw[L + 1][L], hh[L + 1][L];
#pragma unroll
  for (int l = 0; l <= L; ++l)
#pragma unroll
    for (int g = 0; g < L; ++g) hq[l][g] = hu[l][g] = hv[l][g] = hw[l][g] = hh[l][g] = R(0);
  for (int s = sb; s < s1; ++s) {
    // new pairs (s-1, s-1+l), l = 1..L
    R nq[L + 1], nu[L + 1], nv[L + 1], nw[L + 1], nh[L + 1];
#pragma unroll
    for (int l = 1; l <= L; ++l) {
      const R rs = wr[0] + wr[l];
      const R us = wu[0] + wu[l], vs = wv[0] + wv[l], ws = ww[0] + ww[l], hs = wh[0] + wh[l];
      const R uds = DIR == 1 ? vs : ws;
      const R q = (K.aq[l] * rs) * uds;
      nq[l] = q;
      nu[l] = q * us;
      nv[l] = q * vs;
      nw[l] = q * ws;
      nh[l] = q * hs;
    }
    if (s >= s0) {
      // face s: the new pairs of every length and the l-1 previous generations of length l
      R a0 = R(0), a1 = R(0), a2 = R(0), a3 = R(0), a4 = R(0);
#pragma unroll
      for (int l = 1; l <= L; ++l) {
        a0 += nq[l];
        a1 += nu[l];
        a2 += nv[l];
        a3 += nw[l];
        a4 += nh[l];
#pragma unroll
        for (int g = 0; g < l - 1; ++g) {
          a0 += hq[l][g];
          a1 += hu[l][g];
          a2 += hv[l][g];
          a3 += hw[l][g];
          a4 += hh[l][g];
        }
      }
      R ap = R(0);
#pragma unroll
      for (int m = 0; m < L; ++m) ap = fma(K.ap[m], pw[L - 1 - m] + pw[L + m], ap);
      const long long q = DIR == 1 ? ((long long)c * (d.ny + 1) + s) * d.nx + i
                                   : ((long long)s * d.ny + c) * d.nx + i;
      out[q] = R(2) * a0;
      out[nf + q] = a1;
      out[2 * nf + q] = DIR == 1 ? a2 + ap : a2;
      out[3 * nf + q] = DIR == 2 ? a3 + ap : a3;
      out[4 * nf + q] = a4;
    }
    // shift the pair history (generation 0 is the most recent) and the windows
#pragma unroll
    for (int l = 2; l <= L; ++l) {
#pragma unroll
      for (int g = l - 2; g > 0; --g) {
        hq[l][g] = hq[l][g - 1];
        hu[l][g] = hu[l][g - 1];
        hv[l][g] = hv[l][g - 1];
        hw[l][g] = hw[l][g - 1];
        hh[l][g] = hh[l][g - 1];
      }
      hq[l][0] = nq[l];
      hu[l][0] = nu[l];
      hv[l][0] = nv[l];
      hw[l][0] = nw[l];
      hh[l][0] = nh[l];
    }
    if (s + 1 < s1) {
#pragma unroll
      for (int m = 0; m < L; ++m) {
        wr[m] = wr[m + 1];
        wu[m] = wu[m + 1];
        wv[m] = wv[m + 1];
        ww[m] = ww[m + 1];
        wh[m] = wh[m + 1];
      }
#pragma unroll
      for (int m = 0; m < 2 * L - 1; ++m) pw[m] = pw[m + 1];
      const long long n = base + (long long)(s + L) * st;  // node s + L: window of face s + 1
      wr[L] = STRM_LDG(P.rho + n);
      wu[L] = STRM_LDG(P.u + n);
      wv[L] = STRM_LDG(P.v + n);
      ww[L] = STRM_LDG(P.w + n);
      wh[L] = STRM_LDG(P.H + n);
      pw[2 * L - 1] = STRM_LDG(P.p + base + (long long)(s + L) * st);
    }
  }
}

// Characteristic WENO flux at the faces of the WENO list (sensor mode) or at every face (WENO
// everywhere); FP64, or the mixed-precision variant writing FP32 face fluxes.
template <int DIR, bool MIXED>
__device__ __forceinline__ void body_weno(const Dims& d, const Consts& C, const Bufs& B, long long t0,
                                          long long tstride) {
  const bool all = C.weno_mode == 2;
  long long nf = d.nf[DIR];
  long long cnt = all ? nf : (long long)B.wcount[DIR];
  long long st = dir_stride(d, DIR);
  for (long long t = t0; t < cnt; t += tstride) {
    long long q = all ? (DIR == 2 ? zface_order(d, t) : t) : (long long)B.wl[DIR][t];
    if (!index_ok(d, q, nf, kDbgList)) continue;
    int i, j, k;
    face_node<DIR>(d, q, i, j, k);
    if (!stencil_ok(d, i, j, k, DIR, 2, 3, kDbgFace)) continue;
    if (MIXED) {
      float f[5];
      weno_flux_mixed<DIR>(C, B, gidx(d, i, j, k), st, f);
      if (DIR == 0) {  // the x row's offset of the deviation-form central faces
        float c5[5];
        xrow_flux_const(d, C, B, j, k, c5);
#pragma unroll
        for (int c = 0; c < 5; ++c) f[c] -= c5[c];
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) B.fh32[DIR][c * nf + q] = f[c];
    } else {
      double f[5];
      weno_flux<DIR>(C, B, gidx(d, i, j, k), st, f);
#pragma unroll
      for (int c = 0; c < 5; ++c) B.fh64[DIR][c * nf + q] = f[c];
    }
  }
}

// ------------------------------------------------------------------------------ assembly

// The viscous terms from the derivatives at one node (Section 2.1 and Eqs. sigma, heat_vec):
// du[a][b] = d_b u_a, lap[a] = lap u_a, dT, lapT, dmu = grad mu, ddiv = grad(div u), the node's
// mu and velocity; V = (0, V_1, V_2, V_3, V_E).
template <typename R>
__device__ __forceinline__ void viscous_combine(const Coefs<R>& K, const R (&du)[3][3], const R (&lap)[3],
                                                const R (&dT)[3], R lapT, const R (&dmu)[3],
                                                const R (&ddiv)[3], R mu, const R (&uu)[3], R* V) {
  const R div = du[0][0] + du[1][1] + du[2][2];
  const R tdiv = R(2.0 / 3.0) * div;
  // symmetric strain sums S_ab = d_b u_a + d_a u_b
  const R S00 = R(2) * du[0][0], S11 = R(2) * du[1][1], S22 = R(2) * du[2][2];
  const R S01 = du[0][1] + du[1][0], S02 = du[0][2] + du[2][0], S12 = du[1][2] + du[2][1];
  R sm[3];
  sm[0] = fma(dmu[0], S00, fma(dmu[1], S01, dmu[2] * S02));
  sm[1] = fma(dmu[0], S01, fma(dmu[1], S11, dmu[2] * S12));
  sm[2] = fma(dmu[0], S02, fma(dmu[1], S12, dmu[2] * S22));
  R Vm[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) Vm[a] = fma(mu, fma(ddiv[a], R(1.0 / 3.0), lap[a]), fma(-tdiv, dmu[a], sm[a]));
  R work = fma(uu[0], Vm[0], fma(uu[1], Vm[1], uu[2] * Vm[2]));
  // sigma_ij d_j u_i = mu [ sum_ab S_ab d_b u_a - 2/3 div^2 ], and by symmetry
  // sum_ab S_ab d_b u_a = sum_a S_aa d_a u_a + sum_{a<b} S_ab^2
  R diss = fma(S00, du[0][0], fma(S11, du[1][1], fma(S22, du[2][2], fma(S01, S01, fma(S02, S02, S12 * S12)))));
  diss = mu * fma(-tdiv, div, diss);
  R heat = K.cp_pr * (mu * lapT + dmu[0] * dT[0] + dmu[1] * dT[1] + dmu[2] * dT[2]);
  V[0] = R(0);
  V[1] = Vm[0];
  V[2] = Vm[1];
  V[3] = Vm[2];
  V[4] = work + diss + heat;
}

// Viscous terms in Laplacian form at node n (Section 2.1 and Eqs. sigma, heat_vec):
//   V_i = mu lap u_i + mu/3 d_i(div) + d_j mu (d_j u_i + d_i u_j) - 2/3 div d_i mu,
//   V_E = u_i V_i + sigma_ij d_j u_i + k lap T + d_j k d_j T,  k = cp mu / Pr,
// first and second derivatives of order 2L; along y, d/dy = (1/y_eta) d/deta and
// d2/dy2 = (f_etaeta - (y_etaeta/y_eta) f_eta)/y_eta^2; d_i(div) from the ghost-filled div.
template <int L, typename R>
__device__ __forceinline__ void viscous_node(const Consts& C, const Bufs& B, const Dims& d, long long n,
                                             long long q, int j, R* V) {
  const Nodes<R>& P = nodes<R>(B);
  const Coefs<R>& K = coefs<R>(C);
  const Metric<R>& M = metric<R>(B);
  const long long sy = d.px, sz = d.plane;
  const R hy = STRM_LDG(M.inv_hy + j), c2 = STRM_LDG(M.c2y + j), c1 = STRM_LDG(M.c1y + j);
  const R* STRM_RO fld[4] = {P.u, P.v, P.w, P.T};
  R du[3][3], lap[3], dT[3], lapT = R(0);
  if constexpr (std::is_same<R, double>::value) {
    // FP64: first derivatives of the velocity from the sensor; second derivatives here, with
    // the eta-derivative of the stretched-y term taken back from d_y u (f_eta / y_eta^2 term
    // = (y_etaeta / y_eta^2) d_y u)
    const double c1h = STRM_LDG(B.c1h + j);
    const double cc = fma(K.b[0], c2, K.bxz0);  // centre weight of the three second differences
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) du[a][b] = STRM_LDG(B.grad + (3 * a + b) * d.N + q);
      lap[a] = fma(-du[a][1], c1h, lap_c<L>(fld[a], n, sy, sz, K, cc, c2));
    }
    double g3[3];
    const double l3 = lap_c<L>(fld[3], n, sy, sz, K, cc, c2, g3);
    dT[0] = g3[0];
    dT[1] = g3[1] * hy;
    dT[2] = g3[2];
    lapT = fma(-g3[1], c1, l3);
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      R s1, s2, d0, d1v, d2v, l0;
      dsum12<L>(fld[a], n, 1, K.ax, K.b, s1, s2);
      d0 = s1;
      l0 = s2 * K.inv_dx2;
      dsum12<L>(fld[a], n, sy, K.a, K.b, s1, s2);
      d1v = s1 * hy;
      l0 += s2 * c2 - s1 * c1;
      dsum12<L>(fld[a], n, sz, K.az, K.b, s1, s2);
      d2v = s1;
      l0 += s2 * K.inv_dz2;
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
  }
  R dmu[3], ddiv[3];
  dmu[0] = dsum<L>(P.mu, n, 1, K.ax);
  dmu[1] = dsum<L>(P.mu, n, sy, K.a) * hy;
  dmu[2] = dsum<L>(P.mu, n, sz, K.az);
  ddiv[0] = dsum<L>(P.div, n, 1, K.ax);
  ddiv[1] = dsum<L>(P.div, n, sy, K.a) * hy;
  ddiv[2] = dsum<L>(P.div, n, sz, K.az);
  const R uu[3] = {STRM_LDG(P.u + n), STRM_LDG(P.v + n), STRM_LDG(P.w + n)};
  viscous_combine<R>(K, du, lap, dT, lapT, dmu, ddiv, STRM_LDG(P.mu + n), uu, V);
}

// Convective part of the residual at node (i, j, k): R_m = -sum_d (f_{s+1} - f_s)/h_d (Eq.
// num_flux) with the staggered-wall rule; in mixed precision also the FP64 mass difference.
template <typename R>
__device__ __forceinline__ void convective_residual(const Dims& d, const Consts& C, const Bufs& B, int i, int j,
                                                    int k, R* res, double& mass64) {
  const Coefs<R>& K = coefs<R>(C);
  long long qx = ((long long)k * d.ny + j) * (d.nx + 1) + i;
  long long qy = ((long long)k * (d.ny + 1) + j) * d.nx + i;
  long long qz = ((long long)k * d.ny + j) * d.nx + i;
  long long sxy = (long long)d.nx * d.ny;
  R hy = STRM_LDG(metric<R>(B).inv_hy + j);
  bool wlo = C.bc[2] == kBcWall && j == 0, whi = C.bc[3] == kBcWall && j == d.ny - 1;
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const R* fx = face_flux<R>(B, 0) + m * d.nf[0];
    const R* fy = face_flux<R>(B, 1) + m * d.nf[1];
    const R* fz = face_flux<R>(B, 2) + m * d.nf[2];
    R ylo = STRM_LDG(fy + qy), yhi = STRM_LDG(fy + qy + d.nx);
    // staggered wall interface: no mass, x/z momentum or energy crosses it
    if (m != 2) {
      if (wlo) ylo = R(0);
      if (whi) yhi = R(0);
    }
    res[m] = -((STRM_LDG(fx + qx + 1) - STRM_LDG(fx + qx)) * K.inv_dx + (yhi - ylo) * hy +
               (STRM_LDG(fz + qz + sxy) - STRM_LDG(fz + qz)) * K.inv_dz);
    if (m == 0 && sizeof(R) != sizeof(double)) {
      // mixed precision: the mass difference is formed in FP64 from the FP32 face fluxes
      // (the difference of two FP32 values is exact in FP64), so that mass telescopes to
      // FP64 round-off as in the FP64 path
      mass64 = -((to_f64(STRM_LDG(fx + qx + 1)) - to_f64(STRM_LDG(fx + qx))) * C.k64.inv_dx +
                 (to_f64(yhi) - to_f64(ylo)) * STRM_LDG(B.m64.inv_hy + j) +
                 (to_f64(STRM_LDG(fz + qz + sxy)) - to_f64(STRM_LDG(fz + qz))) * C.k64.inv_dz);
    }
  }
}

// The residual of node q: with rk.w, the RK stage update of this node (body_rk_update without
// the forcing terms; the residual stays in registers instead of a round trip through memory),
// else stored to Rout. FP64 in both precisions; mixed precision takes the FP64 mass difference.
template <typename R>
__device__ __forceinline__ void stage_or_store(const Dims& d, const Bufs& B, long long q, const R* res,
                                               double mass64, double* STRM_RO Rout, const RkFuse& rk) {
  if (rk.w) {
    const double ad = B.scal[kScalAdt + rk.stage], bd = B.scal[kScalBdt + rk.stage];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const long long e = m * d.N + q;
      const double rr = (m == 0 && sizeof(R) != sizeof(double)) ? mass64 : to_f64(res[m]);
      double wn = rk.w[e] + bd * rr;
      if (rk.stage != 0) wn += ad * rk.r_old[e];  // alpha_0 = 0
      rk.w[e] = wn;
      rk.r_old[e] = rr;
    }
  } else {
#pragma unroll
    for (int m = 0; m < 5; ++m) Rout[m * d.N + q] = to_f64(res[m]);
    if (sizeof(R) != sizeof(double)) Rout[q] = mass64;
  }
}

// Residual per node: R = -sum_d (f_{s+1} - f_s)/h_d (Eq. num_flux, with the staggered-wall rule)
// plus the viscous terms, in precision R; stored in FP64 with the forcing partial sums.
template <int L, typename R>
__device__ __forceinline__ void body_assemble(const Dims& d, const Consts& C, const Bufs& B,
                                              double* STRM_RO Rout, int blk, double* sh,
                                              const RkFuse& rk = RkFuse{nullptr, nullptr, 0}) {
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  double fpart = 0.0;
  bool live = t < d.N;
  const long long q = live ? node_order(d, t) : t;
  if constexpr (kDebug) {  // stencils of the viscous terms and the faces read (debug builds)
    if (live) {
      int i = (int)(q % d.nx), j = (int)((q / d.nx) % d.ny), k = (int)(q / ((long long)d.nx * d.ny));
      long long qx = ((long long)k * d.ny + j) * (d.nx + 1) + i;
      long long qy = ((long long)k * (d.ny + 1) + j) * d.nx + i;
      long long qz = ((long long)k * d.ny + j) * d.nx + i;
      live = stencil_ok(d, i, j, k, 0, L, L, kDbgNode) && stencil_ok(d, i, j, k, 1, L, L, kDbgNode) &&
             stencil_ok(d, i, j, k, 2, L, L, kDbgNode) && index_ok(d, qx + 1, d.nf[0], kDbgFace) &&
             index_ok(d, qy + d.nx, d.nf[1], kDbgFace) &&
             index_ok(d, qz + (long long)d.nx * d.ny, d.nf[2], kDbgFace);
    }
  }
  if (live) {
    int i = (int)(q % d.nx);
    long long r = q / d.nx;
    int j = (int)(r % d.ny);
    int k = (int)(r / d.ny);
    R res[5] = {R(0), R(0), R(0), R(0), R(0)};
    double mass64 = 0.0;
    if (C.convective) convective_residual<R>(d, C, B, i, j, k, res, mass64);
    if (C.viscous) {
      R V[5];
      viscous_node<L, R>(C, B, d, gidx(d, i, j, k), q, j, V);
#pragma unroll
      for (int m = 1; m < 5; ++m) res[m] += V[m];
    }
    stage_or_store<R>(d, B, q, res, mass64, Rout, rk);
    if (C.forcing) fpart = to_f64(res[1]) * STRM_LDG(B.vol + j);
  }
  if (C.forcing) {
    double s = block_sum(fpart, sh);
    if (threadIdx.x == 0) B.red[blk] = s;
  }
}

}  // namespace strm
