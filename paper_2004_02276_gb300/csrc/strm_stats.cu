// Statistics accumulator (Section 3: Reynolds averages over the homogeneous directions and in
// time, Favre averages as ratios of mass-weighted Reynolds averages). One sample of a state adds
// to FP64 sums the means, over z or over x and z, of 24 point-wise quantities:
//   rho, u, v, w, p, T, rho u, rho v, rho w, rho T, rho uu, rho vv, rho ww, rho uv, rho uw,
//   rho vw, uu, vv, ww, uv, p^2, T^2, rho^2, mu.
// A thread owns one (i, j) column and walks z in order (coalesced along x); the x-z mode then
// reduces each wall-normal row over x in one block (fixed order), so the sums do not depend
// on the launch.
#include "strm_launch.h"

namespace strm {

namespace {

constexpr int kNStat = 24;

__global__ void __launch_bounds__(128) k_stats_columns(Dims d, Consts C, const double* __restrict__ w,
                                                       double* __restrict__ out, int mode) {
  long long ncol = (long long)d.nx * d.ny;
  long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  double s[kNStat];
#pragma unroll
  for (int q = 0; q < kNStat; ++q) s[q] = 0.0;
  for (int k = 0; k < d.nz; ++k) {
    long long n = (long long)k * ncol + col;
    double rho = w[n];
    double u = w[d.N + n] / rho, v = w[2 * d.N + n] / rho, ww = w[3 * d.N + n] / rho;
    double T = (w[4 * d.N + n] / rho - 0.5 * (u * u + v * v + ww * ww)) * C.inv_cv;
    double p = rho * C.r_gas * T;
    const double val[kNStat] = {rho,          u,           v,           ww,          p,
                                T,            rho * u,     rho * v,     rho * ww,    rho * T,
                                rho * u * u,  rho * v * v, rho * ww * ww, rho * u * v, rho * u * ww,
                                rho * v * ww, u * u,       v * v,       ww * ww,     u * v,
                                p * p,        T * T,       rho * rho,   viscosity(C.k64, C.visc_law, T)};
#pragma unroll
    for (int q = 0; q < kNStat; ++q) s[q] += val[q];
  }
  if (mode == 1) {  // z means, accumulated per (i, j)
    double inz = 1.0 / d.nz;
#pragma unroll
    for (int q = 0; q < kNStat; ++q) out[q * ncol + col] += s[q] * inz;
  } else {  // z sums, reduced over x by k_stats_rows
#pragma unroll
    for (int q = 0; q < kNStat; ++q) out[q * ncol + col] = s[q];
  }
}

__global__ void __launch_bounds__(256) k_stats_rows(Dims d, const double* __restrict__ scr,
                                                    double* __restrict__ acc) {
  __shared__ double sh[32];
  int j = blockIdx.x;
  double inv = 1.0 / ((double)d.nx * d.nz);
  for (int q = 0; q < kNStat; ++q) {
    const double* row = scr + ((long long)q * d.ny + j) * d.nx;
    double v = 0.0;
    for (int i = threadIdx.x; i < d.nx; i += blockDim.x) v += row[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) acc[(long long)q * d.ny + j] += v * inv;
    __syncthreads();  // sh is reused by the next quantity
  }
}

}  // namespace

void launch_stats(const Dims& d, const Consts& C, const double* w, double* acc, double* scr, int mode,
                  cudaStream_t s) {
  long long ncol = (long long)d.nx * d.ny;
  unsigned nb = (unsigned)((ncol + 127) / 128);
  if (mode == 1) {
    k_stats_columns<<<nb, 128, 0, s>>>(d, C, w, acc, 1);
  } else {
    k_stats_columns<<<nb, 128, 0, s>>>(d, C, w, scr, 0);
    k_stats_rows<<<d.ny, 256, 0, s>>>(d, scr, acc);
  }
}

}  // namespace strm
