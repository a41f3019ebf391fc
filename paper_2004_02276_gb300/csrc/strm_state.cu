// Node-wise kernels of one grid: primitives (+ CFL partial maxima), ghost fills of the
// primitives and of the sensor fields, the Ducros sensor, RK stage update, forcing, totals and
// flag export. The bodies are in strm_body.cuh.
#include <algorithm>

#include "strm_body.cuh"
#include "strm_launch.h"

namespace strm {

__global__ void __launch_bounds__(256) k_prims(Dims d, Consts C, Bufs B, const double* __restrict__ w,
                                               int want_cfl) {
  __shared__ double sh[32];
  body_prims(d, C, B, w, want_cfl, blockIdx.x, sh);
}

__global__ void __launch_bounds__(256) k_prims_mixed(Dims d, Consts C, Bufs B, const double* __restrict__ w,
                                                     int want_cfl) {
  __shared__ double sh[32];
  body_prims_mixed(d, C, B, w, want_cfl, blockIdx.x, sh);
}

__global__ void k_dt_finalize(Bufs B, int nparts, double cfl, double dt_fixed) {
  __shared__ double sh[32];
  body_dt_finalize(B, nparts, cfl, dt_fixed, sh);
}

__global__ void __launch_bounds__(256) k_ghost_prims(Dims d, Consts C, Bufs B, long long nthreads) {
  body_ghost_prims(d, C, B, nthreads, blockIdx.x);
}

__global__ void k_recycle_mean(Dims d, Consts C, Bufs B) {
  __shared__ double sh[32];
  body_recycle_mean(d, C, B, blockIdx.x, sh);
}

__global__ void k_recycle_scale(Dims d, Consts C, Bufs B) { body_recycle_scale(d, C, B); }

template <typename R>
__global__ void __launch_bounds__(256) k_ghost_scalars(Dims d, Consts C, Bufs B, long long nthreads) {
  body_ghost_scalars<R>(d, C, B, nthreads, blockIdx.x);
}

template <int L>
__global__ void __launch_bounds__(128) k_band_theta(Dims d, Consts C, Bufs B) {
  body_band_theta<L>(d, C, B, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                     (long long)gridDim.x * blockDim.x);
}

template <int L, typename R>
__global__ void __launch_bounds__(256) k_sensor(Dims d, Consts C, Bufs B, int region) {
  body_sensor<L, R>(d, C, B, blockIdx.x, region);
}

__global__ void k_force_finalize(Bufs B, int nparts, double inv_vtot) {
  __shared__ double sh[32];
  body_force_finalize(B, nparts, inv_vtot, sh);
}

__global__ void __launch_bounds__(256) k_rk_update(Dims d, Consts C, Bufs B, double* __restrict__ w,
                                                   double* __restrict__ r_old, int stage) {
  body_rk_update(d, C, B, w, r_old, stage, blockIdx.x);
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

// Prescribed switch input (strm_set_theta): the FP64 sensor field the hybrid switch reads takes
// the caller's values at the interior nodes (after the sensor, before its ghost fill).
__global__ void __launch_bounds__(256) k_theta_set(Dims d, Bufs B, const double* __restrict__ theta) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  int i, j, k;
  node_ijk(d, q, i, j, k);
  B.n64.theta[gidx(d, i, j, k)] = theta[q];
}

// elementwise FP64 <-> FP32 with the integer-pipe conversions of the mixed-precision kernels
__global__ void __launch_bounds__(256) k_convert_d2f(const double* __restrict__ x, float* __restrict__ y,
                                                     long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = d2f(x[q]);
}

__global__ void __launch_bounds__(256) k_convert_f2d(const float* __restrict__ x, double* __restrict__ y,
                                                     long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = f2d(x[q]);
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
  k_ghost_prims<<<blocks_for(n, 256), 256, 0, s>>>(d, C, B, n);
}

void launch_recycle(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  k_recycle_mean<<<d.ny, 256, 0, s>>>(d, C, B);
  k_recycle_scale<<<1, 1, 0, s>>>(d, C, B);
}

void launch_band_theta(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s) {
  unsigned nb = (unsigned)std::min<long long>(blocks_for(d.N, 128), 1216);
  if (C.L == 3) k_band_theta<3><<<nb, 128, 0, s>>>(d, C, B);
  else k_band_theta<2><<<nb, 128, 0, s>>>(d, C, B);
}

long long sensor_inner_nodes(const Dims& d, int L) {
  const long long bx = d.nx - 2 * L, by = d.ny - 2 * L, bz = d.nz - 2 * L;
  return (bx > 0 && by > 0 && bz > 0) ? bx * by * bz : 0;
}

void launch_sensor(const Dims& d, const Consts& C, const Bufs& B, int region, cudaStream_t s) {
  const long long inner = sensor_inner_nodes(d, C.L);
  const long long n = region == 0 ? d.N : (region == 1 ? inner : d.N - inner);
  if (n <= 0) return;
  unsigned nb = blocks_for(n, 256);
  if (C.mixed) {
    if (C.L == 3) k_sensor<3, float><<<nb, 256, 0, s>>>(d, C, B, region);
    else k_sensor<2, float><<<nb, 256, 0, s>>>(d, C, B, region);
  } else {
    if (C.L == 3) k_sensor<3, double><<<nb, 256, 0, s>>>(d, C, B, region);
    else k_sensor<2, double><<<nb, 256, 0, s>>>(d, C, B, region);
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
                      int stage, cudaStream_t s) {
  k_rk_update<<<blocks_for(d.N, 256), 256, 0, s>>>(d, C, B, w, r_old, stage);
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

void launch_theta_set(const Dims& d, const Bufs& B, const double* theta, cudaStream_t s) {
  k_theta_set<<<blocks_for(d.N, 256), 256, 0, s>>>(d, B, theta);
}

void launch_d2f(const double* x, float* y, long long n, cudaStream_t s) {
  if (n > 0) k_convert_d2f<<<(unsigned)std::min<long long>(blocks_for(n, 256), 4096), 256, 0, s>>>(x, y, n);
}

void launch_f2d(const float* x, double* y, long long n, cudaStream_t s) {
  if (n > 0) k_convert_f2d<<<(unsigned)std::min<long long>(blocks_for(n, 256), 4096), 256, 0, s>>>(x, y, n);
}

// Copy n doubles between device memory and a page-locked host buffer mapped into the device's
// address space (src or dst is the mapped pointer; both 16-byte aligned): 16-byte loads and
// stores in a grid-stride loop, the odd last element by one thread. On the GB300 node the
// GPU's loads and stores cross the CPU-GPU link at 188-210 GB/s whatever the buffer's history,
// where the copy engines' device-to-host rate fell to 7-130 GB/s for buffers page-locked some
// seconds earlier.
__global__ void __launch_bounds__(256) k_copy_mapped(const double2* STRM_RO src, double2* STRM_RO dst,
                                                     long long n) {
  const long long n2 = n >> 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
    reinterpret_cast<double*>(dst)[n - 1] = reinterpret_cast<const double*>(src)[n - 1];
}

void launch_copy_mapped(const double* src, double* dst, long long n, int sms, cudaStream_t s) {
  if (n > 0)
    k_copy_mapped<<<(unsigned)std::min<long long>(blocks_for(n / 2 + 1, 256), 8LL * sms), 256, 0, s>>>(
        reinterpret_cast<const double2*>(src), reinterpret_cast<double2*>(dst), n);
}

}  // namespace strm
