// Digital-filter turbulent inflow (Section 3.2: a Klein-type digital filter done as a sequence
// of one-dimensional convolutions, extended to compressible flow by the strong Reynolds analogy,
// with prescribed Reynolds stresses). Once per time step, after the CFL step is known:
//   1. random numbers of zero mean and unit variance, r = sqrt(3) (2u - 1), u from SplitMix64
//      keyed by (draw, velocity component, z index, extended y index); generated where they are
//      used, so no random plane is stored;
//   2. the filter b_l (l = -2n..2n) along y on the plane extended by 2n rows on both sides
//      (k_df_yfilter), then along z, periodic (k_df_zfilter);
//   3. time correlation Psi <- Psi exp(-pi dt / (2 tau)) + psi sqrt(1 - exp(-pi dt / tau)).
// The draw counter lives on the device, so a captured step graph draws a new plane at every
// replay. The ghost states (Cholesky transform and strong Reynolds analogy) are formed by the
// ghost-fill kernel from Psi.
#include <cstdint>

#include "strm_launch.h"

namespace strm {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// one thread per (component m, z index k, y index j): t = sum_l by_l r(j + l)
__global__ void __launch_bounds__(256) k_df_yfilter(Dims d, DFParams F) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long plane = (long long)d.nz * d.ny;
  if (q >= 3 * plane) return;
  int m = (int)(q / plane);
  long long r = q - m * plane;
  int k = (int)(r / d.ny), j = (int)(r - (long long)k * d.ny);
  const int Ny = 2 * F.ny;
  const uint64_t nye = (uint64_t)d.ny + 2 * (uint64_t)Ny;
  const uint64_t draw = (uint64_t)*F.count;
  const uint64_t base = ((draw * 3 + (uint64_t)m) * (uint64_t)d.nz + (uint64_t)k) * nye + (uint64_t)j;
  const double s3 = 1.7320508075688772;  // sqrt(3)
  double s = 0.0;
  for (int l = 0; l <= 2 * Ny; ++l) {
    double u = (double)(splitmix64(F.seed, base + (uint64_t)l) >> 11) * (1.0 / 9007199254740992.0);
    s = fma(__ldg(F.by + l), s3 * (2.0 * u - 1.0), s);
  }
  F.t[q] = s;
}

// one thread per (m, k, j): psi = sum_l bz_l t(k + l mod nz), then the time blend (first draw:
// Psi = psi); thread 0 advances the draw counter (read by k_df_yfilter before this launch).
__global__ void __launch_bounds__(256) k_df_zfilter(Dims d, DFParams F, const double* __restrict__ scal,
                                                    int first) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long plane = (long long)d.nz * d.ny;
  if (q == 0) *F.count += 1;
  if (q >= 3 * plane) return;
  int m = (int)(q / plane);
  long long r = q - m * plane;
  int k = (int)(r / d.ny), j = (int)(r - (long long)k * d.ny);
  const int Nz = 2 * F.nz;
  const double* tm = F.t + m * plane;
  double s = 0.0;
  for (int l = -Nz; l <= Nz; ++l) {
    int kk = k + l;
    kk = ((kk % d.nz) + d.nz) % d.nz;
    s = fma(__ldg(F.bz + l + Nz), tm[(long long)kk * d.ny + j], s);
  }
  if (first) {
    F.psi[q] = s;
  } else {
    const double pi = 3.141592653589793;
    double dt = scal[kScalDt];
    double e1 = exp(-pi * dt / (2.0 * F.tau)), e2 = sqrt(1.0 - exp(-pi * dt / F.tau));
    F.psi[q] = fma(F.psi[q], e1, s * e2);
  }
}

}  // namespace

void launch_df_update(const Dims& d, const DFParams& F, const Bufs& B, bool first, cudaStream_t s) {
  long long n = 3LL * d.nz * d.ny;
  unsigned nb = (unsigned)((n + 255) / 256);
  k_df_yfilter<<<nb, 256, 0, s>>>(d, F);
  k_df_zfilter<<<nb, 256, 0, s>>>(d, F, B.scal, first ? 1 : 0);
}

}  // namespace strm
