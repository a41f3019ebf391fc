// Face kernels of one grid (central energy-consistent flux, characteristic LF-WENO5 at the faces
// the Ducros sensor flags) and the assembly of the residual with the viscous terms.
//
// Per direction: k_classify splits the faces into a WENO list and a central list (one atomic per
// list and block), k_central and k_weno then run over their lists without warp divergence whatever the
// flagged fraction (a per-face branch would run both paths in most warps). k_assemble then forms
// R = -sum_d (f_{s+1} - f_s)/h_d + viscous terms per node and the forcing partial sums. The
// bodies are in strm_body.cuh.
#include "strm_body.cuh"
#include "strm_launch.h"

namespace strm {

template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) k_classify(Dims d, Consts C, Bufs B) {
  body_classify<L, DIR, R>(d, C, B, blockIdx.x);
}

// Sensor mode, y and z faces: the sweep over every face replaces the central list when enough
// faces are central. It computes about 76 FP64 operations per face against the list's 86 but
// also at the WENO faces, so in FP64 (pipe-bound) it pays from about 88 % central faces and is
// chosen from 85 %; in mixed precision (memory-bound) it reads one node per face instead of 2L
// and is chosen from 50 %. The choice is taken on the device from the classification's count,
// so a captured graph keeps both launches.
template <typename R>
__device__ __forceinline__ bool sweep_chosen(unsigned central, long long nf) {
  return sizeof(R) == sizeof(double) ? 20LL * central >= 17LL * nf : 2LL * central >= nf;
}

// use_list: the compacted central list of the sensor mode; yield: the list kernel of a y or z
// direction leaves the faces to the sweep when sweep_chosen.
template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) k_central(Dims d, Consts C, Bufs B, int use_list, int yield) {
  if (yield && sweep_chosen<R>(B.wcount[4 + DIR], d.nf[DIR])) return;
  body_central<L, DIR, R>(d, C, B, use_list, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                          (long long)gridDim.x * blockDim.x);
}

// Sweep over every y or z face (body_central_sweep); in sensor mode it runs only when
// sweep_chosen (the WENO kernel then overwrites the flagged faces).
template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) k_central_sweep(Dims d, Consts C, Bufs B, int sensor) {
  if (sensor && !sweep_chosen<R>(B.wcount[4 + DIR], d.nf[DIR])) return;
  body_central_sweep<L, DIR, R>(d, C, B, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int DIR, bool MIXED>
__global__ void __launch_bounds__(128, MIXED ? 5 : 3) k_weno(Dims d, Consts C, Bufs B) {
  body_weno<DIR, MIXED>(d, C, B, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                        (long long)gridDim.x * blockDim.x);
}

template <int L, typename R>
__global__ void __launch_bounds__(256) k_assemble(Dims d, Consts C, Bufs B, double* __restrict__ Rout,
                                                  RkFuse rk) {
  __shared__ double sh[32];
  body_assemble<L, R>(d, C, B, Rout, blockIdx.x, sh, rk);
}

// ------------------------------------------------------------------------------ launchers

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Threads of the sweep along DIR: one per (x, column, segment of kSweepSeg faces).
static long long sweep_threads(const Dims& d, int dir) {
  const long long nfa = (dir == 1 ? d.ny : d.nz) + 1;
  return (long long)d.nx * (dir == 1 ? d.nz : d.ny) * ((nfa + kSweepSeg - 1) / kSweepSeg);
}

template <int L, int DIR, typename R>
static int faces_one(const Dims& d, const Consts& C, const Bufs& B, bool sensor, unsigned nb, int grid,
                     cudaStream_t s) {
  int n = 0;
  if (sensor) {
    k_classify<L, DIR, R><<<nb, 256, 0, s>>>(d, C, B);
    ++n;
  }
  if constexpr (DIR == 0) {
    k_central<L, DIR, R><<<sensor ? (unsigned)grid : nb, 256, 0, s>>>(d, C, B, sensor ? 1 : 0, 0);
    return n + 1;
  } else {
    k_central_sweep<L, DIR, R><<<blocks_for(sweep_threads(d, DIR), 256), 256, 0, s>>>(d, C, B, sensor ? 1 : 0);
    ++n;
    if (sensor) {
      k_central<L, DIR, R><<<(unsigned)grid, 256, 0, s>>>(d, C, B, 1, 1);
      ++n;
    }
    return n;
  }
}

template <int L, typename R>
static int faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, bool sensor, unsigned nb,
                     int grid, cudaStream_t s) {
  if (dir == 0) return faces_one<L, 0, R>(d, C, B, sensor, nb, grid, s);
  if (dir == 1) return faces_one<L, 1, R>(d, C, B, sensor, nb, grid, s);
  return faces_one<L, 2, R>(d, C, B, sensor, nb, grid, s);
}

// Face stage of one direction: sensor mode classifies, then the x direction runs the central
// list and the y and z directions either sweep every face or run the list (chosen on the device
// from the central count); WENO off sweeps (y, z) or covers (x) every face; WENO everywhere needs
// no central flux. Returns the number of kernels launched.
int launch_faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s) {
  if (C.weno_mode == 2) return 0;
  bool sensor = C.weno_mode == 1;
  unsigned nb = blocks_for(d.nf[dir], 256);
  if (C.mixed) {
    if (C.L == 3) return faces_dir<3, float>(d, C, B, dir, sensor, nb, grid, s);
    return faces_dir<2, float>(d, C, B, dir, sensor, nb, grid, s);
  }
  if (C.L == 3) return faces_dir<3, double>(d, C, B, dir, sensor, nb, grid, s);
  return faces_dir<2, double>(d, C, B, dir, sensor, nb, grid, s);
}

void launch_weno_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s) {
  if (C.mixed) {
    if (dir == 0) k_weno<0, true><<<grid, 128, 0, s>>>(d, C, B);
    else if (dir == 1) k_weno<1, true><<<grid, 128, 0, s>>>(d, C, B);
    else k_weno<2, true><<<grid, 128, 0, s>>>(d, C, B);
  } else {
    if (dir == 0) k_weno<0, false><<<grid, 128, 0, s>>>(d, C, B);
    else if (dir == 1) k_weno<1, false><<<grid, 128, 0, s>>>(d, C, B);
    else k_weno<2, false><<<grid, 128, 0, s>>>(d, C, B);
  }
}

void launch_assemble(const Dims& d, const Consts& C, const Bufs& B, double* R, const RkFuse& rk,
                     cudaStream_t s) {
  unsigned nb = blocks_for(d.N, kRedBlock);
  if (C.mixed) {
    if (C.L == 3) k_assemble<3, float><<<nb, kRedBlock, 0, s>>>(d, C, B, R, rk);
    else k_assemble<2, float><<<nb, kRedBlock, 0, s>>>(d, C, B, R, rk);
  } else {
    if (C.L == 3) k_assemble<3, double><<<nb, kRedBlock, 0, s>>>(d, C, B, R, rk);
    else k_assemble<2, double><<<nb, kRedBlock, 0, s>>>(d, C, B, R, rk);
  }
}

}  // namespace strm
