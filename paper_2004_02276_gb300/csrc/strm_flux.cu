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

template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) k_central(Dims d, Consts C, Bufs B, int use_list) {
  body_central<L, DIR, R>(d, C, B, use_list, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                          (long long)gridDim.x * blockDim.x);
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

template <int L, int DIR, typename R>
static void faces_one(const Dims& d, const Consts& C, const Bufs& B, bool sensor, unsigned nb, int grid,
                      cudaStream_t s) {
  if (sensor) k_classify<L, DIR, R><<<nb, 256, 0, s>>>(d, C, B);
  k_central<L, DIR, R><<<sensor ? (unsigned)grid : nb, 256, 0, s>>>(d, C, B, sensor ? 1 : 0);
}

template <int L, typename R>
static void faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, bool sensor, unsigned nb,
                      int grid, cudaStream_t s) {
  if (dir == 0) faces_one<L, 0, R>(d, C, B, sensor, nb, grid, s);
  else if (dir == 1) faces_one<L, 1, R>(d, C, B, sensor, nb, grid, s);
  else faces_one<L, 2, R>(d, C, B, sensor, nb, grid, s);
}

// Face stage of one direction: sensor mode classifies then runs the central list; WENO off runs
// the central flux over every face; WENO everywhere needs no central flux.
void launch_faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s) {
  if (C.weno_mode == 2) return;
  bool sensor = C.weno_mode == 1;
  unsigned nb = blocks_for(d.nf[dir], 256);
  if (C.mixed) {
    if (C.L == 3) faces_dir<3, float>(d, C, B, dir, sensor, nb, grid, s);
    else faces_dir<2, float>(d, C, B, dir, sensor, nb, grid, s);
  } else {
    if (C.L == 3) faces_dir<3, double>(d, C, B, dir, sensor, nb, grid, s);
    else faces_dir<2, double>(d, C, B, dir, sensor, nb, grid, s);
  }
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
