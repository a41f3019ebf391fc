// Batched ensemble: the device table of instances and the block-to-instance mapping shared by
// the per-kernel-type ensemble kernels (strm_batch.cu) and the persistent stage kernel
// (strm_persist.cu). Internal to the library.
#pragma once

#include "strm_body.cuh"

namespace strm {

struct Inst {
  Dims d;
  Consts C;
  Bufs B;
  double* w;
  double* r_old;
};

// Index spaces of the ensemble kernels: nodes, ghost nodes, faces of x/y/z, wall-normal rows.
enum { kKindNode = 0, kKindGhost = 1, kKindFace = 2, kKindRow = 5, kKinds = 6 };

struct BatchIndex {
  const Inst* inst;  // device table [n]
  const int* start;  // device block starts [kKinds][n + 1]
  int n;
};

__device__ __forceinline__ int find_inst(const int* start, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Instance of the (virtual) block b of kernel kind k, and the block index it plays within the
// instance.
__device__ __forceinline__ const Inst& inst_of_block(const BatchIndex& X, int kind, int b, int& blk) {
  const int* st = X.start + kind * (X.n + 1);
  int e = find_inst(st, X.n, b);
  blk = b - st[e];
  return X.inst[e];
}

__device__ __forceinline__ int inst_blocks(const BatchIndex& X, int kind, int e) {
  const int* st = X.start + kind * (X.n + 1);
  return st[e + 1] - st[e];
}

__device__ __forceinline__ long long ghost_count(const Dims& d) {
  return 2LL * G * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
}

// One RK stage of every instance in one cooperative launch (strm_persist.cu).
struct StageArgs {
  unsigned* bar;               // grid barrier: [0] arrivals, [1] generation, [2] gave-up flag
  unsigned long long limit_ns; // a barrier gives up after this long (all blocks then leave)
  double cfl, dt_fixed;        // stage 0: the step from the CFL number, or the fixed step
  int stage;                   // 0, 1, 2; -1: the right-hand side only (no dt, no update)
  int any_recycle;             // some instance has a recycling inflow
  int total[kKinds];           // virtual blocks per index space
};

// Threads per block of the persistent stage kernel (the ensemble's block partition).
constexpr int kStageBlock = 256;

// Blocks per SM of the persistent stage kernel for L and precision (0 when it cannot run).
int persistent_blocks_per_sm(int L, bool mixed);
// Enqueue one persistent stage launch of grid blocks (a multiple of the SM count).
cudaError_t launch_persistent_stage(int L, bool mixed, const BatchIndex& X, const StageArgs& A, int grid,
                                    cudaStream_t s);

}  // namespace strm
