// Persistent ensemble stage: one cooperative launch runs a whole RK stage of every instance of
// an ensemble (Section 2 right-hand side, then the Eq. RK update). Each block walks the virtual
// blocks of every phase in a grid-stride loop and plays the same device bodies the
// per-kernel-type ensemble kernels run, so every instance computes what its own context
// computes; a grid-wide barrier separates the phases:
//
//   primitives (+ CFL partials at stage 0) | dt (stage 0), recycling means | recycling scale |
//   ghost fill | Ducros sensor | (mixed) FP64 sensor at near-threshold nodes | sensor and
//   divergence ghosts | face classification x, y, z | central and WENO faces x, y, z |
//   assembly | forcing | stage update
//
// Data written in one phase is read by other blocks in later phases of the same launch, so this
// translation unit compiles the bodies with ordinary (coherent) loads instead of the read-only
// path. A block plays several virtual blocks in a row; a __syncthreads after each keeps the
// bodies' shared-memory reductions and list appends of consecutive virtual blocks apart. The
// barrier's waits are bounded: after StageArgs::limit_ns a block gives up, sets the flag that
// every waiting block also reads, and all blocks leave the kernel.
#define STRM_COHERENT_LOADS
#include <type_traits>

#include "strm_batch.h"

namespace strm {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every block resident). Thread 0 of each block
// reads the generation, arrives, and the last arrival resets the count and publishes the next
// generation; the others wait for it, at most limit_ns, and leave early when another block has
// given up. Returns false when this barrier (or an earlier one) gave up.
__device__ bool grid_barrier(unsigned* bar, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      st_release_u32(bar + 1, gen + 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(bar + 1) == gen) {
        if (ld_acquire_u32(bar + 2) != 0u) break;
        if (global_ns() - t0 >= limit_ns) {  // limit 0: the first block that must wait gives up
          atomicOr(bar + 2, 1u);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (ld_acquire_u32(bar + 2) != 0u) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Resident blocks per SM: 2 in FP64 (128 registers; its phases are bound by the FP64 pipe), 4 in
// mixed precision (64 registers; its FP32 and memory-bound phases want the occupancy: 0.76 of the
// per-kernel schedule's rate on the 64-channel ensemble against 0.68 with 2).
template <int L, bool MIXED>
__global__ void __launch_bounds__(kStageBlock, MIXED ? 4 : 2) kb_stage(BatchIndex X, StageArgs A) {
  using R = typename std::conditional<MIXED, float, double>::type;
  __shared__ double sh[32];
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ts = (long long)gridDim.x * blockDim.x;
  const bool rhs_only = A.stage < 0;

  // the face lists and the mixed sensor's band list start empty (appended to after barriers)
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < X.n; e += blockDim.x)
      for (int c = 0; c < 8; ++c) X.inst[e].B.wcount[c] = 0u;

  const int want_cfl = A.stage == 0 && A.dt_fixed <= 0.0;
  for (int b = blockIdx.x; b < A.total[kKindNode]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindNode, b, blk);
    if (MIXED) body_prims_mixed(I.d, I.C, I.B, I.w, want_cfl, blk, sh);
    else body_prims(I.d, I.C, I.B, I.w, want_cfl, blk, sh);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  if (A.stage == 0)
    for (int e = blockIdx.x; e < X.n; e += gridDim.x) {
      body_dt_finalize(X.inst[e].B, inst_blocks(X, kKindNode, e), A.cfl, A.dt_fixed, sh);
      __syncthreads();
    }
  if (A.any_recycle) {
    for (int b = blockIdx.x; b < A.total[kKindRow]; b += gridDim.x) {
      int blk;
      const Inst& I = inst_of_block(X, kKindRow, b, blk);
      if (I.C.bc[0] == kBcRecycle) body_recycle_mean(I.d, I.C, I.B, blk, sh);
      __syncthreads();
    }
    if (!grid_barrier(A.bar, A.limit_ns)) return;
    for (int e = blockIdx.x; e < X.n; e += gridDim.x) {
      const Inst& I = X.inst[e];
      if (I.C.bc[0] == kBcRecycle && threadIdx.x == 0) body_recycle_scale(I.d, I.C, I.B);
    }
    if (!grid_barrier(A.bar, A.limit_ns)) return;
  }

  for (int b = blockIdx.x; b < A.total[kKindGhost]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindGhost, b, blk);
    body_ghost_prims(I.d, I.C, I.B, ghost_count(I.d), blk);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  for (int b = blockIdx.x; b < A.total[kKindNode]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindNode, b, blk);
    body_sensor<L, R>(I.d, I.C, I.B, blk);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;
  if (MIXED) {
    for (int e = 0; e < X.n; ++e) {
      const Inst& I = X.inst[e];
      if (I.C.weno_mode == 1) body_band_theta<L>(I.d, I.C, I.B, t0, ts);
    }
    if (!grid_barrier(A.bar, A.limit_ns)) return;
  }

  for (int b = blockIdx.x; b < A.total[kKindGhost]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindGhost, b, blk);
    body_ghost_scalars<R>(I.d, I.C, I.B, ghost_count(I.d), blk);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  for (int b = blockIdx.x; b < A.total[kKindFace + 0]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindFace + 0, b, blk);
    if (I.C.weno_mode == 1) body_classify<L, 0, R>(I.d, I.C, I.B, blk);
    __syncthreads();
  }
  for (int b = blockIdx.x; b < A.total[kKindFace + 1]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindFace + 1, b, blk);
    if (I.C.weno_mode == 1) body_classify<L, 1, R>(I.d, I.C, I.B, blk);
    __syncthreads();
  }
  for (int b = blockIdx.x; b < A.total[kKindFace + 2]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindFace + 2, b, blk);
    if (I.C.weno_mode == 1) body_classify<L, 2, R>(I.d, I.C, I.B, blk);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  // central and WENO faces write disjoint faces of each direction's flux array
  for (int e = 0; e < X.n; ++e) {
    const Inst& I = X.inst[e];
    const int mode = I.C.weno_mode;
    if (mode != 2) {
      body_central<L, 0, R>(I.d, I.C, I.B, mode == 1 ? 1 : 0, t0, ts);
      body_central<L, 1, R>(I.d, I.C, I.B, mode == 1 ? 1 : 0, t0, ts);
      body_central<L, 2, R>(I.d, I.C, I.B, mode == 1 ? 1 : 0, t0, ts);
    }
    if (mode != 0) {
      body_weno<0, MIXED>(I.d, I.C, I.B, t0, ts);
      body_weno<1, MIXED>(I.d, I.C, I.B, t0, ts);
      body_weno<2, MIXED>(I.d, I.C, I.B, t0, ts);
    }
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  for (int b = blockIdx.x; b < A.total[kKindNode]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindNode, b, blk);
    body_assemble<L, R>(I.d, I.C, I.B, I.B.R, blk, sh);
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  for (int e = blockIdx.x; e < X.n; e += gridDim.x) {
    const Inst& I = X.inst[e];
    body_force_finalize(I.B, inst_blocks(X, kKindNode, e), 1.0 / I.C.vtot, sh);
    __syncthreads();
  }
  if (rhs_only) return;
  if (!grid_barrier(A.bar, A.limit_ns)) return;

  for (int b = blockIdx.x; b < A.total[kKindNode]; b += gridDim.x) {
    int blk;
    const Inst& I = inst_of_block(X, kKindNode, b, blk);
    body_rk_update(I.d, I.C, I.B, I.w, I.r_old, A.stage, blk);
  }
}

namespace {

template <int L, bool MIXED>
int blocks_per_sm_t() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb_stage<L, MIXED>, kStageBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <int L, bool MIXED>
cudaError_t launch_t(const BatchIndex& X, const StageArgs& A, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kStageBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kb_stage<L, MIXED>, X, A);
}

}  // namespace

int persistent_blocks_per_sm(int L, bool mixed) {
  if (L == 3) return mixed ? blocks_per_sm_t<3, true>() : blocks_per_sm_t<3, false>();
  return mixed ? blocks_per_sm_t<2, true>() : blocks_per_sm_t<2, false>();
}

cudaError_t launch_persistent_stage(int L, bool mixed, const BatchIndex& X, const StageArgs& A, int grid,
                                    cudaStream_t s) {
  if (L == 3) return mixed ? launch_t<3, true>(X, A, grid, s) : launch_t<3, false>(X, A, grid, s);
  return mixed ? launch_t<2, true>(X, A, grid, s) : launch_t<2, false>(X, A, grid, s);
}

}  // namespace strm
