// Batched ensemble: many independent grids (uneven sizes, Mach and Reynolds numbers) advanced
// together. Every kernel type of a right-hand side runs as one launch over all instances: the
// node, ghost and face index spaces of the instances are concatenated with each instance padded
// to whole blocks, and a block finds its instance by binary search over per-kernel-type block
// offsets; the list kernels (central and WENO faces) walk the instances in a grid-stride loop.
// One RK3 step of the whole ensemble is captured once as a CUDA graph and replayed. The launch
// shapes of the list kernels are chosen by a small autotuner that times the candidates on the
// ensemble itself.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include "../../include/strm.h"
#include "strm_batch.h"
#include "strm_launch.h"

namespace strm {

// Instance of this block for kernel kind k, and the block index it plays within the instance.
__device__ __forceinline__ const Inst& block_inst(const BatchIndex& X, int kind, int& blk) {
  return inst_of_block(X, kind, blockIdx.x, blk);
}

__global__ void kb_zero_counts(BatchIndex X) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= X.n) return;
  for (int c = 0; c < 8; ++c) X.inst[e].B.wcount[c] = 0u;
}

template <bool MIXED>
__global__ void __launch_bounds__(256) kb_prims(BatchIndex X, int want_cfl) {
  __shared__ double sh[32];
  int blk;
  const Inst& I = block_inst(X, kKindNode, blk);
  if (MIXED) body_prims_mixed(I.d, I.C, I.B, I.w, want_cfl, blk, sh);
  else body_prims(I.d, I.C, I.B, I.w, want_cfl, blk, sh);
}

__global__ void kb_dt_finalize(BatchIndex X, double cfl, double dt_fixed) {
  __shared__ double sh[32];
  const Inst& I = X.inst[blockIdx.x];
  body_dt_finalize(I.B, inst_blocks(X, kKindNode, blockIdx.x), cfl, dt_fixed, sh);
}

__global__ void __launch_bounds__(256) kb_ghost_prims(BatchIndex X) {
  int blk;
  const Inst& I = block_inst(X, kKindGhost, blk);
  body_ghost_prims(I.d, I.C, I.B, ghost_count(I.d), blk);
}

// recycling inflow: spanwise means (one block per row j of every recycling instance), then the
// rescale factor (one block per instance)
__global__ void kb_recycle_mean(BatchIndex X) {
  __shared__ double sh[32];
  int blk;
  const Inst& I = block_inst(X, kKindRow, blk);
  if (I.C.bc[0] != kBcRecycle) return;
  body_recycle_mean(I.d, I.C, I.B, blk, sh);
}

__global__ void kb_recycle_scale(BatchIndex X) {
  const Inst& I = X.inst[blockIdx.x];
  if (I.C.bc[0] == kBcRecycle && threadIdx.x == 0) body_recycle_scale(I.d, I.C, I.B);
}

template <int L, typename R>
__global__ void __launch_bounds__(256) kb_sensor(BatchIndex X) {
  int blk;
  const Inst& I = block_inst(X, kKindNode, blk);
  body_sensor<L, R>(I.d, I.C, I.B, blk);
}

template <int L>
__global__ void __launch_bounds__(128) kb_band_theta(BatchIndex X) {
  long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ts = (long long)gridDim.x * blockDim.x;
  for (int e = 0; e < X.n; ++e) {
    const Inst& I = X.inst[e];
    if (I.C.weno_mode == 1) body_band_theta<L>(I.d, I.C, I.B, t0, ts);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) kb_ghost_scalars(BatchIndex X) {
  int blk;
  const Inst& I = block_inst(X, kKindGhost, blk);
  body_ghost_scalars<R>(I.d, I.C, I.B, ghost_count(I.d), blk);
}

template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) kb_classify(BatchIndex X) {
  int blk;
  const Inst& I = block_inst(X, kKindFace + DIR, blk);
  if (I.C.weno_mode != 1) return;
  body_classify<L, DIR, R>(I.d, I.C, I.B, blk);
}

template <int L, int DIR, typename R>
__global__ void __launch_bounds__(256) kb_central(BatchIndex X) {
  long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ts = (long long)gridDim.x * blockDim.x;
  for (int e = 0; e < X.n; ++e) {
    const Inst& I = X.inst[e];
    int mode = I.C.weno_mode;
    if (mode != 2) body_central<L, DIR, R>(I.d, I.C, I.B, mode == 1 ? 1 : 0, t0, ts);
  }
}

// At most 128 threads per block, with the register budget of 3 (FP64) or 4 (mixed) resident
// blocks per SM: the instance fields read from the table in global memory live in registers,
// where the single-context kernel reads them from its constant parameter bank, and without the
// bound the compiler took 210 (FP64) and 138 (mixed) registers.
template <int DIR, bool MIXED>
__global__ void __launch_bounds__(128, MIXED ? 4 : 3) kb_weno(BatchIndex X) {
  long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ts = (long long)gridDim.x * blockDim.x;
  for (int e = 0; e < X.n; ++e) {
    const Inst& I = X.inst[e];
    if (I.C.weno_mode != 0) body_weno<DIR, MIXED>(I.d, I.C, I.B, t0, ts);
  }
}

// Register budget of 3 (mixed) or 2 (FP64) resident blocks, for the same reason as kb_weno
// (unbounded, the mixed instance took 114 registers against 62 in the single-context kernel).
template <int L, typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) kb_assemble(BatchIndex X) {
  __shared__ double sh[32];
  int blk;
  const Inst& I = block_inst(X, kKindNode, blk);
  body_assemble<L, R>(I.d, I.C, I.B, I.B.R, blk, sh);
}

__global__ void kb_force_finalize(BatchIndex X) {
  __shared__ double sh[32];
  const Inst& I = X.inst[blockIdx.x];
  body_force_finalize(I.B, inst_blocks(X, kKindNode, blockIdx.x), 1.0 / I.C.vtot, sh);
}

__global__ void __launch_bounds__(256) kb_rk_update(BatchIndex X, int stage) {
  int blk;
  const Inst& I = block_inst(X, kKindNode, blk);
  body_rk_update(I.d, I.C, I.B, I.w, I.r_old, stage, blk);
}

}  // namespace strm

using namespace strm;

namespace {


size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

long long ghost_count_host(const Dims& d) {
  return 2LL * G * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
}

struct Tuning {
  int weno_block = 128;
  int weno_per_sm = 8;
  int central_per_sm = 16;
  int persistent = 0;  // 1: one cooperative launch per RK stage (strm_persist.cu)
  int slab_cap = 32;   // largest slab height of the slab traversal order (0: natural order)
};

// A barrier of the persistent stage gave up (error word bit; the context bits are kDbg*).
constexpr unsigned kEnsembleBarrier = 32u;
// Time after which a barrier of the persistent stage gives up.
constexpr unsigned long long kBarrierLimitNs = 10000000000ull;

}  // namespace

struct strm_ensemble {
  int n = 0;
  int L = 3;
  bool mixed = false;
  bool any_recycle = false;
  bool dirty = false;  // an instance's constants changed since the table upload
  cudaStream_t stream = nullptr;
  int sms = 0;
  std::vector<strm_ctx*> ctx;
  std::vector<Inst> inst_host;
  std::vector<int> start_host;  // [kKinds][n + 1]
  int total_blocks[kKinds] = {};
  Inst* inst_dev = nullptr;
  int* start_dev = nullptr;
  unsigned* bar_dev = nullptr;  // persistent-stage barrier [3] (zeroed at creation)
  int stage_grid = 0;           // blocks of the persistent stage launch (0: not available)
  unsigned long long barrier_ns = kBarrierLimitNs;  // a persistent-stage barrier gives up after this
  Tuning tune;
  // graph of one RK step of the ensemble
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double*> g_w, g_r;
  double g_cfl = 0.0, g_dt = 0.0;
  std::vector<double> time_host;
};

namespace {

#define STRME_CK(call)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return record_error(STRM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

BatchIndex index_of(const strm_ensemble* E) { return BatchIndex{E->inst_dev, E->start_dev, E->n}; }

StageArgs stage_args(const strm_ensemble* E, int stage, double cfl, double dt_fixed) {
  StageArgs A = {};
  A.bar = E->bar_dev;
  A.limit_ns = E->barrier_ns;
  A.cfl = cfl;
  A.dt_fixed = dt_fixed;
  A.stage = stage;
  A.any_recycle = E->any_recycle ? 1 : 0;
  for (int k = 0; k < kKinds; ++k) A.total[k] = E->total_blocks[k];
  return A;
}

// One right-hand side of every instance into its workspace residual (and, with dt_mode, the
// per-instance step of stage 0).
template <int L, bool MIXED>
void enqueue_rhs_t(const strm_ensemble* E, bool dt_mode, double cfl, double dt_fixed, cudaStream_t st) {
  using R = typename std::conditional<MIXED, float, double>::type;
  BatchIndex X = index_of(E);
  const Tuning& T = E->tune;
  kb_zero_counts<<<nblocks(E->n, 32), 32, 0, st>>>(X);
  kb_prims<MIXED><<<E->total_blocks[kKindNode], 256, 0, st>>>(X, dt_mode && dt_fixed <= 0.0 ? 1 : 0);
  if (dt_mode) kb_dt_finalize<<<E->n, 1024, 0, st>>>(X, cfl, dt_fixed);
  if (E->any_recycle) {
    kb_recycle_mean<<<E->total_blocks[kKindRow], 256, 0, st>>>(X);
    kb_recycle_scale<<<E->n, 32, 0, st>>>(X);
  }
  // digital-filter inflows: a new plane per step for each instance that has one
  if (dt_mode)
    for (int e = 0; e < E->n; ++e) {
      DFParams F;
      if (ctx_df(E->ctx[e], &F)) launch_df_update(E->inst_host[e].d, F, E->inst_host[e].B, false, st);
    }
  kb_ghost_prims<<<E->total_blocks[kKindGhost], 256, 0, st>>>(X);
  kb_sensor<L, R><<<E->total_blocks[kKindNode], 256, 0, st>>>(X);
  if (MIXED) kb_band_theta<L><<<(unsigned)(E->sms * 8), 128, 0, st>>>(X);
  kb_ghost_scalars<R><<<E->total_blocks[kKindGhost], 256, 0, st>>>(X);
  kb_classify<L, 0, R><<<E->total_blocks[kKindFace + 0], 256, 0, st>>>(X);
  kb_classify<L, 1, R><<<E->total_blocks[kKindFace + 1], 256, 0, st>>>(X);
  kb_classify<L, 2, R><<<E->total_blocks[kKindFace + 2], 256, 0, st>>>(X);
  unsigned cg = (unsigned)(E->sms * T.central_per_sm);
  kb_central<L, 0, R><<<cg, 256, 0, st>>>(X);
  kb_central<L, 1, R><<<cg, 256, 0, st>>>(X);
  kb_central<L, 2, R><<<cg, 256, 0, st>>>(X);
  unsigned wg = (unsigned)(E->sms * T.weno_per_sm);
  kb_weno<0, MIXED><<<wg, T.weno_block, 0, st>>>(X);
  kb_weno<1, MIXED><<<wg, T.weno_block, 0, st>>>(X);
  kb_weno<2, MIXED><<<wg, T.weno_block, 0, st>>>(X);
  kb_assemble<L, R><<<E->total_blocks[kKindNode], 256, 0, st>>>(X);
  kb_force_finalize<<<E->n, 1024, 0, st>>>(X);
}

void enqueue_rhs(const strm_ensemble* E, bool dt_mode, double cfl, double dt_fixed, cudaStream_t st) {
  if (E->tune.persistent && !dt_mode) {  // the tuner's right-hand side: no dt, no update
    launch_persistent_stage(E->L, E->mixed, index_of(E), stage_args(E, -1, cfl, dt_fixed), E->stage_grid, st);
    return;
  }
  if (E->L == 3) {
    if (E->mixed) enqueue_rhs_t<3, true>(E, dt_mode, cfl, dt_fixed, st);
    else enqueue_rhs_t<3, false>(E, dt_mode, cfl, dt_fixed, st);
  } else {
    if (E->mixed) enqueue_rhs_t<2, true>(E, dt_mode, cfl, dt_fixed, st);
    else enqueue_rhs_t<2, false>(E, dt_mode, cfl, dt_fixed, st);
  }
}

int enqueue_step(const strm_ensemble* E, double dt, double cfl, cudaStream_t st) {
  BatchIndex X = index_of(E);
  if (E->tune.persistent) {
    for (int stage = 0; stage < 3; ++stage) {
      cudaError_t e = launch_persistent_stage(E->L, E->mixed, X, stage_args(E, stage, cfl, dt), E->stage_grid, st);
      if (e != cudaSuccess) return record_error(STRM_ECUDA, std::string("persistent stage launch: ") + cudaGetErrorString(e));
    }
    return STRM_OK;
  }
  for (int stage = 0; stage < 3; ++stage) {
    enqueue_rhs(E, stage == 0, cfl, dt, st);
    kb_rk_update<<<E->total_blocks[kKindNode], 256, 0, st>>>(X, stage);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return record_error(STRM_ECUDA, std::string("ensemble launch: ") + cudaGetErrorString(e));
  return STRM_OK;
}

// Point the instance table at the caller's state buffers (re-uploaded only when they change).
int bind_states(strm_ensemble* E, double* const* w, double* const* r_old) {
  bool same = !E->dirty && E->g_w.size() == (size_t)E->n;
  for (int e = 0; e < E->n && same; ++e) same = E->g_w[e] == w[e] && E->g_r[e] == r_old[e];
  if (same) return STRM_OK;
  for (int e = 0; e < E->n; ++e) {
    if (!w[e] || !r_old[e] || w[e] == r_old[e]) return record_error(STRM_EINVAL, "null or aliased state buffer");
    E->inst_host[e].w = w[e];
    E->inst_host[e].r_old = r_old[e];
  }
  STRME_CK(cudaMemcpyAsync(E->inst_dev, E->inst_host.data(), sizeof(Inst) * E->n, cudaMemcpyHostToDevice,
                           E->stream));
  // the copy reads inst_host; wait so that a later change cannot race with it
  STRME_CK(cudaStreamSynchronize(E->stream));
  E->g_w.assign(w, w + E->n);
  E->g_r.assign(r_old, r_old + E->n);
  E->dirty = false;
  if (E->gexec) {
    cudaGraphExecDestroy(E->gexec);
    E->gexec = nullptr;
  }
  return STRM_OK;
}

// Refresh the host copy of instance e's constants and buffers after a boundary change; the
// device table is re-uploaded before the next launch and the step graph re-captured.
void refresh_instance(strm_ensemble* E, int e) {
  Inst& I = E->inst_host[e];
  double* w = I.w;
  double* r = I.r_old;
  int sms;
  ctx_parts(E->ctx[e], &I.d, &I.C, &I.B, &sms);
  I.w = w;
  I.r_old = r;
  E->any_recycle = false;
  for (const Inst& J : E->inst_host)
    if (J.C.bc[0] == kBcRecycle) E->any_recycle = true;
  E->dirty = true;
  if (E->gexec) {
    cudaGraphExecDestroy(E->gexec);
    E->gexec = nullptr;
  }
}

size_t table_bytes(int n) {
  return align256(sizeof(Inst) * (size_t)n) + align256(sizeof(int) * kKinds * (n + 1)) + 256;
}

bool any_df(const strm_ensemble* E) {
  DFParams F;
  for (strm_ctx* c : E->ctx)
    if (ctx_df(c, &F)) return true;
  return false;
}

// Re-upload the instance table (after a change of the instances' slab heights).
int upload_table(strm_ensemble* E) {
  STRME_CK(cudaMemcpyAsync(E->inst_dev, E->inst_host.data(), sizeof(Inst) * E->n, cudaMemcpyHostToDevice,
                           E->stream));
  STRME_CK(cudaStreamSynchronize(E->stream));
  return STRM_OK;
}

// Slab height of every instance: the largest admitted one not above cap (0: natural order).
void apply_slab_cap(strm_ensemble* E, int cap) {
  for (Inst& I : E->inst_host) {
    I.d.slab_ty = slab_rows_for(I.d.nx, I.d.ny, cap);
    I.d.zslab_ty = slab_rows_for(I.d.nx, I.d.ny, cap < 8 ? cap : 8);
  }
  E->tune.slab_cap = cap;
}

// Validate and apply a schedule choice {weno block, WENO blocks per SM, central blocks per SM,
// persistent, slab cap}; the table and the step graph are refreshed at the next advance.
int set_schedule(strm_ensemble* E, const int* c) {
  const bool blk_ok = c[0] == 32 || c[0] == 64 || c[0] == 128;
  if (!blk_ok || c[1] < 1 || c[1] > 64 || c[2] < 1 || c[2] > 64 || (c[3] != 0 && c[3] != 1) ||
      !(c[4] == 0 || c[4] == 8 || c[4] == 16 || c[4] == 32))
    return record_error(STRM_EINVAL, "schedule out of range");
  if (c[3] && E->stage_grid <= 0) return record_error(STRM_EINVAL, "the persistent stage cannot run on this device");
  if (c[3] && any_df(E)) return record_error(STRM_EINVAL, "the persistent stage does not take digital-filter inflows");
  E->tune.weno_block = c[0];
  E->tune.weno_per_sm = c[1];
  E->tune.central_per_sm = c[2];
  E->tune.persistent = c[3];
  apply_slab_cap(E, c[4]);
  E->dirty = true;
  if (E->gexec) {
    cudaGraphExecDestroy(E->gexec);
    E->gexec = nullptr;
  }
  return STRM_OK;
}

void get_schedule(const strm_ensemble* E, int* c) {
  c[0] = E->tune.weno_block;
  c[1] = E->tune.weno_per_sm;
  c[2] = E->tune.central_per_sm;
  c[3] = E->tune.persistent;
  c[4] = E->tune.slab_cap;
}

}  // namespace

extern "C" {

size_t strm_ensemble_workspace_bytes(int n, const strm_grid* grids, const strm_scheme* schemes) {
  if (n < 1 || !grids || !schemes) return 0;
  size_t total = 0;
  for (int e = 0; e < n; ++e) {
    size_t b = strm_workspace_bytes(&grids[e], &schemes[e]);
    if (!b) return 0;
    total += align256(b);
  }
  return total + table_bytes(n);
}

int strm_ensemble_create(strm_ensemble** out, int n, const strm_grid* grids, const strm_phys* phys,
                         const strm_scheme* schemes, const int* bc_y, void* workspace,
                         size_t workspace_bytes, void* stream) {
  if (!out) return record_error(STRM_EINVAL, "ensemble out-pointer is null");
  *out = nullptr;
  if (n < 1 || !grids || !phys || !schemes || !bc_y) return record_error(STRM_EINVAL, "null or empty ensemble");
  for (int e = 1; e < n; ++e)
    if (schemes[e].L != schemes[0].L || schemes[e].precision != schemes[0].precision)
      return record_error(STRM_EINVAL, "ensemble instances must share L and precision");
  size_t need = strm_ensemble_workspace_bytes(n, grids, schemes);
  if (!need) return record_error(STRM_EINVAL, "invalid grid or scheme in the ensemble");
  if (!workspace || ((uintptr_t)workspace & 255)) return record_error(STRM_EINVAL, "workspace null or not 256-byte aligned");
  if (workspace_bytes < need) return record_error(STRM_ENOMEM, "workspace too small: need " + std::to_string(need));
  strm_ensemble* E = new (std::nothrow) strm_ensemble();
  if (!E) return record_error(STRM_ENOMEM, "host allocation failed");
  E->n = n;
  E->L = schemes[0].L;
  E->mixed = schemes[0].precision == STRM_PREC_MIXED;
  E->stream = (cudaStream_t)stream;
  E->inst_host.resize(n);
  E->time_host.assign(n, 0.0);
  char* ws = (char*)workspace;
  size_t off = 0;
  for (int e = 0; e < n; ++e) {
    size_t b = align256(strm_workspace_bytes(&grids[e], &schemes[e]));
    strm_ctx* c = nullptr;
    int rc = strm_init_grid(&c, &grids[e], &phys[e], &schemes[e], ws + off, b, stream);
    if (rc == STRM_OK) rc = strm_set_bc(c, STRM_FACE_YMIN_YMAX, bc_y[e], nullptr, 0);
    if (rc != STRM_OK) {
      if (c) strm_destroy(c);
      strm_ensemble_destroy(E);
      return rc;
    }
    E->ctx.push_back(c);
    Inst& I = E->inst_host[e];
    ctx_parts(c, &I.d, &I.C, &I.B, &E->sms);
    if (I.C.bc[0] == kBcRecycle) E->any_recycle = true;
    I.w = I.r_old = nullptr;
    off += b;
  }
  E->inst_dev = (Inst*)(ws + off);
  E->start_dev = (int*)(ws + off + align256(sizeof(Inst) * (size_t)n));
  E->bar_dev = (unsigned*)(ws + off + align256(sizeof(Inst) * (size_t)n) + align256(sizeof(int) * kKinds * (n + 1)));
  E->stage_grid = persistent_blocks_per_sm(E->L, E->mixed) * E->sms;
  E->start_host.assign(kKinds * (n + 1), 0);
  for (int k = 0; k < kKinds; ++k) {
    int acc = 0;
    for (int e = 0; e < n; ++e) {
      const Dims& d = E->inst_host[e].d;
      int nb;
      if (k == kKindRow) nb = d.ny;  // one block per row
      else {
        long long cnt = k == kKindNode ? d.N : (k == kKindGhost ? ghost_count_host(d) : d.nf[k - kKindFace]);
        nb = (int)nblocks(cnt, 256);
      }
      E->start_host[k * (n + 1) + e] = acc;
      acc += nb;
    }
    E->start_host[k * (n + 1) + n] = acc;
    E->total_blocks[k] = acc;
  }
  cudaError_t ce = cudaMemcpyAsync(E->start_dev, E->start_host.data(), sizeof(int) * E->start_host.size(),
                                   cudaMemcpyHostToDevice, E->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(E->bar_dev, 0, 3 * sizeof(unsigned), E->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(E->stream);
  if (ce != cudaSuccess) {
    strm_ensemble_destroy(E);
    return record_error(STRM_ECUDA, std::string("ensemble table upload: ") + cudaGetErrorString(ce));
  }
  *out = E;
  return STRM_OK;
}

int strm_ensemble_set_bc(strm_ensemble* E, int e, int face, int kind, const double* params, int nparams) {
  if (!E || e < 0 || e >= E->n) return record_error(STRM_EINVAL, "null ensemble or instance out of range");
  int rc = strm_set_bc(E->ctx[e], face, kind, params, nparams);
  if (rc) return rc;
  refresh_instance(E, e);
  return STRM_OK;
}

int strm_ensemble_debug_flags(strm_ensemble* E, unsigned* flags_host) {
  if (!E || !flags_host) return record_error(STRM_EINVAL, "null ensemble or output");
  unsigned acc = 0;
  for (strm_ctx* c : E->ctx) {
    unsigned f = 0;
    int rc = strm_debug_flags(c, &f);
    if (rc) return rc;
    acc |= f;
  }
  unsigned gave_up = 0;
  STRME_CK(cudaMemcpyAsync(&gave_up, E->bar_dev + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, E->stream));
  STRME_CK(cudaStreamSynchronize(E->stream));
  if (gave_up) {  // report once, and reset the barrier (arrivals, generation, flag) for later stages
    acc |= kEnsembleBarrier;
    STRME_CK(cudaMemsetAsync(E->bar_dev, 0, 3 * sizeof(unsigned), E->stream));
    STRME_CK(cudaStreamSynchronize(E->stream));
  }
  *flags_host = acc;
  return STRM_OK;
}

size_t strm_ensemble_inflow_df_bytes(const strm_ensemble* E, int e, const strm_df* df) {
  if (!E || e < 0 || e >= E->n) return 0;
  return strm_inflow_df_bytes(E->ctx[e], df);
}

int strm_ensemble_set_inflow_df(strm_ensemble* E, int e, const strm_df* df, const double* profiles_host,
                                void* buffer, size_t bytes) {
  if (!E || e < 0 || e >= E->n) return record_error(STRM_EINVAL, "null ensemble or instance out of range");
  int rc = strm_set_inflow_df(E->ctx[e], df, profiles_host, buffer, bytes);
  if (rc) return rc;
  refresh_instance(E, e);
  return STRM_OK;
}

int strm_ensemble_advance(strm_ensemble* E, double* const* w, double* const* r_old, int nsteps, double dt,
                          double cfl) {
  if (!E || !w || !r_old) return record_error(STRM_EINVAL, "null ensemble or state table");
  if (nsteps < 0) return record_error(STRM_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) && !(cfl > 0.0)) return record_error(STRM_EINVAL, "need dt > 0 or cfl > 0");
  for (const Inst& I : E->inst_host)
    if ((I.C.bc[0] == kBcPeriodic) != (I.C.bc[1] == kBcPeriodic) ||
        (I.C.bc[2] == kBcPeriodic) != (I.C.bc[3] == kBcPeriodic))
      return record_error(STRM_EINVAL, "an instance has a periodic face opposite a non-periodic one");
  int rc = bind_states(E, w, r_old);
  if (rc) return rc;
  if (nsteps == 0) return STRM_OK;
  if (!E->gexec || E->g_cfl != cfl || E->g_dt != dt) {
    if (E->gexec) {
      STRME_CK(cudaGraphExecDestroy(E->gexec));
      E->gexec = nullptr;
    }
    if (!E->cap) STRME_CK(cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking));
    STRME_CK(cudaStreamBeginCapture(E->cap, cudaStreamCaptureModeThreadLocal));
    int erc = enqueue_step(E, dt, cfl, E->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(E->cap, &graph);
    if (erc) {
      if (graph) cudaGraphDestroy(graph);
      return erc;
    }
    if (e != cudaSuccess) return record_error(STRM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&E->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return record_error(STRM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    E->g_cfl = cfl;
    E->g_dt = dt;
  }
  for (int s = 0; s < nsteps; ++s) STRME_CK(cudaGraphLaunch(E->gexec, E->stream));
  return STRM_OK;
}

int strm_ensemble_set_barrier_limit(strm_ensemble* E, double seconds) {
  if (!E || !(seconds >= 0.0) || seconds > 3600.0) return record_error(STRM_EINVAL, "null ensemble or limit outside [0, 3600] s");
  E->barrier_ns = (unsigned long long)(seconds * 1e9);
  if (E->gexec) {  // the captured graph holds the old limit
    cudaGraphExecDestroy(E->gexec);
    E->gexec = nullptr;
  }
  return STRM_OK;
}

int strm_ensemble_set_schedule(strm_ensemble* E, const int* choice) {
  if (!E || !choice) return record_error(STRM_EINVAL, "null ensemble or schedule");
  return set_schedule(E, choice);
}

int strm_ensemble_tune(strm_ensemble* E, double* const* w, double* const* r_old, int* choice_host) {
  if (!E || !w || !r_old) return record_error(STRM_EINVAL, "null ensemble or state table");
  int rc = bind_states(E, w, r_old);
  if (rc) return rc;
  cudaEvent_t a, b;
  STRME_CK(cudaEventCreate(&a));
  STRME_CK(cudaEventCreate(&b));
  auto time_rhs = [&](float* best_ms) -> int {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(a, E->stream);
      enqueue_rhs(E, false, 0.0, 0.0, E->stream);
      cudaEventRecord(b, E->stream);
      cudaError_t e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) return record_error(STRM_ECUDA, std::string("tune: ") + cudaGetErrorString(e));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      best = std::min(best, ms);
    }
    *best_ms = best;
    return STRM_OK;
  };
  // 1. launch shapes of the per-kernel-type schedule: WENO (the dominant kernel), then the
  //    central-list grid
  E->tune.persistent = 0;
  Tuning bestT = E->tune;
  float best = 1e30f;
  const int blocks[3] = {32, 64, 128}, per_sm[3] = {4, 8, 16};  // kb_weno takes <= 128 threads
  for (int bi = 0; bi < 3 && rc == STRM_OK; ++bi)
    for (int gi = 0; gi < 3 && rc == STRM_OK; ++gi) {
      E->tune.weno_block = blocks[bi];
      E->tune.weno_per_sm = per_sm[gi];
      float ms;
      rc = time_rhs(&ms);
      if (rc == STRM_OK && ms < best) {
        best = ms;
        bestT = E->tune;
      }
    }
  E->tune = bestT;
  const int cper[3] = {8, 16, 32};
  for (int ci = 0; ci < 3 && rc == STRM_OK; ++ci) {
    E->tune.central_per_sm = cper[ci];
    float ms;
    rc = time_rhs(&ms);
    if (rc == STRM_OK && ms < best) {
      best = ms;
      bestT = E->tune;
    }
  }
  E->tune = bestT;
  // 2. schedule: the persistent stage (one cooperative launch) against the per-kernel launches
  if (rc == STRM_OK && E->stage_grid > 0 && !any_df(E)) {
    E->tune.persistent = 1;
    float ms;
    // a launch the device refuses (a configuration error, which does not persist) leaves the
    // persistent schedule out of the choice
    if (time_rhs(&ms) == STRM_OK && ms < best) {
      best = ms;
      bestT = E->tune;
    }
    E->tune = bestT;
  }
  // 3. pencil tile of the slab traversal (assembly and z faces): slab height cap
  const int caps[4] = {32, 16, 8, 0};
  for (int ci = 0; ci < 4 && rc == STRM_OK; ++ci) {
    apply_slab_cap(E, caps[ci]);
    rc = upload_table(E);
    float ms;
    if (rc == STRM_OK) rc = time_rhs(&ms);
    if (rc == STRM_OK && ms < best) {
      best = ms;
      bestT = E->tune;
    }
  }
  E->tune = bestT;
  apply_slab_cap(E, bestT.slab_cap);
  if (rc == STRM_OK) rc = upload_table(E);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (E->gexec) {  // the captured graph holds the old launch shapes
    cudaGraphExecDestroy(E->gexec);
    E->gexec = nullptr;
  }
  if (choice_host) get_schedule(E, choice_host);
  return rc;
}

int strm_ensemble_totals(strm_ensemble* E, double* const* w, double* out_host) {
  if (!E || !w || !out_host) return record_error(STRM_EINVAL, "null argument");
  for (int e = 0; e < E->n; ++e) {
    int rc = strm_conserved_totals(E->ctx[e], w[e], out_host + 5 * e);
    if (rc) return rc;
  }
  return STRM_OK;
}

int strm_ensemble_times(strm_ensemble* E, double* t_host) {
  if (!E || !t_host) return record_error(STRM_EINVAL, "null argument");
  for (int e = 0; e < E->n; ++e) {
    int rc = strm_get_time(E->ctx[e], &t_host[e], nullptr);
    if (rc) return rc;
  }
  return STRM_OK;
}

void strm_ensemble_destroy(strm_ensemble* E) {
  if (!E) return;
  if (E->gexec) cudaGraphExecDestroy(E->gexec);
  if (E->cap) cudaStreamDestroy(E->cap);
  for (strm_ctx* c : E->ctx) strm_destroy(c);
  delete E;
}

}  // extern "C"
