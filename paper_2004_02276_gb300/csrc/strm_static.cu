// Conserved totals without any allocation (strm_conserved_totals_static in include/strm.h).
//
// This variant exists for callers that cannot allocate device memory, for example an in-situ
// monitor attached to a solver that already holds all device memory in its own caching
// allocator, or code running where calling cudaMalloc is not permitted. It needs neither a
// context nor a workspace: its scratch (per-block partial sums and the five results) is the
// file-scope array below, which every GPU that loads this library keeps until the process exits.
#include <cmath>
#include <string>

#include "../../include/strm.h"
#include "strm_dev.cuh"
#include "strm_launch.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticNodesPerThread = 16;
constexpr long long kStaticNodesPerBlock = (long long)kStaticThreads * kStaticNodesPerThread;
constexpr int kStaticMaxBlocks = STRM_STATIC_MAX_NODES / (kStaticThreads * kStaticNodesPerThread);
// partial sums [5][kStaticMaxBlocks], then the five totals
constexpr int kStaticDoubles = 5 * kStaticMaxBlocks + 8;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

int static_fail(int code, const std::string& msg) { return strm::record_error(code, msg); }

// Device address of g_static_scratch in the current context. In host code the array's name is
// only a host-side stand-in, so kernels get this address instead. It is looked up on every call
// (cheap next to the call's synchronisation): an address cached per device could outlive the
// module after a device reset or a released primary context.
cudaError_t static_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = (double*)p;
  return cudaSuccess;
}

struct StaticGrid {
  int nx, ny, nz, y_map;
  double beta, ly, deta, dxdz;
};

// Node volume dx (y_eta deta) dz of row j, with y_eta of the wall-normal map (the maps of
// include/strm.h, as the context's metrics take them).
__device__ __forceinline__ double static_volume(const StaticGrid& g, int j) {
  const double eta = (j + 0.5) * g.deta, b = g.beta;
  double ye;
  if (g.y_map == STRM_MAP_TANH) {
    // y = (ly/2) tanh(b (2 eta - 1)) / tanh(b)
    double A = 0.5 * g.ly / tanh(b);
    double th = tanh(b * (2.0 * eta - 1.0));
    ye = 2.0 * b * A * (1.0 - th * th);
  } else if (g.y_map == STRM_MAP_TANH_ONESIDED) {
    // y = ly (1 - tanh(b (1 - eta)) / tanh(b))
    double A = g.ly / tanh(b);
    double th = tanh(b * (1.0 - eta));
    ye = A * b * (1.0 - th * th);
  } else if (g.y_map == STRM_MAP_ERF) {
    // y = (ly/2) erf(b (2 eta - 1)) / erf(b)
    double sv = 2.0 * eta - 1.0;
    ye = 2.0 * g.ly * b / (sqrt(acos(-1.0)) * erf(b)) * exp(-b * b * sv * sv);
  } else if (g.y_map == STRM_MAP_SINH_ONESIDED) {
    // y = ly sinh(b eta) / sinh(b)
    ye = g.ly * b * cosh(b * eta) / sinh(b);
  } else {
    ye = g.ly;
  }
  return g.dxdz * (ye * g.deta);
}

__global__ void __launch_bounds__(kStaticThreads) k_static_partial(StaticGrid g, const double* __restrict__ w,
                                                                   double* scratch, int nblocks) {
  __shared__ double sh[32];
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long base = (long long)blockIdx.x * kStaticNodesPerBlock;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = 0; t < kStaticNodesPerThread; ++t) {
    long long q = base + (long long)t * kStaticThreads + threadIdx.x;
    if (q < N) {
      double v = static_volume(g, (int)((q / g.nx) % g.ny));
#pragma unroll
      for (int m = 0; m < 5; ++m) acc[m] += w[m * N + q] * v;
    }
  }
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    double s = strm::block_sum(acc[m], sh);
    if (threadIdx.x == 0) scratch[(long long)m * kStaticMaxBlocks + blockIdx.x] = s;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_static_finalize(double* scratch, int nblocks) {
  __shared__ double sh[32];
  for (int m = 0; m < 5; ++m) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[(long long)m * kStaticMaxBlocks + b];
    s = strm::block_sum(s, sh);
    if (threadIdx.x == 0) scratch[5 * kStaticMaxBlocks + m] = s;
    __syncthreads();
  }
}

}  // namespace

extern "C" int strm_conserved_totals_static(const strm_grid* g, const double* w, double out_host[5],
                                            void* stream) {
  if (!g || !w || !out_host) return static_fail(STRM_EINVAL, "null argument");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0))
    return static_fail(STRM_EINVAL, "invalid grid: sizes and lengths must be positive");
  if (g->y_map < STRM_MAP_UNIFORM || g->y_map > STRM_MAP_SINH_ONESIDED)
    return static_fail(STRM_EINVAL, "invalid grid: unknown wall-normal map " + std::to_string(g->y_map));
  if (g->y_map != STRM_MAP_UNIFORM && !(g->beta > 0))
    return static_fail(STRM_EINVAL, "invalid grid: the wall-normal map needs beta > 0");
  long long N = (long long)g->nx * g->ny * g->nz;
  if (N > STRM_STATIC_MAX_NODES)
    return static_fail(STRM_EINVAL, "grid has " + std::to_string(N) + " nodes; the static scratch of "
                                     "strm_conserved_totals_static holds partial sums for at most " +
                                     std::to_string((long long)STRM_STATIC_MAX_NODES) + " nodes");
  double* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess)
    return static_fail(STRM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  StaticGrid sg;
  sg.nx = g->nx;
  sg.ny = g->ny;
  sg.nz = g->nz;
  sg.y_map = g->y_map;
  sg.beta = g->beta;
  sg.ly = g->ly;
  sg.deta = 1.0 / g->ny;
  sg.dxdz = (g->lx / g->nx) * (g->lz / g->nz);
  int nblocks = (int)((N + kStaticNodesPerBlock - 1) / kStaticNodesPerBlock);
  // the five result slots are cleared so a failed launch can never return an old total
  e = cudaMemsetAsync(scratch + 5 * kStaticMaxBlocks, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return static_fail(STRM_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
  k_static_partial<<<nblocks, kStaticThreads, 0, st>>>(sg, w, scratch, nblocks);
  k_static_finalize<<<1, 1024, 0, st>>>(scratch, nblocks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(STRM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(out_host, scratch + 5 * kStaticMaxBlocks, 5 * sizeof(double),
                      cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return static_fail(STRM_ECUDA, std::string("readback: ") + cudaGetErrorString(e));
  for (int m = 0; m < 5; ++m)
    if (!std::isfinite(out_host[m])) return static_fail(STRM_ENONFINITE, "non-finite conserved total");
  return STRM_OK;
}
