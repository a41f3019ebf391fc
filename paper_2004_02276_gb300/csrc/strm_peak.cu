// FMA issue-rate probe (strm_peak_fma in include/strm.h): the denominator of the ALU roofline
// the benchmark reports. On GB300 the FP64 pipe executes two DFMA per clock per SM against 128
// FP32 FMA, and every FP64 kernel of the right-hand side is bound by that pipe, so the roofline
// of the path is an FMA rate, measured here on the GPU at hand rather than taken from a table.
//
// Each thread runs kChains independent FMA chains x <- x * a + b (a, b runtime values, |a| < 1,
// so the chains stay bounded and the compiler can neither fold nor shorten them); enough
// resident warps and chains hide the FMA latency, so the kernel runs at the pipe's issue rate.
// Flops = 2 per FMA. The result is stored only when the runtime flag asks for it, which the
// compiler cannot know, so no chain is removed as dead code.
#include <string>

#include "../../include/strm.h"
#include "strm_launch.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;

static __device__ double g_peak_sink[2];

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(T a, T b, int iters, int store) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (store) g_peak_sink[sizeof(T) == 8 ? 0 : 1] = (double)s;
}

int peak_fail(int code, const std::string& msg) { return strm::record_error(code, msg); }

#define PEAK_CK(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      if (t0) cudaEventDestroy(t0);                                                       \
      if (t1) cudaEventDestroy(t1);                                                       \
      return peak_fail(STRM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    }                                                                                     \
  } while (0)

}  // namespace

extern "C" int strm_peak_fma(int precision, int launches, void* stream, double* tflops_host,
                             double* ms_host) {
  if (precision != STRM_PREC_FP64 && precision != STRM_PREC_MIXED)
    return peak_fail(STRM_EINVAL, "precision must be STRM_PREC_FP64 or STRM_PREC_MIXED (FP32)");
  if (launches < 1 || launches > 1000) return peak_fail(STRM_EINVAL, "launches must be in 1..1000");
  if (!tflops_host) return peak_fail(STRM_EINVAL, "null output");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  int dev = 0, sms = 0;
  PEAK_CK(cudaGetDevice(&dev));
  PEAK_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = precision == STRM_PREC_FP64;
  // about 40 ms per launch at the nominal rates (1.25 TFLOP/s FP64, 80 TFLOP/s FP32)
  const long long threads = (long long)sms * kPeakBlocksPerSm * kPeakThreads;
  const double target_flops = (fp64 ? 1.25e12 : 80e12) * 0.04;
  int iters = (int)(target_flops / (2.0 * kChains * (double)threads));
  if (iters < 16) iters = 16;
  const unsigned grid = (unsigned)(sms * kPeakBlocksPerSm);
  PEAK_CK(cudaEventCreate(&t0));
  PEAK_CK(cudaEventCreate(&t1));
  double best_ms = 0.0;
  for (int l = -1; l < launches; ++l) {  // l = -1: untimed warm-up launch
    PEAK_CK(cudaEventRecord(t0, st));
    if (fp64) k_fma_chains<double><<<grid, kPeakThreads, 0, st>>>(0.999999, 1e-7, iters, 0);
    else k_fma_chains<float><<<grid, kPeakThreads, 0, st>>>(0.999f, 1e-4f, iters, 0);
    PEAK_CK(cudaGetLastError());
    PEAK_CK(cudaEventRecord(t1, st));
    PEAK_CK(cudaEventSynchronize(t1));
    float ms = 0.f;
    PEAK_CK(cudaEventElapsedTime(&ms, t0, t1));
    if (l >= 0 && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  const double flops = 2.0 * kChains * (double)iters * (double)threads;
  *tflops_host = flops / (best_ms * 1e-3) / 1e12;
  if (ms_host) *ms_host = best_ms;
  return STRM_OK;
}
