// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "strm_dev.cuh"

namespace strm {

// Set the thread-local message returned by strm_last_error and return code.
int record_error(int code, const std::string& msg);

}  // namespace strm

struct strm_ctx;

namespace strm {

// The grid, constants and workspace buffers of a context, and the SM count it launches for.
void ctx_parts(strm_ctx* x, Dims* d, Consts* C, Bufs* B, int* sms);

int reduce_blocks(const Dims& d);
void launch_prims(const Dims& d, const Consts& C, const Bufs& B, const double* w, bool want_cfl,
                  cudaStream_t s);
void launch_dt_finalize(const Dims& d, const Bufs& B, double cfl, double dt_fixed, cudaStream_t s);
void launch_ghost_prims(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s);
void launch_recycle(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s);
// digital-filter inflow: filter half-widths (grid points), integral time, seed, and the device
// arrays of the caller's inflow buffer (filter coefficients, y-filtered plane, Psi, draw counter)
struct DFParams {
  int ny, nz;
  double tau;
  unsigned long long seed;
  const double* by;
  const double* bz;
  double* t;
  double* psi;
  unsigned long long* count;
};
// draw and filter one plane and blend it into Psi (first: Psi = the plane)
void launch_df_update(const Dims& d, const DFParams& F, const Bufs& B, bool first, cudaStream_t s);
// the digital-filter inflow of a context, if its x-min face has one
bool ctx_df(strm_ctx* x, DFParams* F);
// one statistics sample of w: mode 0 adds x-z means to acc[24][ny] (scr holds [24][ny][nx]
// column sums), mode 1 adds z means to acc[24][ny][nx]
void launch_stats(const Dims& d, const Consts& C, const double* w, double* acc, double* scr, int mode,
                  cudaStream_t s);
// Ducros sensor over region 0 (all interior nodes), 1 (the nodes whose stencils read no ghost:
// sensor_inner_nodes of them) or 2 (the others)
long long sensor_inner_nodes(const Dims& d, int L);
void launch_sensor(const Dims& d, const Consts& C, const Bufs& B, int region, cudaStream_t s);
// mixed precision: FP64 theta at the nodes the sensor listed as near the switch threshold
void launch_band_theta(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s);
void launch_ghost_scalars(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s);
// prescribed switch input: the FP64 sensor field at the interior nodes from theta[N]
void launch_theta_set(const Dims& d, const Bufs& B, const double* theta, cudaStream_t s);
// returns the number of kernels launched
int launch_faces_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s);
void launch_weno_dir(const Dims& d, const Consts& C, const Bufs& B, int dir, int grid, cudaStream_t s);
// residual into R, or (rk.w set) the RK stage update of w and r_old without writing R
void launch_assemble(const Dims& d, const Consts& C, const Bufs& B, double* R, const RkFuse& rk,
                     cudaStream_t s);
void launch_force_finalize(const Dims& d, const Consts& C, const Bufs& B, cudaStream_t s);
// stage update s of Eq. RK with the weights k_dt_finalize stored for this step
void launch_rk_update(const Dims& d, const Consts& C, const Bufs& B, double* w, double* r_old,
                      int stage, cudaStream_t s);
void launch_apply_forcing(const Dims& d, const Bufs& B, double* rhs, cudaStream_t s);
void launch_totals(const Dims& d, const Bufs& B, const double* w, cudaStream_t s);
void launch_flags(const Dims& d, const Consts& C, const Bufs& B, int dir, unsigned char* out,
                  cudaStream_t s);
// elementwise d2f / f2d over n elements
void launch_d2f(const double* x, float* y, long long n, cudaStream_t s);
void launch_f2d(const float* x, double* y, long long n, cudaStream_t s);
// copy n doubles between device memory and a mapped page-locked host buffer (16-byte aligned)
void launch_copy_mapped(const double* src, double* dst, long long n, int sms, cudaStream_t s);
void launch_export_sensor(const Dims& d, const Consts& C, const Bufs& B, double* theta, double* div,
                          cudaStream_t s);

}  // namespace strm
