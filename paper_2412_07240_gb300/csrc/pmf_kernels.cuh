// Launchers of libpmf's kernels (host side).
#pragma once

#include "pmf_internal.cuh"

namespace pmf {

// ---- plain float64 path (pmf_fp64.cu) -----------------------------------
int fp64_partials_blocks(const Dims& d);
void launch_prior_f64(const Dims& d, const DevState* st, const double* P0inv, const double* m0,
                      double* X, cudaStream_t s);
void launch_moments_f64(const Dims& d, DevState* st, int stage, double* b0, double* b1,
                        double* partials, int flip, int use_pending, const double* pend,
                        cudaStream_t s);
void launch_moments_f32(const Dims& d, DevState* st, const float* X, double* partials,
                        cudaStream_t s);
void launch_meas_f64(const Dims& d, const MeasParams& mp, DevState* st, double* b0, double* b1,
                     double* partials, cudaStream_t s);
void launch_time_f64(const Dims& d, const TimeConsts& tc, DevState* st, double* b0, double* b1,
                     double* partials, double* pend, double* const* interp,
                     double* const* hfwd, double* const* hinv, double* scratch, cudaStream_t s);
void launch_export_f64(const Dims& d, const DevState* st, const double* b0, const double* b1,
                       double* out, cudaStream_t s);

// Shared with the float32 n_x = 4 path: the frame kernel (regrid decision,
// sub-step coefficients).
void launch_frame(const TimeConsts& tc, DevState* st, double* pend, cudaStream_t s);

// Launch counts of the launchers above (per call).
constexpr int kLaunchesMeasF64 = 3;   // emin, apply, finalize (+1 memset)
inline int launches_time_f64(int nx) { return 1 + nx + 1 + 3 * nx + 1 + 2; }

}  // namespace pmf
