// Float32 path for n_x = 4 grids (pmf_f4.cu): tables, scratch and launchers.
#pragma once

#include <string>

#include "pmf_internal.cuh"

namespace pmf {

struct F4Tables {
  double2* mtab = nullptr;     // terrain waves: per-axis phase tables (4 waves x 4 axes x 64)
  float* lo = nullptr;         // per point: smaller mixture exponent (or the exponent)
  float* gap = nullptr;        // per point: gap to the other mixture exponent
  double* hfwd[4] = {};        // per axis: forward Hartley matrix / N (float64)
  float* wfwd[4] = {};         // per axis: (H I)^T, columns padded to a multiple of 8
  float* winv[4] = {};         // per axis: H^T (inverse transform), padded likewise
  double* shear = nullptr;     // band-limited re-alignment: pass coefficients (shear4_setup layout)
};

// PMF_OK if the float32 4-D kernels can hold this grid.
int f4_supported(const pmf_config* cfg, std::string* why);
int f4_alloc(const pmf_config* cfg, F4Tables* t);
void f4_free(F4Tables* t);
// Measurement and time update; each returns its number of kernel launches.
int f4_meas(const Dims& d, const MeasParams& mp, DevState* st, const F4Tables& t, float* b0, float* b1,
            double* partials, cudaStream_t s);
int f4_time(const Dims& d, const TimeConsts& tc, DevState* st, const F4Tables& t, float* b0, float* b1,
            double* partials, double* pend, cudaStream_t s);

}  // namespace pmf
