// Fused tensor-core path of libpmf (pmf_tc.cu): host-side interface.
#pragma once

#include <string>

#include "pmf_internal.cuh"

namespace pmf {

// Device tables of the fused kernel (per context).
struct TcTables {
  void* hart[MAXN];   // split Hartley matrices per axis, canonical smem layout
  size_t hart_bytes[MAXN];
  int prec;
};

// PMF_OK if the fused kernel can hold this grid at this precision.
int tc_supported(const pmf_config* cfg, std::string* why);
int tc_build_tables(const pmf_config* cfg, TcTables* t, std::string* why);
void tc_free_tables(TcTables* t);
// Prior weights and their moments; returns the number of kernel launches.
int tc_prior(const Dims& d, DevState* st, const double* prior_aux, float* X, double* partials,
             cudaStream_t s);
// One fused launch: measurement update (if mp) then time update (if tc).
int tc_step(const Dims& d, const pmf_config& cfg, const TcTables* t, const MeasParams* mp,
            const TimeConsts* tc, DevState* st, float* b0, float* b1, cudaStream_t s);

}  // namespace pmf
