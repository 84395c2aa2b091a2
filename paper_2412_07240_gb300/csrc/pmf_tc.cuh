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
  int fft;            // 2-D: Hartley transforms in shared memory (tc2_form)
};

// Resident description of one filter of a batch (device memory).
struct FilterSlot {
  DevState* st;
  float* buf0;
  float* buf1;
  const uint8_t* hart[2];   // split Hartley planes per axis
  const float* sctab[2];    // (cos, sin)(pi m / N) tables per axis
  int N0, N1;
  const MeasParams* mp;     // measurement model of the filter
  const TimeConsts* tc;     // constants of the filter's current tau
  void* plan;               // batched epochs: the front kernel's results (tc_plan_bytes)
  int fft;                  // 1: Hartley transforms in shared memory (tc2_form), 0: GEMMs
};

// One filter's request in a batched epoch: flags bit 0 = measurement update
// with z, bit 1 = time update with the slot's constants.
struct StepItem {
  int slot;
  int flags;
  double z[PMF_MAX_NZ];
};

// Resident description of one 1-D filter (device memory).
struct Slot1 {
  DevState* st;
  float* buf0;
  float* buf1;
  const float* tab;         // cas(2 pi r / N), r < N, then (cos, sin)(pi m / N), m = -N..N
  int N;
  const MeasParams* mp;
  const TimeConsts* tc;
  int mode;                 // Hartley transforms: 0 matrix-vector, 1 shared-memory FFT
};

// PMF_OK if the fused kernel can hold this grid at this precision.
int tc_supported(const pmf_config* cfg, std::string* why);
int tc_build_tables(const pmf_config* cfg, TcTables* t, std::string* why);
// Split Hartley planes and the (cos, sin)(pi m / N) table of one axis size (one allocation).
// cls: size class of the kernels that read it (128: every fused kernel; 64:
// the compact planned kernel of batched filters whose axes are all <= 64).
int tc_build_axis_table(int N, int precision, void** dev, size_t* hart_bytes, int cls = 128);
size_t tc_axis_table_bytes(int N, int precision, int cls = 128);
// Form of the Hartley transforms of a 2-D filter: 0 the tensor-core GEMMs,
// 1 the shared-memory FFT (axis sizes 2^a 3^b, not with BF16X6, whose
// operand planes fill the scratch the FFT form needs).  TRANSFORM_AUTO times
// both on a scratch filter the first time a (N0, N1, precision) is used and
// caches the choice in autotune_2d.json beside the library (the environment
// variable PMF_2D_FORM=fft|gemm overrides it).
bool tc2_fft_ok(int N0, int N1, int precision);
int tc2_form(const pmf_config* cfg, cudaStream_t s);
// Size class of a 2-D filter in batched epochs: the largest axis rounded up
// to 64, 96 or 128.
inline int tc_class(int N0, int N1) {
  const int m = N0 > N1 ? N0 : N1;
  return m <= 64 ? 64 : m <= 96 ? 96 : 128;
}
// ... for a filter in the given transform form: the size-96 class keeps its
// staging tile in the W region, which the FFT form needs as scratch, so an
// FFT-form filter of that class runs in the size-128 class (the precision
// does not change the class: BF16X6 has no FFT form).
inline int tc_class_form(int N0, int N1, int fft, int precision) {
  (void)precision;
  const int c = tc_class(N0, N1);
  return fft && c == 96 ? 128 : c;
}
// Device bytes of one filter's plan (the front kernel's results of an epoch).
size_t tc_plan_bytes();
void tc_free_tables(TcTables* t);
// Bounded mbarrier wait in a one-warp kernel (see pmf_selftest_bounded_wait).
int tc_wait_probe(long long polls, int arrive, cudaStream_t s);
// Prior weights and their moments; returns the number of kernel launches.
int tc_prior(const Dims& d, DevState* st, const double* prior_aux, float* X, double* partials,
             cudaStream_t s);
// One fused launch: measurement update (if mp) then time update (if tc).
int tc_step(const Dims& d, const pmf_config& cfg, const TcTables* t, const MeasParams* mp,
            const TimeConsts* tc, DevState* st, float* b0, float* b1, cudaStream_t s);

// 3-D grids (pmf_tc3.cu): per-filter device state (tc3_alloc) and epochs of
// one or many filters, every stage one launch over all of them.
int tc3_alloc(void** handle);
size_t tc3_state_bytes();   // device bytes one tc3_alloc holds
void tc3_free(void* handle);
int tc3_step(void* handle, const Dims& d, const pmf_config& cfg, const TcTables* t, const MeasParams* mp,
             const TimeConsts* tcs, DevState* st, float* b0, float* b1, cudaStream_t s);

// One filter's epoch in a batched 3-D launch sequence (mp / tc null: no
// measurement / time update); host structs are copied at the call.
struct Tc3Item {
  void* handle;             // tc3_alloc state of the filter
  Dims d;
  const TcTables* t;
  const MeasParams* mp;
  const TimeConsts* tc;
  DevState* st;
  float* b0;
  float* b1;
};
// Pinned and device staging of the per-filter descriptors of one sequence;
// reserve waits for the previous sequence's copies from it.
struct Tc3Stage {
  void* h_jobs;
  int* h_first;
  void* d_jobs;
  int* d_first;
  int cap;
  cudaEvent_t ev;
};
int tc3_stage_reserve(Tc3Stage* g, int n);
void tc3_stage_free(Tc3Stage* g);
// Launches the sequence for items[0..n) on stream s; returns the number of
// launches, or minus a PMF_ERR_* code.
int tc3_batch(const Tc3Item* items, int n, int precision, Tc3Stage* g, cudaStream_t s);

// A batched epoch as a front kernel over all k items, then the planned
// transform kernels: items [0, k128) of size class 128, [k128, k128 + k96) of
// class 96, the rest of class 64 (the last two on stream s2 when it is given,
// joined back into s through the events, so the classes share the SMs).  tcs
// (if not null, in device memory) holds each item's time-update constants in
// place of the slot's.  Returns the number of launches.
int tc_batch_epoch(int precision, const FilterSlot* slots, const StepItem* items, int k, int k128, int k96,
                   cudaStream_t s, const TimeConsts* tcs = nullptr, cudaStream_t s2 = nullptr,
                   cudaEvent_t ev_fork = nullptr, cudaEvent_t ev_join = nullptr);

// 1-D grids (pmf_tc1.cu): CUDA-core kernel, N a multiple of 8 in [16, 512].
int tc1_supported(const pmf_config* cfg, std::string* why);
size_t tc1_table_bytes(int N);
int tc1_build_table(int N, void** dev);
int tc1_step(int N, const void* table, const MeasParams* mp, const TimeConsts* tc, DevState* st, float* b0,
             float* b1, cudaStream_t s, int mode);
// Transform form for size N chosen by timing both on a scratch filter (once
// per N and process; cached in autotune.json beside the library).  The
// environment variable PMF_1D_FORM=fft|matvec overrides the choice.
// Transform form of a 1-D filter: the config's choice, or tc1_mode for AUTO.
int tc1_form(const pmf_config* cfg, const void* table, cudaStream_t s);
int tc1_mode(int N, const void* table, cudaStream_t s);
int tc1_batch_step(const Slot1* slots, const StepItem* items, const TimeConsts* tcs, int k, cudaStream_t s);
// {mean[2], cov[4], status, 0} of filters ids[0..k) into out (8 doubles each),
// then their status words cleared; returns the number of launches.
int tc_batch_gather(DevState* st, const int* ids, int k, double* out, cudaStream_t s);

}  // namespace pmf
