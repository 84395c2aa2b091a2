// Moments of a float64 weight array without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need the moments:
// hosts that own every byte of device memory through their own allocator and
// forbid libraries from allocating, and real-time loops that must not pay the
// latency or the failure mode of an allocation (cudaMalloc may synchronise
// the device and may fail under memory pressure).  pmf_moments_noalloc serves
// them: it is the block-partial-sum moment reduction of the float64 path with
// its partial sums in a fixed file-scope device array instead of a context's
// scratch buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "pmf.h"
#include "pmf_internal.cuh"

namespace {

using pmf::kMomentSlots;
using pmf::tot_S2;

constexpr int kThreads = 256;
constexpr int kMaxBlocks = PMF_NOALLOC_MAX_POINTS / kThreads;   // one partial per 256 points

// Shared by every call on a device, kept until the process exits; each call
// overwrites the partials of the blocks it launches before reading them.
__device__ __align__(256) double g_partials[kMaxBlocks * kMomentSlots];

constexpr int kMaxDevices = 64;
double* g_ptr[kMaxDevices] = {nullptr};
std::mutex g_mu;

// Device address of g_partials on the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

struct Geo {
  int nx;
  int N[PMF_MAX_NX];
  long long P;
  double c[PMF_MAX_NX];
  double M[PMF_MAX_NX * PMF_MAX_NX];
};

// One block per 256 consecutive points: S0, S1[n], S2 in frame coordinates u
// (the kMomentSlots layout of tot_S2).
__global__ void k_partials(Geo g, const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sm[kThreads / 32][kMomentSlots];
  double a[kMomentSlots] = {};
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p < g.P) {
    long long t = p;
    double u[PMF_MAX_NX] = {};
    for (int m = g.nx - 1; m >= 0; --m) {
      u[m] = (double)(t % g.N[m]) - 0.5 * (g.N[m] - 1);
      t /= g.N[m];
    }
    const double x = w[p];
    a[0] = x;
    for (int i = 0; i < g.nx; ++i) a[1 + i] = x * u[i];
    for (int i = 0; i < g.nx; ++i)
      for (int j = i; j < g.nx; ++j) a[tot_S2(g.nx, i, j)] = x * u[i] * u[j];
  }
  for (int i = 0; i < kMomentSlots; ++i)
    for (int o = 16; o; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < kMomentSlots; ++i) sm[threadIdx.x >> 5][i] = a[i];
  __syncthreads();
  if (threadIdx.x < kMomentSlots) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += sm[k][threadIdx.x];
    part[(size_t)blockIdx.x * kMomentSlots + threadIdx.x] = s;
  }
}

// Sum the partials and write {S0, mean[nx], cov[nx*nx]} (x = c + M u).
__global__ void k_finish(Geo g, const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double sm[kThreads / 32][kMomentSlots];
  __shared__ double tot[kMomentSlots];
  double a[kMomentSlots] = {};
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
    for (int i = 0; i < kMomentSlots; ++i) a[i] += part[(size_t)b * kMomentSlots + i];
  for (int i = 0; i < kMomentSlots; ++i)
    for (int o = 16; o; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < kMomentSlots; ++i) sm[threadIdx.x >> 5][i] = a[i];
  __syncthreads();
  if (threadIdx.x < kMomentSlots) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += sm[k][threadIdx.x];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int n = g.nx;
  const double S0 = tot[0];
  out[0] = S0;
  if (S0 == 0.0 || !isfinite(S0)) {
    // no mass (or a non-finite sum): the moments are undefined
    for (int i = 0; i < n + n * n; ++i) out[1 + i] = nan("");
    return;
  }
  double mu[4], S2[16], Cu[16], cov[16];
  for (int a2 = 0; a2 < n; ++a2) mu[a2] = tot[1 + a2] / S0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) S2[i * n + j] = tot[tot_S2(n, i, j)];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Cu[i * n + j] = S2[i * n + j] / S0 - mu[i] * mu[j];
  pmf::congruence(n, g.M, Cu, cov);
  for (int i = 0; i < n; ++i) {
    double m = g.c[i];
    for (int j = 0; j < n; ++j) m += g.M[i * n + j] * mu[j];
    out[1 + i] = m;
  }
  for (int i = 0; i < n * n; ++i) out[1 + n + i] = cov[i];
}

}  // namespace

extern "C" int pmf_moments_noalloc(const double* weights, int nx, const int* N, const double* c,
                                   const double* M, double* out, void* cuda_stream) {
  if (!weights || !N || !c || !M || !out || nx < 1 || nx > PMF_MAX_NX) return PMF_ERR_ARG;
  Geo g{};
  g.nx = nx;
  g.P = 1;
  for (int m = 0; m < nx; ++m) {
    if (N[m] < 1) return PMF_ERR_ARG;
    g.N[m] = N[m];
    g.P *= N[m];   // at most 2^20 * (2^31 - 1): no overflow before the check below
    if (g.P > PMF_NOALLOC_MAX_POINTS) return PMF_ERR_ARG;
    g.c[m] = c[m];
  }
  for (int i = 0; i < nx * nx; ++i) g.M[i] = M[i];
  double* part = nullptr;
  if (scratch_for_current_device(&part) != cudaSuccess) return PMF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nb = (int)((g.P + kThreads - 1) / kThreads);
  k_partials<<<nb, kThreads, 0, s>>>(g, weights, part);
  k_finish<<<1, kThreads, 0, s>>>(g, part, nb, out);
  return cudaGetLastError() == cudaSuccess ? PMF_OK : PMF_ERR_CUDA;
}
