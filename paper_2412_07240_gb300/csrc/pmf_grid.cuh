// Device helpers shared by the kernels that walk a whole grid (the float64
// path and the float32 n_x = 4 path): index unflattening, the measurement
// exponent in float64, block sums and the moment accumulators.
#pragma once

#include <cmath>

#include "pmf_internal.cuh"

namespace pmf {

__device__ __forceinline__ void unflatten(const Dims& d, long long p, int* j) {
  for (int m = d.nx - 1; m >= 0; --m) {
    j[m] = (int)(p % d.N[m]);
    p /= d.N[m];
  }
}

__device__ __forceinline__ double wrap_pi(double r) {
  const double two_pi = 6.283185307179586476925286766559;
  const double pi = 3.14159265358979323846264338327950;
  return r - two_pi * ceil((r - pi) / two_pi);
}

// e(x) = 1/2 r^T R^{-1} r with r = z - h(x) (eq. meas).
__device__ inline double meas_exponent_f64(const MeasParams& mp, const double* x) {
  double r[PMF_MAX_NZ];
  if (mp.kind == PMF_MEAS_LINEAR) {
    for (int i = 0; i < mp.nz; ++i) {
      double h = 0.0;
      for (int a = 0; a < mp.nx; ++a) h += mp.H[i * mp.nx + a] * x[a];
      r[i] = mp.z[i] - h;
    }
  } else if (mp.kind == PMF_MEAS_RANGE) {
    r[0] = mp.z[0] - sqrt(x[0] * x[0] + x[1] * x[1]);
  } else if (mp.kind == PMF_MEAS_TERRAIN_GM) {
    // terrain altitude at (p_x, p_y) = (x_0, x_2); -log of the two-component
    // Gaussian mixture of the residual (constants from the host: gm = {1/(2 v1),
    // 1/(2 v2), log terms c1, c2, means mu1, mu2}), in log-sum-exp form
    double h = mp.p[16];
    for (int i = 0; i < 4; ++i) h += mp.p[4 * i] * sin(mp.p[4 * i + 1] * x[0] + mp.p[4 * i + 2] * x[2] + mp.p[4 * i + 3]);
    const double rr = mp.z[0] - h;
    const double m1 = (rr - mp.gm[4]) * (rr - mp.gm[4]) * mp.gm[0] + mp.gm[2];
    const double m2 = (rr - mp.gm[5]) * (rr - mp.gm[5]) * mp.gm[1] + mp.gm[3];
    const double lo = fmin(m1, m2);
    return lo - log1p(exp(-fabs(m1 - m2)));
  } else {
    r[0] = wrap_pi(mp.z[0] - atan2(x[1], x[0]));
    r[1] = mp.z[1] - x[2];
  }
  double e = 0.0;
  for (int i = 0; i < mp.nz; ++i)
    for (int k = 0; k < mp.nz; ++k) e += r[i] * mp.Rinv[i * mp.nz + k] * r[k];
  return 0.5 * e;
}

template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* smem /* [32*NV] */, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < nw ? smem[lane * NV + i] : 0.0;
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) out[i] = t;
    }
  }
}

// Moment accumulators in frame coordinates u: S0, S1[n], S2 (layout of tot_S2).
__device__ __forceinline__ void acc_moments(double* acc, double p, const double* u, int nx) {
  acc[0] += p;
  for (int a = 0; a < nx; ++a) acc[1 + a] += p * u[a];
  for (int a = 0; a < nx; ++a)
    for (int b = a; b < nx; ++b) acc[tot_S2(nx, a, b)] += p * u[a] * u[b];
}

}  // namespace pmf
