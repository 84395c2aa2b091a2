// Finite-difference comparator of the paper (Sec. III-B, III-C) on the GPU.
//
// One-dimensional model dx = a x dt + q dw on N interior nodes with zero
// (Dirichlet) boundary values; the explicit central-difference scheme of
// eq. fdiff, tridiag(a_t, b_t, a_t) with a_t = q dt / (2 delta^2) and
// b_t = 1 - q dt / delta^2 - dt a, applied l times while the spacing moves as
// delta_n = e^{a dt} delta_{n-1} (eq. gridMov).  All factors share the
// eigenvectors r^(j) = sin(i j pi / (N+1)), so the product is applied in the
// sine-transform form of eq. FST:
//   P' = 2/(N+1) R diag(prod_n lambda_n) R P,
//   lambda_n^(j) = b_t + 2 a_t cos(j pi / (N+1)) at spacing delta_n,
// i.e. two DST-I matrix products (float64) with the eigenvalue product fused
// into the first one's epilogue.
#include <cmath>
#include <vector>

#include "pmf.h"

namespace {

// Y[g][k] = s[k] * sum_i X[g][i] R[k][i] with R[k][i] = sin((k+1)(i+1) pi / (N+1))
// taken from tab[m] = sin(m pi / (N+1)), m = (k+1)(i+1) mod 2(N+1).
__global__ void k_dst_f64(const double* __restrict__ X, const double* __restrict__ tab,
                          const double* __restrict__ s, double* __restrict__ Y, int N, int count) {
  __shared__ double Xs[16][17];
  __shared__ double Rs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int g = blockIdx.y * 16 + ty;   // grid (row of X)
  const int k = blockIdx.x * 16 + tx;   // output node
  const int period = 2 * (N + 1);
  double acc = 0.0;
  for (int i0 = 0; i0 < N; i0 += 16) {
    Xs[ty][tx] = (g < count && i0 + tx < N) ? X[(size_t)g * N + i0 + tx] : 0.0;
    const int kk = blockIdx.x * 16 + ty, ii = i0 + tx;
    Rs[ty][tx] = (kk < N && ii < N) ? tab[(int)(((long long)(kk + 1) * (ii + 1)) % period)] : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(Xs[ty][t], Rs[tx][t], acc);
    __syncthreads();
  }
  if (g < count && k < N) Y[(size_t)g * N + k] = s[k] * acc;
}

}  // namespace

extern "C" int pmf_fdm_transition(const double* P_in, double* P_out, double* work, int N, int count, double q,
                                  double a, double dt, int l, double delta0, void* cuda_stream) {
  if (!P_in || !P_out || !work || N < 1 || N > (1 << 20) || count < 1 || l < 0 || !(delta0 > 0.0) ||
      !std::isfinite(q) || !std::isfinite(a) || !std::isfinite(dt) || P_in == P_out)
    return PMF_ERR_ARG;
  // host: sine table, eigenvalue product times 2/(N+1) split over the two products
  const size_t nY = (size_t)count * N;
  std::vector<double> h(2 * (N + 1) + 2 * N);
  double* tab = h.data();
  double* lam = tab + 2 * (N + 1);
  double* ones = lam + N;
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < 2 * (N + 1); ++m) tab[m] = std::sin(m * pi / (N + 1));
  for (int j = 0; j < N; ++j) {
    lam[j] = 2.0 / (N + 1);
    ones[j] = 1.0;
  }
  double delta = delta0;
  for (int n = 0; n < l; ++n) {
    const double at = q * dt / (2.0 * delta * delta), bt = 1.0 - q * dt / (delta * delta) - dt * a;
    for (int j = 0; j < N; ++j) lam[j] *= bt + 2.0 * at * std::cos((j + 1) * pi / (N + 1));
    delta *= std::exp(a * dt);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* Y = work;
  double* d_tab = work + nY;
  // pageable source: the copy is staged before the call returns, so h may go
  if (cudaMemcpyAsync(d_tab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PMF_ERR_CUDA;
  const dim3 blk(16, 16), grd((N + 15) / 16, (count + 15) / 16);
  k_dst_f64<<<grd, blk, 0, s>>>(P_in, d_tab, d_tab + 2 * (N + 1), Y, N, count);
  k_dst_f64<<<grd, blk, 0, s>>>(Y, d_tab, d_tab + 2 * (N + 1) + N, P_out, N, count);
  return cudaGetLastError() == cudaSuccess ? PMF_OK : PMF_ERR_CUDA;
}
