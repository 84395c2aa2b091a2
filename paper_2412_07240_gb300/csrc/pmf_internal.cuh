// Internal declarations of libpmf: device state layout, per-update constants
// and float64 small-matrix helpers shared by host and device code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pmf.h"

#define PMF_HD __host__ __device__ __forceinline__

namespace pmf {

constexpr int MAXN = PMF_MAX_NX;
constexpr int MAXL = PMF_MAX_SUBSTEPS;

// Grid geometry: nx axes, N[m] points along axis m, C order.
struct Dims {
  int nx;
  int N[MAXN];
  long long P;
};

// Constants of one time update that depend only on the model and tau
// (computed on the host in float64, passed by value to the frame kernel).
struct TimeConsts {
  int nx, l, exact;
  int N[MAXN];
  int realign_mode;  // PMF_REALIGN_*
  double tau, dt, g, span, rho_max;
  double Q[16];       // diffusion
  double Phi[16];     // e^{A tau}
  double PhiInv[16];  // e^{-A tau}
  double Qb[16];      // int_0^tau e^{-A s} Q e^{-A^T s} ds
  double Estep[16];   // e^{-A dt}
  // e^{-A q dt} Q e^{-A^T q dt}, q = 1..l, packed 00,01,02,11,12,22 then 03,13,23,33
  double Qt[MAXL][10];
};

// 8-byte words of a TimeConsts that a time update reads: everything up to the
// sub-step rows it uses (Qt is the last member; the exact multiplier reads none
// of them but one row is kept).
PMF_HD int tc_words(const TimeConsts* tc) {
  const int rows = tc->exact ? 1 : tc->l;
  return (int)((sizeof(TimeConsts) - sizeof(tc->Qt) + sizeof(tc->Qt[0]) * rows) / 8);
}

// Index of the symmetric entry (a, b) in the packed order of TimeConsts::Qt.
PMF_HD int packed_sym(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  if (hi == 3) return 6 + lo;
  return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// Pending frame {c, M, Minv, V} (written by the frame computation, committed
// by the finalisation): fixed offsets for n <= 3, and for n = 4.
PMF_HD int pend_M(int n) { return n == 4 ? 4 : 3; }
PMF_HD int pend_Mi(int n) { return n == 4 ? 20 : 12; }
PMF_HD int pend_V(int n) { return n == 4 ? 36 : 21; }
constexpr int kPendSize = 40;
// Prior constants handed to the initial-PDF kernels: P0^{-1} row-major with
// row stride n at [0, n*n), m0 at [kAuxM0, kAuxM0 + n).
constexpr int kAuxM0 = 16;
constexpr int kAuxSize = 20;
// Slots of the moment sums {S0, S1[n], S2}: 10 cover n <= 3, 15 cover n = 4.
constexpr int kMomentSlots = 15;

// Moment sums tot = {S0, S1[n], S2 packed as TimeConsts::Qt}: the second
// moments start at 4 for n <= 3 (the {S0, S1[3], S2[6]} layout) and at 5 for n = 4.
PMF_HD int tot_S2(int n, int a, int b) { return (n == 4 ? 5 : 4) + packed_sym(a, b); }


// Measurement update parameters (by value).
struct MeasParams {
  int kind, nz, nx;
  double z[PMF_MAX_NZ];
  double Rinv[9];
  double H[PMF_MAX_NZ * PMF_MAX_NX];
  double p[PMF_MEAS_NPARAM];
  double gm[6];   // TERRAIN_GM: 1/(2 v1), 1/(2 v2), log(v_g)/2 - log w_g (g = 1, 2; common shift, min log 2), mu1, mu2
};

// Frame, moments and per-update scalars of one filter (float64).  Frame
// x = c + M u; weights stored in one of two buffers (cur), true weight =
// pscale * stored.  Kernels that do scalar work on it copy it to shared or
// local memory first.
struct FrameState {
  double c[4], M[16], Minv[16], V;
  double mean[4], cov[16];
  double S0, pscale, g;
  // regrid of the current time update
  double rs[4], rd[4];   // separable: u_old_m = rs_m + rd_m * u_new_m
  double B[16], b[4];    // realigned: u_old = B u_new + b
  double hc[2];          // at the frame centre: atan2(c_2, c_1) and c_1^2 + c_2^2 (n_x = 3)
  int cur, status, realign, l, exact, pad;
};

// Per-filter device state: the frame state, the exponent minimum of the
// measurement update and the diffusion coefficients per sub-step (Euler) or
// integrated (exact): psi_n(k) = 1 + sum_a pa[n][a] kappa_a^2 + sum_{a<b} pb[n][ab] kt_a kt_b.
struct DevState {
  FrameState f;
  unsigned long long emin_bits;
  double pa[MAXL][4];
  double pb[MAXL][6];    // cross pairs 01, 02, 12, 03, 13, 23
};

// ---------------------------------------------------------------------------
// float64 n x n helpers (row-major, n <= 4 on the device; <= 8 on the host)
// ---------------------------------------------------------------------------
PMF_HD void mm(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      C[i * n + j] = s;
    }
}

// C = A B^T
PMF_HD void mmt(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[j * n + k];
      C[i * n + j] = s;
    }
}

// C = A S A^T (S symmetric), symmetrised
PMF_HD void congruence(int n, const double* A, const double* S, double* C) {
  double T[64];
  mm(n, A, S, T);
  mmt(n, T, A, C);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double v = 0.5 * (C[i * n + j] + C[j * n + i]);
      C[i * n + j] = C[j * n + i] = v;
    }
}

PMF_HD double det(int n, const double* A) {
  if (n == 1) return A[0];
  if (n == 2) return A[0] * A[3] - A[1] * A[2];
  if (n == 3)
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
  // n = 4: expansion along the first row
  double s = 0.0;
  for (int c = 0; c < 4; ++c) {
    double m[9];
    for (int r = 1, k = 0; r < 4; ++r)
      for (int cc = 0; cc < 4; ++cc)
        if (cc != c) m[k++] = A[r * 4 + cc];
    const double minor = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                         m[2] * (m[3] * m[7] - m[4] * m[6]);
    s += ((c & 1) ? -1.0 : 1.0) * A[c] * minor;
  }
  return s;
}

// Gauss-Jordan inverse with partial pivoting; returns false if singular.
PMF_HD bool inv(int n, const double* A, double* Ai) {
  double W[64], I[64];
  for (int i = 0; i < n * n; ++i) { W[i] = A[i]; I[i] = 0.0; }
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(W[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(W[r * n + c]) > best) { best = fabs(W[r * n + c]); p = r; }
    if (!(best > 0.0)) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        double t = W[c * n + k]; W[c * n + k] = W[p * n + k]; W[p * n + k] = t;
        t = I[c * n + k]; I[c * n + k] = I[p * n + k]; I[p * n + k] = t;
      }
    double d = 1.0 / W[c * n + c];
    for (int k = 0; k < n; ++k) { W[c * n + k] *= d; I[c * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = W[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { W[r * n + k] -= f * W[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
    }
  }
  for (int i = 0; i < n * n; ++i) Ai[i] = I[i];
  return true;
}

// Lower Cholesky factor; returns false if not positive definite.
PMF_HD bool chol(int n, const double* A, double* L) {
  for (int i = 0; i < n * n; ++i) L[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return false;
    double d = sqrt(s);
    L[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / d;
    }
  }
  return true;
}

PMF_HD int popc(unsigned v) {
  int c = 0;
  while (v) { c += v & 1u; v >>= 1; }
  return c;
}

}  // namespace pmf
