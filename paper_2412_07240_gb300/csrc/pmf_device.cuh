// Device functions shared by the float64 kernels and the tensor-core and
// float32 kernels: regrid/frame decision, sub-step diffusion coefficients and
// moment finalisation (float64, in the lanes of one warp).
#pragma once

#include "pmf_internal.cuh"

namespace pmf {


// ---------------------------------------------------------------------------
// Fixed-size float64 helpers (fully unrolled, registers only).  On GB300 a
// dependent float64 FMA costs ~64 cycles and a division ~430, so the per-epoch
// frame work avoids loops over local arrays and divides once per inverse.
// ---------------------------------------------------------------------------
template <int n>
__device__ __forceinline__ void mm_t(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) s = fma(A[i * n + k], B[k * n + j], s);
      C[i * n + j] = s;
    }
}

// C = A S A^T for symmetric S (upper triangle computed, mirrored).
template <int n>
__device__ __forceinline__ void cong_t(const double* A, const double* S, double* C) {
  double T[n * n];
  mm_t<n>(A, S, T);
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = i; j < n; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) s = fma(T[i * n + k], A[j * n + k], s);
      C[i * n + j] = s;
      C[j * n + i] = s;
    }
}

template <int n>
__device__ __forceinline__ double det_t(const double* A) {
  if (n == 4) return det(4, A);
  if (n == 1) return A[0];
  if (n == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Passes of one axis order (false if a leading block is singular); val = the
// largest |alpha|.
__device__ inline bool shear3_order(const double* B, const double* bb, const int* a, double* cand, double* val) {
  *val = 0.0;
  for (int i = 0; i < 24; ++i) cand[i] = 0.0;
  for (int k = 3; k >= 1; --k) {
    const int ax = a[k - 1], i = 3 - k;   // data order index
    double coef[3] = {0.0, 0.0, 0.0}, alpha[2] = {0.0, 0.0};
    const int ns = k - 1;
    if (ns == 1) {
      const double d = B[a[0] * 3 + a[0]];
      if (fabs(d) <= 1e-12 * fmax(1.0, fabs(d))) return false;
      alpha[0] = B[ax * 3 + a[0]] / d;
    } else if (ns == 2) {
      const double s00 = B[a[0] * 3 + a[0]], s01 = B[a[0] * 3 + a[1]];
      const double s10 = B[a[1] * 3 + a[0]], s11 = B[a[1] * 3 + a[1]];
      const double det = s00 * s11 - s01 * s10;
      const double mx = fmax(fmax(fabs(s00), fabs(s01)), fmax(fabs(s10), fabs(s11)));
      if (fabs(det) <= 1e-12 * fmax(1.0, mx) * fmax(1.0, mx)) return false;
      // alpha = B[ax, S] inv(B_SS), inv = [s11 -s01; -s10 s00] / det
      const double r0 = B[ax * 3 + a[0]], r1 = B[ax * 3 + a[1]];
      alpha[0] = (r0 * s11 - r1 * s10) / det;
      alpha[1] = (-r0 * s01 + r1 * s00) / det;
    }
    for (int m = 0; m < ns; ++m) *val = fmax(*val, fabs(alpha[m]));
    double gamma = bb[ax];
    for (int m = 0; m < ns; ++m) {
      coef[a[m]] = alpha[m];
      gamma -= alpha[m] * bb[a[m]];
    }
    for (int t = ns; t < 3; ++t) {          // T = {a_k..a_3}
      double v = B[ax * 3 + a[t]];
      for (int m = 0; m < ns; ++m) v -= alpha[m] * B[a[m] * 3 + a[t]];
      coef[a[t]] = v;
    }
    cand[8 * i] = ax;
    for (int m = 0; m < 3; ++m) cand[8 * i + 1 + m] = coef[m];
    cand[8 * i + 4] = gamma;
  }
  return true;
}

// Pass coefficients of the 3-D band-limited re-alignment for the frame's map
// u_old = B w + b: per pass in data order pc[8 i] = axis, pc[8 i + 1..3] =
// coefficient of each axis, pc[8 i + 4] = gamma; pc[24] = 1, or 0 (and false)
// when every order has a singular leading block.  The order minimises the
// largest |alpha|; orders within a relative 1e-9 of the minimum are tied
// (orders sharing their alpha sets tie exactly in real arithmetic) and the
// first tied one in lexicographic order is taken.
__device__ inline bool shear3_setup(const FrameState& f, double* pc) {
  const int orders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  double vals[6], cand[24], vmin = INFINITY;
  for (int o = 0; o < 6; ++o) {
    vals[o] = INFINITY;
    double v;
    if (shear3_order(f.B, f.b, orders[o], cand, &v)) vals[o] = v;
    vmin = fmin(vmin, vals[o]);
  }
  for (int i = 0; i < 25; ++i) pc[i] = 0.0;
  for (int o = 0; o < 6 && isfinite(vmin); ++o)
    if (vals[o] <= vmin * (1.0 + 1e-9)) {   // first tied order
      double v;
      shear3_order(f.B, f.b, orders[o], cand, &v);
      for (int i = 0; i < 24; ++i) pc[i] = cand[i];
      pc[24] = 1.0;
      return true;
    }
  return false;
}

// The same factorisation for n = 4: pass k (applied for k = 4, .., 1) along
// a_k with S = {a_1..a_{k-1}} on old and T = {a_k..a_4} on new coordinates,
// alpha = B[a_k, S] B[S, S]^{-1} (leading blocks up to 3 x 3, inverted by the
// adjugate), beta = B[a_k, T] - alpha B[S, T], gamma = b[a_k] - alpha b[S];
// a leading block is singular when |det| <= 1e-12 max(1, max |entry|)^|S|.
// Candidate layout per pass in data order: cand[10 i] = axis, cand[10 i + 1..4]
// = coefficient of each axis, cand[10 i + 5] = gamma.
__device__ inline bool shear4_order(const double* B, const double* bb, const int* a, double* cand, double* val) {
  *val = 0.0;
  for (int i = 0; i < 40; ++i) cand[i] = 0.0;
  for (int k = 4; k >= 1; --k) {
    const int ax = a[k - 1], i = 4 - k, ns = k - 1;
    double S[9], inv[9], alpha[3] = {0.0, 0.0, 0.0}, coef[4] = {0.0, 0.0, 0.0, 0.0};
    double mx = 0.0;
    for (int r = 0; r < ns; ++r)
      for (int c = 0; c < ns; ++c) {
        S[r * 3 + c] = B[a[r] * 4 + a[c]];
        mx = fmax(mx, fabs(S[r * 3 + c]));
      }
    double det = 1.0;
    if (ns == 1) {
      det = S[0];
      inv[0] = 1.0 / det;
    } else if (ns == 2) {
      det = S[0] * S[4] - S[1] * S[3];
      inv[0] = S[4] / det;
      inv[1] = -S[1] / det;
      inv[3] = -S[3] / det;
      inv[4] = S[0] / det;
    } else if (ns == 3) {
      const double c00 = S[4] * S[8] - S[5] * S[7], c01 = S[5] * S[6] - S[3] * S[8], c02 = S[3] * S[7] - S[4] * S[6];
      det = S[0] * c00 + S[1] * c01 + S[2] * c02;
      inv[0] = c00 / det;
      inv[3] = c01 / det;
      inv[6] = c02 / det;
      inv[1] = (S[2] * S[7] - S[1] * S[8]) / det;
      inv[4] = (S[0] * S[8] - S[2] * S[6]) / det;
      inv[7] = (S[1] * S[6] - S[0] * S[7]) / det;
      inv[2] = (S[1] * S[5] - S[2] * S[4]) / det;
      inv[5] = (S[2] * S[3] - S[0] * S[5]) / det;
      inv[8] = (S[0] * S[4] - S[1] * S[3]) / det;
    }
    if (ns > 0) {
      double lim = 1e-12;
      for (int r = 0; r < ns; ++r) lim *= fmax(1.0, mx);
      if (!(fabs(det) > lim)) return false;
    }
    for (int c = 0; c < ns; ++c) {
      double v = 0.0;
      for (int r = 0; r < ns; ++r) v += B[ax * 4 + a[r]] * inv[r * 3 + c];
      alpha[c] = v;
      *val = fmax(*val, fabs(v));
    }
    double gamma = bb[ax];
    for (int m = 0; m < ns; ++m) {
      coef[a[m]] = alpha[m];
      gamma -= alpha[m] * bb[a[m]];
    }
    for (int t = ns; t < 4; ++t) {
      double v = B[ax * 4 + a[t]];
      for (int m = 0; m < ns; ++m) v -= alpha[m] * B[a[m] * 4 + a[t]];
      coef[a[t]] = v;
    }
    cand[10 * i] = ax;
    for (int m = 0; m < 4; ++m) cand[10 * i + 1 + m] = coef[m];
    cand[10 * i + 5] = gamma;
  }
  return true;
}

// Pass coefficients of the 4-D band-limited re-alignment (layout of
// shear4_order, pc[40] = 1), or false (pc[40] = 0) when every order has a
// singular leading block.  The 24 axis orders are visited in lexicographic
// order; the order minimising the largest |alpha| is taken, orders within a
// relative 1e-9 of the minimum being tied and the first tied one chosen.
__device__ inline bool shear4_setup(const FrameState& f, double* pc) {
  int ord[24][4];
  {
    int p[4] = {0, 1, 2, 3};
    for (int o = 0; o < 24; ++o) {
      for (int m = 0; m < 4; ++m) ord[o][m] = p[m];
      // next permutation in lexicographic order
      int i = 2;
      while (i >= 0 && p[i] > p[i + 1]) --i;
      if (i < 0) break;
      int j = 3;
      while (p[j] < p[i]) --j;
      const int t = p[i];
      p[i] = p[j];
      p[j] = t;
      for (int l = i + 1, r = 3; l < r; ++l, --r) {
        const int u = p[l];
        p[l] = p[r];
        p[r] = u;
      }
    }
  }
  double vals[24], cand[40], vmin = INFINITY;
  for (int o = 0; o < 24; ++o) {
    vals[o] = INFINITY;
    double v;
    if (shear4_order(f.B, f.b, ord[o], cand, &v)) vals[o] = v;
    vmin = fmin(vmin, vals[o]);
  }
  for (int i = 0; i < 41; ++i) pc[i] = 0.0;
  for (int o = 0; o < 24 && isfinite(vmin); ++o)
    if (vals[o] <= vmin * (1.0 + 1e-9)) {
      double v;
      shear4_order(f.B, f.b, ord[o], cand, &v);
      for (int i = 0; i < 40; ++i) pc[i] = cand[i];
      pc[40] = 1.0;
      return true;
    }
  return false;
}

// Diffusion coefficients of sub-step q in the new frame (any thread):
// Q_u(t_q) = M'^{-1} Qt_q M'^{-T}, Qt_q = e^{-A q dt} Q e^{-A^T q dt} (host),
// pa = dt/2 Q_u,aa and pb = dt Q_u,ab (01, 02, 12); for the exact multiplier
// the integrated Q_b takes the place of dt Qt.
template <int n>
__device__ inline void frame_substep(const TimeConsts& tc, const double* Mpi, int q, double* pa, double* pb) {
  double Qt[n * n], Qu[n * n];
  const double* src = tc.exact ? tc.Qb : nullptr;
#pragma unroll
  for (int a = 0; a < n; ++a)
#pragma unroll
    for (int b = 0; b < n; ++b) {
      Qt[a * n + b] = src ? src[a * n + b] : tc.Qt[q][packed_sym(a, b)];
    }
  cong_t<n>(Mpi, Qt, Qu);
  const double w = tc.exact ? 1.0 : tc.dt;
#pragma unroll
  for (int a = 0; a < 4; ++a) pa[a] = a < n ? 0.5 * w * Qu[(a < n ? a : 0) * (n + 1)] : 0.0;
  // cross pairs 01, 02, 12, 03, 13, 23
  const int pi[6] = {0, 0, 1, 0, 1, 2}, pj[6] = {1, 2, 2, 3, 3, 3};
#pragma unroll
  for (int k = 0; k < 6; ++k) pb[k] = pj[k] < n ? w * Qu[(pj[k] < n ? pi[k] * n + pj[k] : 0)] : 0.0;
}

// ---------------------------------------------------------------------------
// Regrid decision and moment finalisation in warp lanes: all 32 lanes of one
// warp call them.  A float64 instruction costs GB300 ~64 cycles whatever the
// number of active lanes (and independent instructions of one thread do not
// overlap), so the entries of the small products run in parallel lanes: lane
// e < n*n (of each half-warp where both halves work) holds entry
// (e / n, e % n), lanes < n hold per-axis values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lget(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Regrid decision of one time update in lanes, for any n <= 4 (both
// branches).  From the current moments and frame: the pulled-back predicted
// covariance e^{-A tau} P_pred e^{-A^T tau} = cov + Q_b, its whitened
// correlation in the frame, and either the separable rescale/recentre
// (M' = M D, centre moved towards the mean by a multiple of 1/64 node, D with
// an 8-bit mantissa) or a re-aligned frame M' = e^{-A tau} chol(P_pred)
// diag(2 span / N) with 12-bit entries.  Writes the regrid map into st, the
// inverse of M' into Mpi and the pending frame after the move by e^{A tau}
// into pend (offsets pend_*).  Lane e < n*n holds matrix entry (e / n, e % n),
// lanes < n per-axis values; the products, the Cholesky factor (column by
// column) and the inverse (adjugate) run in parallel lanes.  Used for the
// re-alignment branch and for n = 4.
template <int n>
__device__ inline void frame_warp_full(const TimeConsts& tc, FrameState* st, double* pend, double* Mpi) {
  constexpr int nn = n * n;
  const int lane = threadIdx.x & 31;
  const int e = lane < nn ? lane : 0;
  const int i = e / n, j = e % n;
  const int a = lane < n ? lane : 0;
  // Su = Minv (cov + Qb) Minv^T (upper triangle mirrored)
  const double S = st->cov[e] + tc.Qb[e];
  double T = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) T = fma(st->Minv[i * n + k], lget(S, k * n + j), T);
  double C = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) C = fma(lget(T, i * n + k), st->Minv[j * n + k], C);
  const double Su = lget(C, i <= j ? e : j * n + i);
  const double Saa = lget(Su, a * (n + 1));
  bool realign = false;
  if (n >= 2) {
    const double r2 = tc.rho_max * tc.rho_max;
    const double Sii = lget(Su, i * (n + 1)), Sjj = lget(Su, j * (n + 1));
    realign = __any_sync(0xffffffffu, lane < nn && i < j && Su * Su > r2 * Sii * Sjj);
  }
  double Mp = 0.0, Mpie = 0.0;
  if (realign) {
    // Pp = Phi S Phi^T, its Cholesky factor L (lane (i, k) holds L_ik, i >= k)
    double U = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) U = fma(tc.Phi[i * n + k], lget(S, k * n + j), U);
    double W = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) W = fma(lget(U, i * n + k), tc.Phi[j * n + k], W);
    const double Pp = lget(W, i <= j ? e : j * n + i);
    double L = 0.0;
    bool pd = true;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      double t = Pp;
#pragma unroll
      for (int m = 0; m < k; ++m) t -= lget(L, i * n + m) * lget(L, k * n + m);
      const double dkk = lget(t, k * n + k);
      pd = pd && dkk > 0.0;
      const double d = sqrt(fmax(dkk, 0.0)), rd = 1.0 / d;
      if (lane < nn && j == k && i >= k) L = i == k ? d : t * rd;
    }
    if (pd) {
      // Mp = e^{-A tau} L diag(2 span / N), entries rounded to a 12-bit mantissa
      double T2 = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) T2 = fma(tc.PhiInv[i * n + k], lget(L, k * n + j), T2);
      int ex;
      const double f = frexp(T2 * (2.0 * tc.span / tc.N[j]), &ex);
      Mp = ldexp(rint(ldexp(f, 12)), ex - 12);
      // Mpi = adj(Mp) / det(Mp): lane (i, j) forms the cofactor of entry (i, j)
      double cof;
      if constexpr (n == 1) {
        cof = 1.0;
      } else {
        constexpr int m = n - 1;
        double mv[m * m];
#pragma unroll
        for (int rr = 0; rr < m; ++rr)
#pragma unroll
          for (int cc = 0; cc < m; ++cc)
            mv[rr * m + cc] = lget(Mp, (rr + (rr >= i)) * n + cc + (cc >= j));
        cof = ((i + j) & 1 ? -1.0 : 1.0) * det_t<m>(mv);
      }
      double dt = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) dt = fma(lget(Mp, k), lget(cof, k), dt);
      Mpie = lget(cof, j * n + i) * (1.0 / dt);
    } else {
      realign = false;   // not positive definite: keep the separable regrid
    }
  }
  // centre shift towards the mean, a multiple of 1/64 node (lanes a)
  const double dd = st->mean[a] - st->c[a];
  double dm = 0.0;
#pragma unroll
  for (int b = 0; b < n; ++b) dm = fma(st->Minv[a * n + b], lget(dd, b), dm);
  dm = rint(dm * 64.0) * (1.0 / 64.0);
  double cn = st->c[a];
#pragma unroll
  for (int b = 0; b < n; ++b) cn = fma(st->M[a * n + b], lget(dm, b), cn);
  if (realign) {
    // regrid map u_old = B u_new + b with B = Minv Mp, b = the shift
    double Bv = 0.0;
#pragma unroll
    for (int k = 0; k < n; ++k) Bv = fma(st->Minv[i * n + k], lget(Mp, k * n + j), Bv);
    __syncwarp();
    if (lane < nn) st->B[lane] = Bv;
    if (lane < n) st->b[lane] = dm;
  } else {
    // separable scale with an 8-bit mantissa (lanes a)
    const double sd = sqrt(fmax(Saa, 0.0));
    int ex;
    const double f = frexp(2.0 * tc.span * sd / tc.N[a], &ex);
    const double D = ldexp(rint(ldexp(f, 8)), ex - 8);
    const double rD = 1.0 / D;
    Mp = st->M[e] * lget(D, j);
    Mpie = st->Minv[e] * lget(rD, i);
    __syncwarp();
    if (lane < n) {
      st->rs[lane] = dm;
      st->rd[lane] = D;
    }
  }
  // pending frame after the move: Phi Mp, Mpi PhiInv, centre Phi c'
  double nM = 0.0, nMi = 0.0, pc = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) {
    nM = fma(tc.Phi[i * n + k], lget(Mp, k * n + j), nM);
    nMi = fma(lget(Mpie, i * n + k), tc.PhiInv[k * n + j], nMi);
    pc = fma(tc.Phi[a * n + k], lget(cn, k), pc);
  }
  double nMv[nn];
#pragma unroll
  for (int q = 0; q < nn; ++q) nMv[q] = lget(nM, q);
  const double det = det_t<n>(nMv);
  if (lane < nn) {
    pend[pend_M(n) + lane] = nM;
    pend[pend_Mi(n) + lane] = nMi;
    Mpi[lane] = Mpie;
  }
  if (lane < n) pend[lane] = pc;
  if (lane == 0) {
    st->realign = realign ? 1 : 0;
    st->exact = tc.exact;
    st->l = tc.exact ? 1 : tc.l;
    st->g = tc.g;
    pend[pend_V(n)] = fabs(det);
  }
  __syncwarp();
}

template <int n>
__device__ inline void frame_warp(const TimeConsts& tc, FrameState* st, double* pend, double* Mpi) {
  if constexpr (n == 4) {
    frame_warp_full<4>(tc, st, pend, Mpi);
    return;
  }
  constexpr int nn = n * n;
  const int lane = threadIdx.x & 31, h = lane & 15;
  const bool up = lane >= 16;
  const int e = h < nn ? h : 0;   // matrix entry of this lane
  const int i = e / n, j = e % n;
  const int a = h < n ? h : 0;    // axis of this lane
  // Su = Minv (cov + Qb) Minv^T (upper triangle as in cong_t, mirrored)
  const double S = st->cov[e] + tc.Qb[e];
  double T = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) T = fma(st->Minv[i * n + k], lget(S, k * n + j), T);
  double C = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) C = fma(lget(T, i * n + k), st->Minv[j * n + k], C);
  const double Su = lget(C, i <= j ? e : j * n + i);
  const double Saa = lget(Su, a * (n + 1));
  bool realign = false;
  if (n >= 2) {
    const double r2 = tc.rho_max * tc.rho_max;
    const double Sii = lget(Su, i * (n + 1)), Sjj = lget(Su, j * (n + 1));
    realign = __any_sync(0xffffffffu, lane < nn && i < j && Su * Su > r2 * Sii * Sjj);
  }
  if (realign) {
    frame_warp_full<n>(tc, st, pend, Mpi);
    return;
  }
  // centre shift towards the mean, a multiple of 1/64 node (lanes a)
  const double dd = st->mean[a] - st->c[a];
  double dm = 0.0;
#pragma unroll
  for (int b = 0; b < n; ++b) dm = fma(st->Minv[a * n + b], lget(dd, b), dm);
  dm = rint(dm * 64.0) * (1.0 / 64.0);
  double cn = st->c[a];
#pragma unroll
  for (int b = 0; b < n; ++b) cn = fma(st->M[a * n + b], lget(dm, b), cn);
  // separable scale with an 8-bit mantissa (lanes a)
  const double sd = sqrt(fmax(Saa, 0.0));
  int ex;
  const double f = frexp(2.0 * tc.span * sd / tc.N[a], &ex);
  const double D = ldexp(rint(ldexp(f, 8)), ex - 8);
  const double rD = 1.0 / D;
  // Mp = M D (column j scaled), Mpi = D^{-1} Minv (row i scaled)
  const double Mp = st->M[e] * lget(D, j);
  const double Mpie = st->Minv[e] * lget(rD, i);
  // pending frame: nM = Phi Mp (lower half-warp), nMi = Mpi PhiInv (upper
  // half) and its centre Phi c' (upper lanes nn .. nn + n - 1)
  const int pc = h - nn;
  const bool is_pc = up && pc >= 0 && pc < n;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const double m1 = lget(Mpie, i * n + k), m2 = lget(Mp, k * n + j), m3 = lget(cn, k);
    double x, y;
    if (is_pc) {
      x = tc.Phi[pc * n + k];
      y = m3;
    } else if (up) {
      x = m1;
      y = tc.PhiInv[k * n + j];
    } else {
      x = tc.Phi[i * n + k];
      y = m2;
    }
    s = fma(x, y, s);
  }
  double nMv[nn];
#pragma unroll
  for (int q = 0; q < nn; ++q) nMv[q] = lget(s, q);
  const double det = det_t<n>(nMv);
  if (!up && h < nn) {
    pend[3 + h] = s;
    Mpi[h] = Mpie;
  }
  if (up && h < nn) pend[12 + h] = s;
  if (is_pc) pend[pc] = s;
  if (lane < n) {
    st->rs[lane] = dm;
    st->rd[lane] = D;
  }
  if (lane == 0) {
    st->realign = 0;
    st->exact = tc.exact;
    st->l = tc.exact ? 1 : tc.l;
    st->g = tc.g;
    pend[21] = fabs(det);
  }
  __syncwarp();
}

template <int n>
__device__ inline bool finalize_warp(FrameState* st, const double* tot, int use_pending, const double* pend) {
  constexpr int nn = n * n;
  const int lane = threadIdx.x & 31, h = lane & 15;
  const bool up = lane >= 16;
  const double S0 = tot[0];
  if (!(S0 > 0.0) || !isfinite(S0)) {
    if (lane == 0) st->status = PMF_ERR_DEGENERATE;
    __syncwarp();
    return false;
  }
  const int e = h < nn ? h : 0;
  const int i = e / n, j = e % n;
  const int a = h < n ? h : 0;
  const double* c = use_pending ? pend : st->c;
  const double* M = use_pending ? pend + pend_M(n) : st->M;
  const double V = use_pending ? pend[pend_V(n)] : st->V;
  const double r = 1.0 / S0;
  const double mu = tot[1 + a] * r;
  const double mui = lget(mu, i), muj = lget(mu, j);
  const double Cu = fma(tot[tot_S2(n, i, j)], r, -mui * muj);
  // T = M Cu (lower half-warp) and the mean c + M mu (upper lanes a)
  double s = up ? c[a] : 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const double cu = lget(Cu, k * n + j), mk = lget(mu, k);
    const double x = up ? M[a * n + k] : M[i * n + k], y = up ? mk : cu;
    s = fma(x, y, s);
  }
  double C = 0.0;
#pragma unroll
  for (int k = 0; k < n; ++k) C = fma(lget(s, i * n + k), M[j * n + k], C);
  const double cov = lget(C, i <= j ? e : j * n + i);
  double Mv = 0.0, Miv = 0.0;
  if (use_pending) {
    Mv = pend[pend_M(n) + e];
    Miv = pend[pend_Mi(n) + e];
  }
  __syncwarp();
  if (up && h < n) st->mean[h] = s;
  if (lane < nn) st->cov[lane] = cov;
  if (use_pending) {
    if (lane < n) st->c[lane] = pend[lane];
    if (lane < nn) {
      st->M[lane] = Mv;
      st->Minv[lane] = Miv;
    }
    if (lane == 0) st->V = V;
  }
  if (lane == 0) {
    st->S0 = S0;
    st->pscale = r / V;
  }
  __syncwarp();
  return true;
}

}  // namespace pmf
