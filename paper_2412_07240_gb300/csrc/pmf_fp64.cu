// Plain float64 path of the spectral point-mass filter: one small kernel per
// step of the method, all data in global memory.  It is the reference GPU
// implementation against which the mixed-precision tensor-core path is
// compared, and it serves grids of any even size and n_x <= 4.
//
// Per time update (Sec. V-B algorithm on the moving grid, eq. gridMov):
//   frame       regrid decision and per-sub-step diffusion coefficients
//   realign     multilinear re-alignment (or copy) of the weights
//   interp x n  trigonometric regrid (eq. interFreq) along each axis
//   fwd x n     per-axis Hartley transform (real form of eq. fourtrsf)
//   psi         diffusion multiplier and trace factor (algorithm steps 2-4),
//               with the separable-to-n-D Hartley parity fix-up
//   inv x n     per-axis inverse Hartley transform (step 5)
//   moments     normalisation constant and moments (step 6)
// Per measurement update (eq. filt): exponent minimum, likelihood multiply
// with moment partial sums, finalisation.
#include <cmath>

#include "pmf_internal.cuh"
#include "pmf_kernels.cuh"
#include "pmf_grid.cuh"
#include "pmf_device.cuh"

namespace pmf {

__global__ void k_meas_emin_f64(Dims d, MeasParams mp, DevState* st) {
  double emin = INFINITY;
  const double* c = st->f.c;
  const double* M = st->f.M;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    unflatten(d, p, j);
    double x[MAXN];
    for (int a = 0; a < d.nx; ++a) {
      x[a] = c[a];
      for (int b = 0; b < d.nx; ++b) x[a] += M[a * d.nx + b] * (j[b] - 0.5 * (d.N[b] - 1));
    }
    emin = fmin(emin, meas_exponent_f64(mp, x));
  }
  for (int o = 16; o; o >>= 1) emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, o));
  if ((threadIdx.x & 31) == 0)
    atomicMin(&st->emin_bits, (unsigned long long)__double_as_longlong(emin));
}

__global__ void k_meas_apply_f64(Dims d, MeasParams mp, DevState* st, double* b0, double* b1,
                                 double* partials) {
  __shared__ double sm[32 * kMomentSlots];
  const int cur = st->f.cur;
  const double* in = cur ? b1 : b0;
  double* out = cur ? b0 : b1;
  const double emin = __longlong_as_double((long long)st->emin_bits);
  const double ps = st->f.pscale;
  double acc[kMomentSlots] = {};
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    unflatten(d, p, j);
    double u[MAXN], x[MAXN];
    for (int a = 0; a < d.nx; ++a) u[a] = j[a] - 0.5 * (d.N[a] - 1);
    for (int a = 0; a < d.nx; ++a) {
      x[a] = st->f.c[a];
      for (int b = 0; b < d.nx; ++b) x[a] += st->f.M[a * d.nx + b] * u[b];
    }
    const double v = in[p] * ps * exp(-(meas_exponent_f64(mp, x) - emin));
    out[p] = v;
    acc_moments(acc, v, u, d.nx);
  }
  block_sum<kMomentSlots>(acc, sm, partials + blockIdx.x * kMomentSlots);
}

// Sum block partials, finalise moments and the normaliser.  use_pending: the
// weights are on the frame written by k_frame (time update) and that frame is
// committed here.  flip: buffer parity change of the update.
// The moments are formed by warp 0 in parallel lanes (finalize_warp: one
// matrix entry per lane) on a shared copy of the frame state.
__global__ void k_finalize(Dims d, DevState* st, const double* partials, int nblocks, int flip,
                           int use_pending, const double* pend /* c, M, Minv, V */) {
  __shared__ double sm[32 * kMomentSlots];
  __shared__ double tot[kMomentSlots];
  __shared__ FrameState fs;
  constexpr int kWords = sizeof(FrameState) / 8;
  double acc[kMomentSlots] = {};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int i = 0; i < kMomentSlots; ++i) acc[i] += partials[b * kMomentSlots + i];
  block_sum<kMomentSlots>(acc, sm, tot);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  bool ok;
  if (d.nx == 1) ok = finalize_warp<1>(&fs, tot, use_pending, pend);
  else if (d.nx == 2) ok = finalize_warp<2>(&fs, tot, use_pending, pend);
  else if (d.nx == 3) ok = finalize_warp<3>(&fs, tot, use_pending, pend);
  else ok = finalize_warp<4>(&fs, tot, use_pending, pend);
  if (ok && threadIdx.x == 0) fs.cur ^= flip;
  __syncwarp();
  for (int i = threadIdx.x; i < kWords; i += 32)
    ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
}

// Regrid decision (warp 0, lane-parallel, on a shared copy of the frame
// state) and the diffusion coefficients of every sub-step (one thread each)
// of one time update.
// The constants are staged in shared memory first: the lanes read different
// entries, which the parameter (constant) bank would serialise.
template <int n>
__device__ void frame_body(const TimeConsts& tcp, DevState* st, double* pend) {
  __shared__ FrameState fs;
  __shared__ double Mpi[16];
  __shared__ TimeConsts tc;
  constexpr int kWords = sizeof(FrameState) / 8;
  const int tc_w = tc_words(&tcp);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  for (int i = threadIdx.x; i < tc_w; i += blockDim.x)
    ((unsigned long long*)&tc)[i] = ((const unsigned long long*)&tcp)[i];
  __syncthreads();
  if (threadIdx.x < 32) frame_warp<n>(tc, &fs, pend, Mpi);
  __syncthreads();
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
  const int l = tc.exact ? 1 : tc.l;
  for (int q = threadIdx.x; q < l; q += blockDim.x) frame_substep<n>(tc, Mpi, q, st->pa[q], st->pb[q]);
}

__global__ void k_frame(const __grid_constant__ TimeConsts tc, DevState* st, double* pend) {
  if (tc.nx == 1) frame_body<1>(tc, st, pend);
  else if (tc.nx == 2) frame_body<2>(tc, st, pend);
  else if (tc.nx == 3) frame_body<3>(tc, st, pend);
  else frame_body<4>(tc, st, pend);
}

// Periodic-sinc interpolation matrix of one axis (eq. interFreq evaluated at
// the new nodes): I[q, j] = sin(pi v) / (N tan(pi v / N)), v = y_q - u_j;
// rows of new nodes outside the old box are zero; identity when re-aligned.
__global__ void k_build_interp_f64(Dims d, const DevState* st, int axis, double* I) {
  const int N = d.N[axis];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int q = idx / N, j = idx % N;
  if (st->f.realign) {
    I[idx] = q == j ? 1.0 : 0.0;
    return;
  }
  const double y = st->f.rs[axis] + st->f.rd[axis] * (q - 0.5 * (N - 1));
  if (fabs(y) > 0.5 * N) {
    I[idx] = 0.0;
    return;
  }
  const double v = y - (j - 0.5 * (N - 1));
  I[idx] = v == 0.0 ? 1.0 : sinpi(v) * cospi(v / N) / (N * sinpi(v / N));
}

// Band-limited re-alignment of a 2-D grid (shear mode), one of two line-wise
// passes, one CTA per line.  With u_old = B u_new + b and (p, q) = (0, 1) if
// |B_10 / B_00| <= |B_01 / B_11| else (1, 0) (the smaller line-dependent shift
// in pass 1; exact on trigonometric polynomials when B is triangular):
//   pass 1: lines along axis q through old node i of axis p, evaluated at
//           u_q = (B_qp / B_pp)(u_i - b_p) + b_q + (det B / B_pp) v;
//   pass 2: lines along axis p through new node v of axis q, evaluated at
//           u_p = B_pp w + B_pq v + b_p, times the normaliser.
// On each line: X_s = (1/N) sum_j f_j e^{-2 pi i j s / N} (s = 0..N/2) and the
// trigonometric interpolant (eq. interFreq)
//   p(x) = X_0 + 2 sum_{0<s<N/2} Re(X_s e^{2 pi i s x / N}) + X_{N/2} cos(pi x)
// at x = u + (N-1)/2; positions outside the old box give 0.  Pass 1 reads
// buf[cur] into scratch, pass 2 writes buf[cur^1].
__global__ void k_shear_f64(Dims d, const DevState* st, int pass, double* b0, double* b1, double* scratch) {
  extern __shared__ double sm[];
  const FrameState& f = st->f;
  if (!f.realign) return;
  // pass order making pass 1's line-dependent shift the smaller: |B_10 / B_00| <= |B_01 / B_11|
  const int p = fabs(f.B[2]) * fabs(f.B[3]) <= fabs(f.B[1]) * fabs(f.B[0]) ? 0 : 1, q = 1 - p;
  const double Bpp = f.B[p * 2 + p], Bpq = f.B[p * 2 + q], Bqp = f.B[q * 2 + p], Bqq = f.B[q * 2 + q];
  const int Np = d.N[p], Nq = d.N[q];
  const int N = pass == 1 ? Nq : Np, H = N / 2;
  const double* in = pass == 1 ? (f.cur ? b1 : b0) : scratch;
  double* out = pass == 1 ? scratch : (f.cur ? b0 : b1);
  const int line = blockIdx.x;
  if (line >= (pass == 1 ? Np : Nq)) return;
  // element (index along p, index along q) of the C-order 2-D grid
  auto at = [&](int ip, int iq) -> long long {
    return p == 0 ? (long long)ip * d.N[1] + iq : (long long)iq * d.N[1] + ip;
  };
  double* fl = sm;
  double* Xr = fl + N;
  double* Xi = Xr + H + 1;
  double* cs = Xi + H + 1;
  double* sn = cs + N;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    fl[t] = pass == 1 ? in[at(line, t)] : in[at(t, line)];
    sincospi(2.0 * t / N, &sn[t], &cs[t]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s <= H; s += blockDim.x) {
    double re = 0.0, im = 0.0;
    int r = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(fl[j], cs[r], re);
      im = fma(-fl[j], sn[r], im);
      r += s;
      if (r >= N) r -= N;
    }
    Xr[s] = re / N;
    Xi[s] = im / N;
  }
  __syncthreads();
  const double ul = line - 0.5 * ((pass == 1 ? Np : Nq) - 1);   // the line's fixed coordinate
  const double ps = pass == 2 ? f.pscale : 1.0;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const double ut = t - 0.5 * (N - 1);
    const double pos = pass == 1 ? (Bqp / Bpp) * (ul - f.b[p]) + f.b[q] + (Bpp * Bqq - Bpq * Bqp) / Bpp * ut
                                 : Bpp * ut + Bpq * ul + f.b[p];
    double v = 0.0;
    if (fabs(pos) <= 0.5 * N) {
      const double x = pos + 0.5 * (N - 1);
      double sx, cx;
      sincospi(2.0 * x / N, &sx, &cx);
      double zr = 1.0, zi = 0.0;   // e^{2 pi i s x / N}
      v = Xr[0];
      for (int k = 1; k < H; ++k) {
        const double nr = zr * cx - zi * sx;
        zi = zr * sx + zi * cx;
        zr = nr;
        v += 2.0 * (Xr[k] * zr - Xi[k] * zi);
      }
      v += Xr[H] * cospi(x);
    }
    if (pass == 1) out[at(line, t)] = v;
    else out[at(t, line)] = ps * v;
  }
}

// Band-limited re-alignment of a 4-D grid: the four line-wise passes of
// shear4_setup (pmf_device.cuh), written by k_shear4_setup as pc[10 i] = axis,
// pc[10 i + 1..4] = coefficient of each axis, pc[10 i + 5] = gamma (data
// order), pc[40] = 1 (0 and status DEGENERATE if every order is singular).
__global__ void k_shear4_setup(DevState* st, double* pc) {
  if (!st->f.realign) return;
  if (!shear4_setup(st->f, pc)) st->f.status = PMF_ERR_DEGENERATE;
}

// One pass of the 4-D band-limited re-alignment: one CTA per line along the
// pass's axis (surplus CTAs exit), the line's DFT coefficients from an exact
// twiddle table and the trigonometric interpolant (eq. interFreq) at its
// positions, as in k_shear3_f64.  Buffers: pass 0 buf[cur] -> scratch, pass 1
// scratch -> buf[cur], pass 2 buf[cur] -> scratch, pass 3 scratch ->
// buf[cur ^ 1] with pscale.
__global__ void k_shear4_f64(Dims d, const DevState* st, const double* pc, int pass, double* b0, double* b1,
                             double* scratch) {
  extern __shared__ double sm[];
  const FrameState& f = st->f;
  if (!f.realign || pc[40] == 0.0) return;
  double* bc = f.cur ? b1 : b0;
  double* bn = f.cur ? b0 : b1;
  const double* in = (pass & 1) ? scratch : bc;
  double* out = pass == 3 ? bn : (pass & 1) ? bc : scratch;
  const int a = (int)pc[10 * pass];
  const double* coef = pc + 10 * pass + 1;
  const double gamma = pc[10 * pass + 5];
  int o[3], no = 0;
  for (int m = 0; m < 4; ++m)
    if (m != a) o[no++] = m;
  const int N = d.N[a], H = N / 2;
  const long long lines = d.P / N;
  const long long line = blockIdx.x;
  if (line >= lines) return;
  long long stride[4];
  stride[3] = 1;
  for (int m = 2; m >= 0; --m) stride[m] = stride[m + 1] * d.N[m + 1];
  long long rest = line, base = 0;
  double offset = gamma;
  for (int q = 2; q >= 0; --q) {
    const int m = o[q];
    const int i = (int)(rest % d.N[m]);
    rest /= d.N[m];
    base += i * stride[m];
    offset += coef[m] * (i - 0.5 * (d.N[m] - 1));
  }
  const long long sa = stride[a];
  double* fl = sm;
  double* Xr = fl + N;
  double* Xi = Xr + H + 1;
  double* cs = Xi + H + 1;
  double* sn = cs + N;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    fl[t] = in[base + t * sa];
    sincospi(2.0 * t / N, &sn[t], &cs[t]);
  }
  __syncthreads();
  for (int sidx = threadIdx.x; sidx <= H; sidx += blockDim.x) {
    double re = 0.0, im = 0.0;
    int r = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(fl[j], cs[r], re);
      im = fma(-fl[j], sn[r], im);
      r += sidx;
      if (r >= N) r -= N;
    }
    Xr[sidx] = re / N;
    Xi[sidx] = im / N;
  }
  __syncthreads();
  const double ps = pass == 3 ? f.pscale : 1.0;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const double pos = offset + coef[a] * (t - 0.5 * (N - 1));
    double v = 0.0;
    if (fabs(pos) <= 0.5 * N) {
      const double x = pos + 0.5 * (N - 1);
      double sx, cx;
      sincospi(2.0 * x / N, &sx, &cx);
      double zr = 1.0, zi = 0.0;   // e^{2 pi i s x / N}
      v = Xr[0];
      for (int k = 1; k < H; ++k) {
        const double nr = zr * cx - zi * sx;
        zi = zr * sx + zi * cx;
        zr = nr;
        v += 2.0 * (Xr[k] * zr - Xi[k] * zi);
      }
      v += Xr[H] * cospi(x);
    }
    out[base + t * sa] = ps * v;
  }
}

// Band-limited re-alignment of a 3-D grid (shear mode): the map u_old = B w + b
// factored into three line-wise passes.  With an axis order (a_1, a_2, a_3),
// pass k (applied in the order k = 3, 2, 1) resamples along a_k; the axes
// S = {a_1..a_{k-1}} still carry old coordinates and T = {a_k..a_3} new ones,
// and the old coordinate a_k of a node is
//   alpha . u_S + beta . w_T + gamma,  alpha = B[a_k, S] B[S, S]^{-1},
//   beta = B[a_k, T] - alpha B[S, T],  gamma = b[a_k] - alpha b[S].
// The order and coefficients come from shear3_setup (pmf_device.cuh);
// k_shear3_setup (one thread) writes them, per pass in data order, as
// pc[8 i] = axis, pc[8 i + 1..3] = coefficient of each axis, pc[8 i + 4] =
// gamma, and pc[24] = 1 (0 and status DEGENERATE if every order has a
// singular leading block).
__global__ void k_shear3_setup(DevState* st, double* pc) {
  if (!st->f.realign) return;
  if (!shear3_setup(st->f, pc)) st->f.status = PMF_ERR_DEGENERATE;
}

// One pass of the 3-D band-limited re-alignment: one CTA per line along the
// pass's axis (surplus CTAs exit); per line the DFT coefficients from an exact
// twiddle table, then the trigonometric interpolant (eq. interFreq) at the
// line's positions by a recurrence from an exactly formed e^{2 pi i x / N};
// positions outside the old box give 0.  Buffers: pass 0 buf[cur] -> scratch,
// pass 1 scratch -> buf[cur] (the old grid is no longer needed), pass 2
// buf[cur] -> buf[cur ^ 1] with pscale.
__global__ void k_shear3_f64(Dims d, const DevState* st, const double* pc, int pass, double* b0, double* b1,
                             double* scratch) {
  extern __shared__ double sm[];
  const FrameState& f = st->f;
  if (!f.realign || pc[24] == 0.0) return;
  double* bc = f.cur ? b1 : b0;
  double* bn = f.cur ? b0 : b1;
  const double* in = pass == 1 ? scratch : bc;
  double* out = pass == 0 ? scratch : pass == 1 ? bc : bn;
  const int last = pass == 2;
  const int a = (int)pc[8 * pass];
  const double* coef = pc + 8 * pass + 1;
  const double gamma = pc[8 * pass + 4];
  const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
  const int N = d.N[a], H = N / 2, N1 = d.N[o1], N2 = d.N[o2];
  const int line = blockIdx.x;
  if (line >= N1 * N2) return;
  const int i1 = line / N2, i2 = line % N2;
  long long stride[3];
  stride[2] = 1;
  stride[1] = d.N[2];
  stride[0] = (long long)d.N[1] * d.N[2];
  const long long base = i1 * stride[o1] + i2 * stride[o2], sa = stride[a];
  double* fl = sm;
  double* Xr = fl + N;
  double* Xi = Xr + H + 1;
  double* cs = Xi + H + 1;
  double* sn = cs + N;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    fl[t] = in[base + t * sa];
    sincospi(2.0 * t / N, &sn[t], &cs[t]);
  }
  __syncthreads();
  for (int sidx = threadIdx.x; sidx <= H; sidx += blockDim.x) {
    double re = 0.0, im = 0.0;
    int r = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(fl[j], cs[r], re);
      im = fma(-fl[j], sn[r], im);
      r += sidx;
      if (r >= N) r -= N;
    }
    Xr[sidx] = re / N;
    Xi[sidx] = im / N;
  }
  __syncthreads();
  const double offset = gamma + coef[o1] * (i1 - 0.5 * (N1 - 1)) + coef[o2] * (i2 - 0.5 * (N2 - 1));
  const double ps = last ? f.pscale : 1.0;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const double pos = offset + coef[a] * (t - 0.5 * (N - 1));
    double v = 0.0;
    if (fabs(pos) <= 0.5 * N) {
      const double x = pos + 0.5 * (N - 1);
      double sx, cx;
      sincospi(2.0 * x / N, &sx, &cx);
      double zr = 1.0, zi = 0.0;   // e^{2 pi i s x / N}
      v = Xr[0];
      for (int k = 1; k < H; ++k) {
        const double nr = zr * cx - zi * sx;
        zi = zr * sx + zi * cx;
        zr = nr;
        v += 2.0 * (Xr[k] * zr - Xi[k] * zi);
      }
      v += Xr[H] * cospi(x);
    }
    out[base + t * sa] = ps * v;
  }
}

// Stage 0 of the time update: multilinear re-alignment when the frame was
// re-aligned, otherwise a scaled copy (both fold the normalisation scale in).
// In the shear mode a re-aligned frame is filled by k_shear_f64 (2-D) or
// k_shear3_f64 (3-D) instead.
__global__ void k_realign_f64(Dims d, const DevState* st, double* b0, double* b1, int mode) {
  const int cur = st->f.cur;
  const double* in = cur ? b1 : b0;
  double* out = cur ? b0 : b1;
  const double ps = st->f.pscale;
  const int n = d.nx;
  if (st->f.realign && mode == PMF_REALIGN_SHEAR) return;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    if (!st->f.realign) {
      out[p] = ps * in[p];
      continue;
    }
    int j[MAXN];
    unflatten(d, p, j);
    double z[MAXN];
    int f[MAXN];
    double w[MAXN];
    for (int a = 0; a < n; ++a) {
      double uo = st->f.b[a];
      for (int b = 0; b < n; ++b) uo += st->f.B[a * n + b] * (j[b] - 0.5 * (d.N[b] - 1));
      z[a] = uo + 0.5 * (d.N[a] - 1);
      const double fl = floor(z[a]);
      f[a] = (int)fmax(fmin(fl, 1e9), -1e9);
      w[a] = z[a] - fl;
    }
    double s = 0.0;
    for (int corner = 0; corner < (1 << n); ++corner) {
      double wt = 1.0;
      long long off = 0;
      bool ok = true;
      for (int a = 0; a < n; ++a) {
        const int bit = (corner >> a) & 1;
        const int i = f[a] + bit;
        wt *= bit ? w[a] : 1.0 - w[a];
        ok = ok && i >= 0 && i < d.N[a];
        off = off * d.N[a] + (ok ? i : 0);
      }
      if (ok) s += wt * in[off];
    }
    out[p] = ps * s;
  }
}

// Per-axis transform Y = W x_axis X (float64, 16x16 shared-memory tiles).
// Buffers: reads bufs[(cur+stage)&1], writes the other one.
__global__ void k_axis_gemm_f64(Dims d, int axis, const double* W, const DevState* st, int stage,
                                double* b0, double* b1) {
  __shared__ double Ls[16][17];
  __shared__ double Rs[16][17];
  const int par = (st->f.cur + stage) & 1;
  const double* X = par ? b1 : b0;
  double* Y = par ? b0 : b1;
  const int N = d.N[axis];
  long long inner = 1;
  for (int m = axis + 1; m < d.nx; ++m) inner *= d.N[m];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long o = blockIdx.z;
  if (inner == 1) {
    // rows of X (one line each) times W^T: C[r][k] = sum_j X[r][j] W[k][j]
    const long long r = blockIdx.y * 16LL + ty;
    const int k = blockIdx.x * 16 + tx;
    const long long rows = d.P / N;
    double acc = 0.0;
    for (int j0 = 0; j0 < N; j0 += 16) {
      const long long rr = blockIdx.y * 16LL + ty;
      Ls[ty][tx] = (rr < rows && j0 + tx < N) ? X[rr * N + j0 + tx] : 0.0;
      const int kk = blockIdx.x * 16 + ty;
      Rs[ty][tx] = (kk < N && j0 + tx < N) ? W[(long long)kk * N + j0 + tx] : 0.0;
      __syncthreads();
#pragma unroll
      for (int t = 0; t < 16; ++t) acc += Ls[ty][t] * Rs[tx][t];
      __syncthreads();
    }
    if (r < rows && k < N) Y[r * N + k] = acc;
  } else {
    // C[o][k][i] = sum_j W[k][j] X[o][j][i]
    const int k = blockIdx.y * 16 + ty;
    const long long i = blockIdx.x * 16LL + tx;
    const double* Xo = X + o * N * inner;
    double acc = 0.0;
    for (int j0 = 0; j0 < N; j0 += 16) {
      Ls[ty][tx] = (k < N && j0 + tx < N) ? W[(long long)k * N + j0 + tx] : 0.0;
      Rs[ty][tx] = (j0 + ty < N && i < inner) ? Xo[(long long)(j0 + ty) * inner + i] : 0.0;
      __syncthreads();
#pragma unroll
      for (int t = 0; t < 16; ++t) acc += Ls[ty][t] * Rs[t][tx];
      __syncthreads();
    }
    if (k < N && i < inner) Y[o * N * inner + (long long)k * inner + i] = acc;
  }
}

// Diffusion multiplier Psi and trace factor applied in the Hartley domain
// (algorithm steps 2-4), one thread per orbit {sigma . k} of sign flips.
// The separable Hartley coefficients S are split into parity components T_B
// (odd in the axes of B), the multiplier into its jointly-even parity
// components Psi_E, and the true-Fourier product is formed per component:
//   T'_C = sum_{|E| even} (-1)^{|E|/2 + |E & C|} Psi_E T_{E ^ C}.
__global__ void k_psi_f64(Dims d, const DevState* st, int stage, double* b0, double* b1) {
  const int par = (st->f.cur + stage) & 1;
  double* X = par ? b1 : b0;
  const int n = d.nx;
  long long reps = 1;
  int H[MAXN];
  for (int a = 0; a < n; ++a) { H[a] = d.N[a] / 2 + 1; reps *= H[a]; }
  const int l = st->f.l;
  const double g = st->f.g;
  const int exact = st->f.exact;
  const int ns = 1 << n;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < reps;
       r += (long long)gridDim.x * blockDim.x) {
    int k[MAXN];
    long long t = r;
    for (int a = n - 1; a >= 0; --a) { k[a] = (int)(t % H[a]); t /= H[a]; }
    double S[16], Psi[16];
    long long idx[16];
    for (int s = 0; s < ns; ++s) {
      long long off = 0;
      double kap2[MAXN], kt[MAXN];
      for (int a = 0; a < n; ++a) {
        const int N = d.N[a];
        const int ka = ((s >> a) & 1) ? (N - k[a]) % N : k[a];
        off = off * N + ka;
        const int w = ka < N / 2 ? ka : ka - N;      // fftshift(-N/2 : N/2-1)
        const double kap = two_pi * w / N;
        kap2[a] = kap * kap;
        kt[a] = (2 * ka == N) ? 0.0 : kap;           // first-derivative: Nyquist omitted
      }
      idx[s] = off;
      S[s] = X[off];
      double den = 1.0, ex = 0.0;
      for (int q = 0; q < l; ++q) {
        double e = 0.0;
        for (int a = 0; a < n; ++a) e += st->pa[q][a] * kap2[a];
        if (n > 1) e += st->pb[q][0] * kt[0] * kt[1];
        if (n > 2) e += st->pb[q][1] * kt[0] * kt[2] + st->pb[q][2] * kt[1] * kt[2];
        if (n > 3) e += st->pb[q][3] * kt[0] * kt[3] + st->pb[q][4] * kt[1] * kt[3] + st->pb[q][5] * kt[2] * kt[3];
        den *= 1.0 + e;
        ex += e;
      }
      Psi[s] = exact ? exp(-ex) : 1.0 / den;
    }
    double T[16], Pe[16], Tp[16];
    for (int B = 0; B < ns; ++B) {
      double tb = 0.0, pe = 0.0;
      for (int s = 0; s < ns; ++s) {
        const double chi = (popc((unsigned)(B & s)) & 1) ? -1.0 : 1.0;
        tb += chi * S[s];
        pe += chi * Psi[s];
      }
      T[B] = tb / ns;
      Pe[B] = pe / ns;
    }
    for (int C = 0; C < ns; ++C) {
      double acc = 0.0;
      for (int E = 0; E < ns; ++E) {
        const int pe = popc((unsigned)E);
        if (pe & 1) continue;
        const int sgn = ((pe / 2) + popc((unsigned)(E & C))) & 1;
        acc += (sgn ? -1.0 : 1.0) * Pe[E] * T[E ^ C];
      }
      Tp[C] = acc * g;
    }
    for (int s = 0; s < ns; ++s) {
      double v = 0.0;
      for (int C = 0; C < ns; ++C) v += ((popc((unsigned)(C & s)) & 1) ? -1.0 : 1.0) * Tp[C];
      X[idx[s]] = v;
    }
  }
}

// Moment partial sums of a float32 weight array (prior of the tensor-core path).
__global__ void k_moments_f32(Dims d, const float* X, double* partials) {
  __shared__ double sm[32 * kMomentSlots];
  double acc[kMomentSlots] = {};
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    unflatten(d, p, j);
    double u[MAXN];
    for (int a = 0; a < d.nx; ++a) u[a] = j[a] - 0.5 * (d.N[a] - 1);
    acc_moments(acc, (double)X[p], u, d.nx);
  }
  block_sum<kMomentSlots>(acc, sm, partials + blockIdx.x * kMomentSlots);
}

__global__ void k_moments_f64(Dims d, const DevState* st, int stage, const double* b0,
                              const double* b1, double* partials) {
  __shared__ double sm[32 * kMomentSlots];
  const int par = (st->f.cur + stage) & 1;
  const double* X = par ? b1 : b0;
  double acc[kMomentSlots] = {};
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    unflatten(d, p, j);
    double u[MAXN];
    for (int a = 0; a < d.nx; ++a) u[a] = j[a] - 0.5 * (d.N[a] - 1);
    acc_moments(acc, X[p], u, d.nx);
  }
  block_sum<kMomentSlots>(acc, sm, partials + blockIdx.x * kMomentSlots);
}

// Initial weights: Gaussian prior sampled on the initial frame (unnormalised).
__global__ void k_prior_f64(Dims d, const DevState* st, const double* P0inv, const double* m0,
                            double* X) {
  const int n = d.nx;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    unflatten(d, p, j);
    double dx[MAXN];
    for (int a = 0; a < n; ++a) {
      double x = st->f.c[a];
      for (int b = 0; b < n; ++b) x += st->f.M[a * n + b] * (j[b] - 0.5 * (d.N[b] - 1));
      dx[a] = x - m0[a];
    }
    double q = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) q += dx[a] * P0inv[a * n + b] * dx[b];
    X[p] = exp(-0.5 * q);
  }
}

// Scale the current weights by pscale into a float64 output buffer.
__global__ void k_export_f64(Dims d, const DevState* st, const double* b0, const double* b1,
                             double* out) {
  const double* X = st->f.cur ? b1 : b0;
  const double ps = st->f.pscale;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x)
    out[p] = ps * X[p];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int grid_for(long long work, int threads, int cap) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

int fp64_partials_blocks(const Dims& d) { return grid_for(d.P, 256, 1024); }

void launch_prior_f64(const Dims& d, const DevState* st, const double* P0inv, const double* m0,
                      double* X, cudaStream_t s) {
  k_prior_f64<<<grid_for(d.P, 256, 4096), 256, 0, s>>>(d, st, P0inv, m0, X);
}

void launch_moments_f64(const Dims& d, DevState* st, int stage, double* b0, double* b1,
                        double* partials, int flip, int use_pending, const double* pend,
                        cudaStream_t s) {
  const int nb = fp64_partials_blocks(d);
  k_moments_f64<<<nb, 256, 0, s>>>(d, st, stage, b0, b1, partials);
  k_finalize<<<1, 256, 0, s>>>(d, st, partials, nb, flip, use_pending, pend);
}

void launch_moments_f32(const Dims& d, DevState* st, const float* X, double* partials,
                        cudaStream_t s) {
  const int nb = fp64_partials_blocks(d);
  k_moments_f32<<<nb, 256, 0, s>>>(d, X, partials);
  k_finalize<<<1, 256, 0, s>>>(d, st, partials, nb, 0, 0, nullptr);
}

void launch_meas_f64(const Dims& d, const MeasParams& mp, DevState* st, double* b0, double* b1,
                     double* partials, cudaStream_t s) {
  cudaMemsetAsync(&st->emin_bits, 0xff, sizeof(unsigned long long), s);
  k_meas_emin_f64<<<grid_for(d.P, 256, 1024), 256, 0, s>>>(d, mp, st);
  const int nb = fp64_partials_blocks(d);
  k_meas_apply_f64<<<nb, 256, 0, s>>>(d, mp, st, b0, b1, partials);
  k_finalize<<<1, 256, 0, s>>>(d, st, partials, nb, 1, 0, nullptr);
}

void launch_time_f64(const Dims& d, const TimeConsts& tc, DevState* st, double* b0, double* b1,
                     double* partials, double* pend, double* const* interp,
                     double* const* hfwd, double* const* hinv, double* scratch, cudaStream_t s) {
  const int n = d.nx;
  k_frame<<<1, MAXL, 0, s>>>(tc, st, pend);
  for (int a = 0; a < n; ++a)
    k_build_interp_f64<<<grid_for((long long)d.N[a] * d.N[a], 256, 1 << 20), 256, 0, s>>>(
        d, st, a, interp[a]);
  k_realign_f64<<<grid_for(d.P, 256, 4096), 256, 0, s>>>(d, st, b0, b1, tc.realign_mode);
  if (tc.realign_mode == PMF_REALIGN_SHEAR && n == 3 && scratch) {
    int Nmax = 0, Nmin = 1 << 30;
    for (int a = 0; a < 3; ++a) {
      Nmax = d.N[a] > Nmax ? d.N[a] : Nmax;
      Nmin = d.N[a] < Nmin ? d.N[a] : Nmin;
    }
    const size_t smem = sizeof(double) * (4 * (size_t)Nmax + 2);
    cudaFuncSetAttribute(k_shear3_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    double* pc = scratch + d.P;   // pass coefficients after the intermediate grid
    const unsigned lines = (unsigned)(d.P / Nmin);   // enough for the pass with the most lines
    k_shear3_setup<<<1, 1, 0, s>>>(st, pc);
    for (int pass = 0; pass < 3; ++pass)
      k_shear3_f64<<<lines, 128, smem, s>>>(d, st, pc, pass, b0, b1, scratch);
  }
  if (tc.realign_mode == PMF_REALIGN_SHEAR && n == 4 && scratch) {
    int Nmax = 0, Nmin = 1 << 30;
    for (int a = 0; a < 4; ++a) {
      Nmax = d.N[a] > Nmax ? d.N[a] : Nmax;
      Nmin = d.N[a] < Nmin ? d.N[a] : Nmin;
    }
    const size_t smem = sizeof(double) * (4 * (size_t)Nmax + 2);
    cudaFuncSetAttribute(k_shear4_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    double* pc = scratch + d.P;   // pass coefficients after the intermediate grid
    const unsigned lines = (unsigned)(d.P / Nmin);
    k_shear4_setup<<<1, 1, 0, s>>>(st, pc);
    for (int pass = 0; pass < 4; ++pass)
      k_shear4_f64<<<lines, 128, smem, s>>>(d, st, pc, pass, b0, b1, scratch);
  }
  if (tc.realign_mode == PMF_REALIGN_SHEAR && n == 2 && scratch) {
    const int Nmax = d.N[0] > d.N[1] ? d.N[0] : d.N[1];
    const size_t smem = sizeof(double) * (4 * (size_t)Nmax + 2);
    cudaFuncSetAttribute(k_shear_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // pass 1 runs over the old nodes of axis p, pass 2 over the new nodes of axis q;
    // both axis counts are launched and surplus CTAs of the shorter axis exit
    k_shear_f64<<<Nmax, 128, smem, s>>>(d, st, 1, b0, b1, scratch);
    k_shear_f64<<<Nmax, 128, smem, s>>>(d, st, 2, b0, b1, scratch);
  }
  int stage = 1;
  auto gemm = [&](int a, const double* W) {
    const int N = d.N[a];
    long long inner = 1, outer = 1;
    for (int m = a + 1; m < n; ++m) inner *= d.N[m];
    for (int m = 0; m < a; ++m) outer *= d.N[m];
    dim3 blk(16, 16);
    dim3 grd;
    if (inner == 1) {
      grd = dim3((N + 15) / 16, (unsigned)((d.P / N + 15) / 16), 1);
    } else {
      grd = dim3((unsigned)((inner + 15) / 16), (N + 15) / 16, (unsigned)outer);
    }
    k_axis_gemm_f64<<<grd, blk, 0, s>>>(d, a, W, st, stage, b0, b1);
    ++stage;
  };
  for (int a = 0; a < n; ++a) gemm(a, interp[a]);
  for (int a = 0; a < n; ++a) gemm(a, hfwd[a]);
  long long reps = 1;
  for (int a = 0; a < n; ++a) reps *= d.N[a] / 2 + 1;
  k_psi_f64<<<grid_for(reps, 128, 4096), 128, 0, s>>>(d, st, stage, b0, b1);
  for (int a = 0; a < n; ++a) gemm(a, hinv[a]);
  launch_moments_f64(d, st, stage, b0, b1, partials, stage & 1, 1, pend, s);
}

void launch_frame(const TimeConsts& tc, DevState* st, double* pend, cudaStream_t s) {
  k_frame<<<1, MAXL, 0, s>>>(tc, st, pend);
}

void launch_export_f64(const Dims& d, const DevState* st, const double* b0, const double* b1,
                       double* out, cudaStream_t s) {
  k_export_f64<<<grid_for(d.P, 256, 4096), 256, 0, s>>>(d, st, b0, b1, out);
}

}  // namespace pmf
