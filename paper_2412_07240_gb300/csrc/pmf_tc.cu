// Fused tensor-core path: one CTA carries one 2-D filter through a whole epoch
// with its grid resident on chip.
//
//   measurement update (eq. filt)   registers: likelihood relative to the frame
//                                   centre, exponent minimum, moments
//   frame (float64, one thread)     regrid decision, diffusion coefficients
//   R1  regrid along axis 1         tcgen05 GEMM, periodic-sinc matrix I1
//   F1  Hartley along axis 1        tcgen05 GEMM, H1 (TMA bulk copy)
//   R0  regrid along axis 0         tcgen05 GEMM, operand read MN-major
//   F0  Hartley along axis 0        tcgen05 GEMM, H0
//   Psi diffusion multiplier and trace factor with the separable-to-2-D
//       Hartley parity fix-up (Sec. V-B algorithm steps 2-4)
//   V0  inverse along axis 0        tcgen05 GEMM, H0 (still resident)
//   V1  inverse along axis 1        tcgen05 GEMM, H1, operand MN-major
//   normalisation and moments (step 6), weights written back to HBM.
//
// Every GEMM is D[128 lines x Nout] = A[128 x K] * W[Nout x K]^T with M = 128
// lines (unused lines ignored), the accumulator in TMEM and both operands in
// shared memory in the no-swizzle canonical layout of 8-row x 16-byte core
// matrices, 16 core matrices per 8-row block.  The epilogue thread that owns
// TMEM lane r writes row r of the next operand, so the operand of the next
// GEMM along the other axis is the same bytes read MN-major: no transposes.
//
// Precisions: FP16X3 / BF16X3 split each operand into hi + lo 16-bit planes and
// issue hi*hi + hi*lo + lo*hi (FP32 accumulate); FP16 operands carry a
// power-of-two scale per stage (max |value| -> 2^14).  BF16X6 (2-D filters
// only) splits each operand into hi + mid + lo BF16 planes and issues the six
// products of combined order at most two, smallest first (hi*lo, lo*hi,
// mid*mid, hi*mid, mid*hi, hi*hi).  TF32 issues one kind::tf32 product on
// float32 planes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "pmf_device.cuh"
#include "pmf_model.cuh"
#include "pmf_kernels.cuh"
#include "pmf_tc.cuh"
#include "pmf_tcops.cuh"

namespace pmf {

namespace {

constexpr uint32_t kTmemCols = 128;

// Size classes of the fused kernel: C is the largest axis a CTA holds.
//   C = 128: 512 threads (4 TMEM lane quadrants x 4 column groups), 16-bit
//            operand planes of 128 x 128, one CTA per SM;
//   C = 64 : 256 threads (4 quadrants x 2 column groups), planes of 64 x 64
//            (the lanes >= 64 of every accumulator are garbage, so the A
//            planes keep 64 rows);
//   C = 96 : 256 threads, planes of 96 x 96.
// Dynamic shared memory: the A operand planes, the W operand planes and a
// float32 staging tile of C rows x (C + 4) floats (the padding makes row
// access conflict-free).  Where three regions do not fit, the staging tile
// shares a region:
//   alias (class 96): the tile lies in the W region.  The weights are staged
//     there before the first matrix is built, the spectrum is written there
//     after the forward transforms and H0 is copied in again for the
//     inverse; the multilinear gather and the band-limited re-alignment use
//     the A region as scratch.  Two CTAs per SM.
//   sina (classes 128 and 64 in BF16X6, three planes per operand, in the
//     planned kernel; the single-filter kernel keeps the alias, where the
//     warps that convert the weights run beside warp 0's float64 frame
//     decision): the tile lies in the A region (class 64: four CTAs per SM
//     instead of three).  The weights arrive there and the spectrum is written
//     there once the MMAs that read A have completed; each conversion of the
//     tile into the A planes goes through registers (all threads read their
//     part, synchronise, then write).  W is then free whenever the tile is
//     live, so it holds I1 while the weights arrive, keeps H0 across the
//     multiplier and is the re-alignments' scratch.  (In class 96 the
//     registers of the in-place conversion cost more than the reload saves.)
template <int P, int C, bool kPlanned = true>
struct Smem {
  static constexpr int threads = C == 128 ? 512 : 256;
  static constexpr int sstr = C + 4;
  static constexpr bool alias = C == 96 || (!kPlanned && C == 128 && Fmt<P>::planes == 3);
  static constexpr bool sina = kPlanned && (C == 128 || C == 64) && Fmt<P>::planes == 3;
  static constexpr int offA = 0;
  static constexpr int abytes = Fmt<P>::planes * Lay<P, C, C>::plane;
  static constexpr int sbytes = C * sstr * 4;
  static constexpr int wbytes = Fmt<P>::planes * Lay<P, C>::wplane;
  static constexpr int scr = C * (C + 2) * 4;   // band-limited re-alignment scratch
  static constexpr int areg = alias ? (abytes > scr ? abytes : scr) : sina && sbytes > abytes ? sbytes : abytes;
  static constexpr int wreg = alias ? (wbytes > sbytes ? wbytes : sbytes) : sina && scr > wbytes ? scr : wbytes;
  static constexpr int offW = (areg + 1023) / 1024 * 1024;
  static constexpr int offS = alias ? offW : sina ? offA : offW + (wreg + 1023) / 1024 * 1024;
  static constexpr int bytes = alias || sina ? offW + wreg : offS + sbytes;
  // work items (8 columns of a row) per thread of an in-place conversion
  static constexpr int items = (C * C / 8 + threads - 1) / threads;
};
constexpr int kThreads = 512;                // the single-filter kernel (class 128)
static_assert(Smem<PMF_PREC_BF16X6, 128>::bytes <= 200 * 1024 && Smem<PMF_PREC_BF16X6, 128, false>::bytes <= 200 * 1024,
              "class-128 BF16X6 planes and static state fit");

// One filter launched alone: everything by value in the kernel parameters.
struct FusedJob {
  DevState* st;
  float* buf0;
  float* buf1;
  const uint8_t* hart[2];   // per axis: Hartley planes (hi then lo for 16-bit formats)
  const float* sctab[2];    // per axis: (cos, sin)(pi m / N), m = -N..N
  int N0, N1, do_meas, do_time, fft;
  MeasParams mp;
  TimeConsts tc;
};

// What one CTA works on: the filter's resident data and this epoch's request.
struct FusedView {
  DevState* st;
  float* buf0;
  float* buf1;
  const uint8_t* hart[2];
  const float* sctab[2];
  int N0, N1, do_meas, do_time;
  const MeasParams* mp;     // measurement model
  const double* z;          // measurement of this epoch
  const TimeConsts* tc;     // model constants of this time update
  const struct BatchPlan* plan;   // planned transform kernel: the front kernel's results
  int fft;                  // Hartley transforms in shared memory instead of GEMMs
};

// The constants of the update are kept in shared memory only by the kernels
// that compute the frame (the fused kernel and the batch front kernel); the
// planned transform kernel reads the front kernel's results instead.
template <bool kKeep>
struct TcHolder {
  TimeConsts tc;
};
template <>
struct TcHolder<false> {};

// Static shared memory of one CTA (threads T, largest axis C; kTc: the time
// constants; kRows: the regrid rows and axis tables of the fused kernel).
template <int T, int C, bool kTc, bool kRows = kTc>
struct SharedT : TcHolder<kTc> {
  static constexpr int kT = T;
  static constexpr int kStr = C + 4;   // staging row stride (floats)
  MeasParams mp;
  FrameState fs;           // working copy of the filter's frame state
  uint64_t mbar_mma, mbar_tma;
  uint32_t tmem;
  int abort, degenerate, realign_mode, wmax_bits;
  float redf[2][T / 32];
  DF redm[T / 32][6];
  double tot[10];
  double pend[24];
  double Mpi[9];
  float pa[MAXL][2];
  float pb[MAXL];
  float g, ps, gsc;
  // frame-relative measurement constants
  float mc[2], mM[4], mr0[3], mRinv[9], mH[6], mcn;
  // per axis: regrid rows and the (cos, sin)(pi m / N) table, m = -N..N, in
  // the kernels that compute the frame; the planned transform kernel reads
  // the plan's rows and the axis tables from global memory instead (its
  // static shared memory then admits one more CTA per SM in classes 96 / 64)
  RegridRowsT<kRows ? C : 1> rows[2];
  float sct[2][kRows ? 2 * (2 * C + 1) : 1];
};

// What the batch front kernel hands to the planned transform kernel for one
// filter and epoch: whether the time update runs, the pending frame after the
// move (finalisation input), the sub-step coefficients in float32, the trace
// factor and the regrid rows of both axes (unused after a re-alignment).
struct BatchPlan {
  double pend[24];
  float pa[MAXL][2];
  float pb[MAXL];
  float g, gsc;
  int ok;
  float wmax;   // max |weight| the front kernel wrote (before the scale pscale); -1 if it wrote none
  RegridRowsT<128> rows[2];
};

// Block max of non-negative per-thread values (result in every thread).
template <class SH>
__device__ __forceinline__ float block_max(SH& sh, float v, int slot) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh.redf[slot][threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.0f;
#pragma unroll
  for (int w = 0; w < SH::kT / 32; ++w) m = fmaxf(m, sh.redf[slot][w]);
  return m;
}

template <class SH>
__device__ __forceinline__ float block_min(SH& sh, float v, int slot) {
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh.redf[slot][threadIdx.x >> 5] = v;
  __syncthreads();
  float m = INFINITY;
#pragma unroll
  for (int w = 0; w < SH::kT / 32; ++w) m = fminf(m, sh.redf[slot][w]);
  return m;
}

// Sum the per-thread moment sums over the block into sh.tot ({S0, S1[3],
// S2[6]} layout, float64); valid in warp 0 after the call.  The sums stay in
// double-float through both the warp and the cross-warp reduction; six lanes
// of warp 0 convert the totals to float64 (GB300 issues float64 at a small
// fraction of the float32 rate, so no per-warp or single-thread float64 loop).
template <class SH>
__device__ __forceinline__ void block_moments(SH& sh, const Moments& m) {
  constexpr int kThreads = SH::kT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DF a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = m.s[i];
    for (int o = 16; o; o >>= 1) {
      DF b{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
      a[i] = df_add(a[i], b);
    }
  }
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 6; ++i) sh.redm[warp][i] = a[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      a[i] = lane < kThreads / 32 ? sh.redm[lane][i] : DF{0.0f, 0.0f};
      // the whole warp, so that lanes 0..5 below all hold the totals
      for (int o = 16; o; o >>= 1) {
        DF b{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
        a[i] = df_add(a[i], b);
      }
    }
    // lane i < 6 converts accumulator i; {S0, S1_0, S1_1, S2_00, S2_01, S2_11}
    // go to tot[0, 1, 2, 4, 5, 7], the n_x = 3 slots are zero
    DF mine = a[0];
#pragma unroll
    for (int i = 1; i < 6; ++i)
      if (lane == i) mine = a[i];
    const int slot = lane < 3 ? lane : lane == 3 ? 4 : lane == 4 ? 5 : lane == 5 ? 7 : lane == 6 ? 3
                   : lane == 7 ? 6 : lane;
    if (lane < 6) sh.tot[slot] = (double)mine.hi + (double)mine.lo;
    else if (lane < 10) sh.tot[slot] = 0.0;
    __syncwarp();
  }
}

// Frame-relative measurement constants of one update (registers).
struct MeasK {
  float c0, c1, m00, m01, m10, m11, r00, r01, h00, h01, h10, h11, ri00, ri01, ri11, cn;
  int kind, nz;
};

template <class SH>
__device__ __forceinline__ MeasK meas_k(const SH& sh) {
  return MeasK{sh.mc[0], sh.mc[1], sh.mM[0], sh.mM[1], sh.mM[2], sh.mM[3], sh.mr0[0], sh.mr0[1], sh.mH[0],
               sh.mH[1], sh.mH[2], sh.mH[3], sh.mRinv[0], sh.mRinv[1], sh.mRinv[3], sh.mcn, sh.mp.kind, sh.mp.nz};
}

// 1/2 r^T R^{-1} r with the residual formed relative to the frame centre c:
// d = M u, and r = r0 - (change of h from c to c + d), r0 = z - h(c) in float64;
// linear h: r = r0 - H d; range: |c + d| - |c| = (2 c.d + |d|^2) / (|c + d| + |c|).
__device__ __forceinline__ float meas_e(const MeasK& k, float u0, float u1) {
  const float d0 = k.m00 * u0 + k.m01 * u1, d1 = k.m10 * u0 + k.m11 * u1;
  float r0, r1 = 0.0f;
  if (k.kind == PMF_MEAS_LINEAR) {
    r0 = k.r00 - (k.h00 * d0 + k.h01 * d1);
    if (k.nz > 1) r1 = k.r01 - (k.h10 * d0 + k.h11 * d1);
  } else {
    const float x0 = k.c0 + d0, x1 = k.c1 + d1;
    const float den = sqrtf(x0 * x0 + x1 * x1) + k.cn;
    const float num = 2.0f * (k.c0 * d0 + k.c1 * d1) + d0 * d0 + d1 * d1;
    r0 = k.r00 - (den > 0.0f ? __fdividef(num, den) : 0.0f);
  }
  float e = r0 * k.ri00 * r0;
  if (k.nz > 1) e += 2.0f * r0 * k.ri01 * r1 + r1 * k.ri11 * r1;
  return 0.5f * e;
}

// Exponent shift of a linear measurement without a pass over the grid: the
// minimum over the grid box |u_m| <= a_m of the convex quadratic
// e(u) = 1/2 (r0 - G u)^T Ri (r0 - G u), G = H M (the continuous form of
// meas_e), by the interior minimiser or, outside the box, the minima along
// its four edges.  The grid point nearest the minimiser lies at most half a
// cell away per axis (on a face or at a corner, exactly on it along the
// normal), so the grid's minimum exceeds the result by at most
// (Hq00 + Hq11 + 2 |Hq01|) / 8, Hq = G^T Ri G; below 40 the shifted
// likelihood exp(shift - e) neither overflows (shift <= e) nor leaves the
// largest weights near float32's range limit.  Returns false beyond that
// (sharp likelihoods on coarse grids: the caller takes the grid minimum).
// Every thread computes the same float32 operations, so all hold the same
// shift.  The shift cancels in the normalisation (eq. filt).
__device__ __forceinline__ bool linear_eshift(const MeasK& k, float a0, float a1, float* shift) {
  const bool two = k.nz > 1;
  const float g00 = k.h00 * k.m00 + k.h01 * k.m10, g01 = k.h00 * k.m01 + k.h01 * k.m11;
  const float g10 = two ? k.h10 * k.m00 + k.h11 * k.m10 : 0.0f, g11 = two ? k.h10 * k.m01 + k.h11 * k.m11 : 0.0f;
  const float r00 = k.r00, r01 = two ? k.r01 : 0.0f;
  const float q00 = k.ri00, q01 = two ? k.ri01 : 0.0f, q11 = two ? k.ri11 : 0.0f;
  // Ri G (2 x 2), Hq = G^T Ri G, b = G^T Ri r0, c = 1/2 r0^T Ri r0
  const float p00 = q00 * g00 + q01 * g10, p01 = q00 * g01 + q01 * g11;
  const float p10 = q01 * g00 + q11 * g10, p11 = q01 * g01 + q11 * g11;
  const float h00 = g00 * p00 + g10 * p10, h01 = g00 * p01 + g10 * p11, h11 = g01 * p01 + g11 * p11;
  const float b0 = p00 * r00 + p10 * r01, b1 = p01 * r00 + p11 * r01;
  const float c = 0.5f * (r00 * (q00 * r00 + q01 * r01) + r01 * (q01 * r00 + q11 * r01));
  if (!((h00 + h11 + 2.0f * fabsf(h01)) * 0.125f <= 40.0f)) return false;
  auto ev = [&](float u0, float u1) { return 0.5f * (h00 * u0 * u0 + 2.0f * h01 * u0 * u1 + h11 * u1 * u1) - b0 * u0 - b1 * u1 + c; };
  const float det = h00 * h11 - h01 * h01;
  if (det > 1e-6f * (h00 * h11 + 1e-30f)) {
    const float u0 = (h11 * b0 - h01 * b1) / det, u1 = (h00 * b1 - h01 * b0) / det;
    if (fabsf(u0) <= a0 && fabsf(u1) <= a1) {
      *shift = ev(u0, u1);
      return isfinite(*shift);
    }
  }
  // minimum on the boundary: each edge is a 1-D quadratic in the free coordinate
  float best = INFINITY;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int fixed = e >> 1;                        // axis held at +-a
    const float uf = (e & 1) ? (fixed ? a1 : a0) : -(fixed ? a1 : a0);
    const float af = fixed ? a0 : a1;                // range of the free coordinate
    const float hoo = fixed ? h00 : h11, hfo = h01, bo = fixed ? b0 : b1;
    float t = hoo > 0.0f ? (bo - hfo * uf) / hoo : 0.0f;
    t = fminf(fmaxf(t, -af), af);
    float v = fixed ? ev(t, uf) : ev(uf, t);
    if (!(hoo > 0.0f)) v = fminf(fixed ? ev(-af, uf) : ev(uf, -af), fixed ? ev(af, uf) : ev(uf, af));
    best = fminf(best, v);
  }
  *shift = best;
  return isfinite(best);
}

// Staging rows r < nr, columns < nc (a multiple of 8) -> operand planes
// (scaled by s).  Consecutive threads take consecutive rows, eight columns
// each: in the core-matrix layout 8 consecutive rows of 8 columns are 128
// contiguous bytes, written with one 16-byte store per thread and plane.
template <int P, int C = 128>
__device__ __forceinline__ void stage_to_operand(uint8_t* A, const float* S, int nr, int nc, float s,
                                                 int t0, int tstep) {
  const int q8 = nc / 8;
  for (int t = t0; t < nr * q8; t += tstep) {
    const int r = t % nr, c = (t / nr) * 8;
    const float* src = S + r * (C + 4) + c;
    store8<P, C, false, C>(A, r, c, *(const float4*)src, *(const float4*)(src + 4), s);
  }
}

// The same in place, when the staging tile lies inside the A region: each of
// the T threads reads its (at most kItems) row segments into registers, the
// block synchronises, then the planes are written.  The caller makes the
// tile's writes visible before and fences the planes for the MMA after.
template <int P, int C, int kItems, int T>
__device__ __forceinline__ void stage_to_operand_inplace(uint8_t* A, const float* S, int nr, int nc, float s) {
  const int q8 = nc / 8, tot = nr * q8;
  float4 v[kItems][2];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int t = threadIdx.x + k * T;
    if (t < tot) {
      const int r = t % nr, c = (t / nr) * 8;
      const float* src = S + r * (C + 4) + c;
      v[k][0] = *(const float4*)src;
      v[k][1] = *(const float4*)(src + 4);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int t = threadIdx.x + k * T;
    if (t < tot) store8<P, C, false, C>(A, t % nr, (t / nr) * 8, v[k][0], v[k][1], s);
  }
}

template <int T, int C>
__device__ __forceinline__ float stage_max(const float* S, int nr, int nc) {
  const int q4 = nc / 4;
  float m = 0.0f;
  for (int t = threadIdx.x; t < nr * q4; t += T) {
    const int r = t / q4, c = (t % q4) * 4;
    m = amax4(m, *(const float4*)(S + r * (C + 4) + c));
  }
  return m;
}

// Out-of-line copies of the helpers called from several places of the epoch:
// a kernel that runs once on cold caches fetches their code once (the batch
// kernel, whose CTAs follow each other on an SM, keeps them inline).
template <class SH>
__device__ __noinline__ void block_moments_out(SH& sh, const Moments& m) { block_moments(sh, m); }
__device__ __noinline__ bool finalize_warp_out(FrameState* st, const double* tot, int use_pending,
                                               const double* pend) {
  return finalize_warp<2>(st, tot, use_pending, pend);
}
template <int P, int C, int R>
__device__ __noinline__ void build_interp_out(const RegridRowsT<R>& rows, uint8_t* W, int N, const float* sctab,
                                              float sw, int realign, int t0, int tstep) {
  build_interp<P, C, R>(rows, W, N, sctab, sw, realign, t0, tstep);
}
template <int R>
__device__ __noinline__ void regrid_rows_out(RegridRowsT<R>& rows, double rs, double rd, int N, int t0, int tstep) {
  regrid_rows(rows, rs, rd, N, t0, tstep);
}
template <int P, int C>
__device__ __noinline__ void issue_stage_out(uint32_t tmem, uint32_t a_base, int a_mn, uint32_t w_base, int nout,
                                             int K, uint32_t mbar) {
  issue_stage<P, C, C>(tmem, a_base, a_mn, w_base, nout, K, mbar);
}
template <int P, int C>
__device__ __noinline__ void stage_to_operand_out(uint8_t* A, const float* S, int nr, int nc, float s, int t0,
                                                  int tstep) {
  stage_to_operand<P, C>(A, S, nr, nc, s, t0, tstep);
}

// Band-limited re-alignment on the staging tile (shear mode): the two
// line-wise passes of the float64 path (k_shear_f64: the trigonometric
// interpolant of eq. interFreq of each line, evaluated at that line's affine
// positions) in float32, all lines of a pass at once; the lines' DFT
// coefficients go to C ((lines) x (N + 2) floats, the free operand regions).
// Twiddles e^{2 pi i r / N} come exactly from the (cos, sin)(pi m / N) tables;
// an evaluation point x = m + f takes e^{2 pi i x / N} from the table entry of
// m and sincospi of f, then powers by recurrence.  Returns this thread's
// max |weight| of the re-aligned tile.
template <class SH>
__device__ __noinline__ float shear_stage(const SH& sh, float* S, float* C, int N0, int N1, const float* sct0,
                                          const float* sct1) {
  constexpr int kThreads = SH::kT, kSStr = SH::kStr;
  const FrameState& fs = sh.fs;
  // pass order making pass 1's line-dependent shift the smaller: |B_10 / B_00| <= |B_01 / B_11|
  const int p = fabs(fs.B[2]) * fabs(fs.B[3]) <= fabs(fs.B[1]) * fabs(fs.B[0]) ? 0 : 1, q = 1 - p;
  const double Bpp = fs.B[p * 2 + p], Bpq = fs.B[p * 2 + q], Bqp = fs.B[q * 2 + p], Bqq = fs.B[q * 2 + q];
  const float r1 = (float)(Bqp / Bpp), d1 = (float)((Bpp * Bqq - Bpq * Bqp) / Bpp);
  const float bp = (float)fs.b[p], bq = (float)fs.b[q], fpp = (float)Bpp, fpq = (float)Bpq;
  const int Np = p ? N1 : N0, Nq = q ? N1 : N0;
  auto at = [&](int ip, int iq) { return p == 0 ? ip * kSStr + iq : iq * kSStr + ip; };
  float smax = 0.0f;
  for (int pass = 1; pass <= 2; ++pass) {
    const int L = pass == 1 ? Np : Nq, N = pass == 1 ? Nq : Np, H = N / 2;
    const float* sct = (pass == 1 ? q : p) ? sct1 : sct0;
    const float rN = 1.0f / (float)N;
    for (int it = threadIdx.x; it < L * (H + 1); it += kThreads) {
      const int line = it / (H + 1), sidx = it - line * (H + 1);
      float re = 0.0f, im = 0.0f;
      int r = 0;
      for (int j = 0; j < N; ++j) {
        const float fj = pass == 1 ? S[at(line, j)] : S[at(j, line)];
        const int m = 2 * r <= N ? 2 * r : 2 * r - 2 * N;   // 2 pi r / N = pi m / N
        re = fmaf(fj, sct[2 * (m + N)], re);
        im = fmaf(-fj, sct[2 * (m + N) + 1], im);
        r += sidx;
        if (r >= N) r -= N;
      }
      C[line * (N + 2) + 2 * sidx] = re * rN;
      C[line * (N + 2) + 2 * sidx + 1] = im * rN;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < L * N; it += kThreads) {
      const int line = it / N, t = it - line * N;
      const float ul = line - 0.5f * (L - 1), ut = t - 0.5f * (N - 1);
      const float pos = pass == 1 ? fmaf(d1, ut, fmaf(r1, ul - bp, bq)) : fmaf(fpp, ut, fmaf(fpq, ul, bp));
      float v = 0.0f;
      if (fabsf(pos) <= 0.5f * N) {
        const float x = pos + 0.5f * (N - 1);
        const float mf = rintf(x), fr = x - mf;
        int mi = (int)mf % N;
        if (mi < 0) mi += N;
        const int mm = 2 * mi <= N ? 2 * mi : 2 * mi - 2 * N;
        const float cm = sct[2 * (mm + N)], sm = sct[2 * (mm + N) + 1];
        float sf, cf;
        sincospif(2.0f * fr * rN, &sf, &cf);
        const float wr = cm * cf - sm * sf, wi = cm * sf + sm * cf;   // e^{2 pi i x / N}
        const float* X = C + line * (N + 2);
        float zr = 1.0f, zi = 0.0f;
        v = X[0];
        for (int k = 1; k < H; ++k) {
          const float nr = zr * wr - zi * wi;
          zi = zr * wi + zi * wr;
          zr = nr;
          v += 2.0f * (X[2 * k] * zr - X[2 * k + 1] * zi);
        }
        v += X[2 * H] * ((((int)mf) & 1) ? -cospif(fr) : cospif(fr));   // cos(pi x)
      }
      if (pass == 1) S[at(line, t)] = v;
      else S[at(t, line)] = v;
      if (pass == 2) smax = fmaxf(smax, fabsf(v));
    }
    __syncthreads();
  }
  return smax;
}

// Diffusion multiplier and trace factor in the Hartley domain (Sec. V-B
// algorithm steps 2-4) on the staging tile T[k1][k0], one thread per orbit
// {(+-k0, +-k1)}: with S_s the four separable coefficients (bit 0 of s flips
// k0, bit 1 flips k1), T_B their parity components and Psi_E those of the
// jointly even multiplier (E = 0 even-even, E = 3 odd-odd),
//   T'_C = Psi_0 T_C - (-1)^{|3 & C|} Psi_3 T_{3 ^ C},
// then back to the separable coefficients; gsc = trace factor / (N0 N1).
// Psi(k0, k1) and Psi(-k0, k1) differ only in the sign of the cross term.
template <class SH>
__device__ void psi_stage(const SH& sh, float* S, int N0, int N1, int l, int exact) {
  constexpr int kThreads = SH::kT, kSStr = SH::kStr;
  const int H0n = N0 / 2 + 1, H1n = N1 / 2 + 1;
  const float w0s = 6.28318530717958647692f / (float)N0, w1s = 6.28318530717958647692f / (float)N1;
  // r = k1 H0n + k0: (r + 1/2) / H0n is at least 1/(2 H0n) away from an integer,
  // so the float product truncates to k1 exactly (r < 2^13)
  const float rH0 = 1.0f / (float)H0n;
  for (int r = threadIdx.x; r < H0n * H1n; r += kThreads) {
    const int k1 = (int)(((float)r + 0.5f) * rH0);
    const int k0 = r - k1 * H0n;
    const int i0[2] = {k0, k0 ? N0 - k0 : 0};
    const int i1[2] = {k1, k1 ? N1 - k1 : 0};
    float Sv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) Sv[s] = S[i1[s >> 1] * kSStr + i0[s & 1]];
    const float k0f = w0s * (float)k0, k1f = w1s * (float)k1;
    const float q0 = k0f * k0f, q1 = k1f * k1f;
    // first-derivative coefficients: zero at the Nyquist index
    const float qx = ((2 * k0 == N0) ? 0.0f : k0f) * ((2 * k1 == N1) ? 0.0f : k1f);
    float den0 = 1.0f, den1 = 1.0f, ex0 = 0.0f, ex1 = 0.0f;
    for (int qq = 0; qq < l; ++qq) {
      const float b = sh.pa[qq][0] * q0 + sh.pa[qq][1] * q1;
      const float e0 = b + sh.pb[qq] * qx, e1 = b + sh.pb[qq] * (-qx);
      den0 *= 1.0f + e0;
      den1 *= 1.0f + e1;
      ex0 += e0;
      ex1 += e1;
    }
    const float P0 = exact ? expf(-ex0) : __frcp_rn(den0), P1 = exact ? expf(-ex1) : __frcp_rn(den1);
    const float pe0 = 0.5f * (P0 + P1), pe3 = 0.5f * (P0 - P1);
    float T[4];
#pragma unroll
    for (int B = 0; B < 4; ++B) {
      float tb = 0.0f;
#pragma unroll
      for (int s = 0; s < 4; ++s) tb += ((__popc(B & s) & 1) ? -1.0f : 1.0f) * Sv[s];
      T[B] = 0.25f * tb;
    }
    float Tp[4];
#pragma unroll
    for (int C = 0; C < 4; ++C) {
      const float sg3 = ((1 + __popc(3 & C)) & 1) ? -1.0f : 1.0f;
      Tp[C] = (pe0 * T[C] + sg3 * pe3 * T[3 ^ C]) * sh.gsc;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float o = 0.0f;
#pragma unroll
      for (int C = 0; C < 4; ++C) o += ((__popc(C & s) & 1) ? -1.0f : 1.0f) * Tp[C];
      S[i1[s >> 1] * kSStr + i0[s & 1]] = o;
    }
  }
}

// ---- shared-memory form of the per-axis Hartley transforms ------------------
// (the FFT form of steps 1 and 5 of the Sec. V-B algorithm, an alternative to
// the tensor-core contraction for axis sizes 2^a 3^b)

// e^{-2 pi i a / N}, 0 <= a < N, from the (cos, sin)(pi m / N) table (m = -N..N).
__device__ __forceinline__ float2 twiddle(const float* sct, int a, int N) {
  const int m = 2 * a <= N ? 2 * a : 2 * a - 2 * N;
  return make_float2(sct[2 * (m + N)], -sct[2 * (m + N) + 1]);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Hartley transforms of L real lines of length N (L even) held in the float32
// tile S, element (l, j) at S[l * ls + j * es], in place.  Two lines form one
// complex line z = x_{2p} + i x_{2p+1}; its DFT Z (radix-3 then radix-2
// Stockham passes, self-sorting, between X and Y, L/2 x N float2 each, neither
// aliasing S) gives both transforms, F_{2p,k} = (Z_k + conj Z_{N-k}) / 2,
// F_{2p+1,k} = (Z_k - conj Z_{N-k}) / (2i), and H = Re F - Im F (cas = cos + sin).
// Ends with a block barrier.
template <int T>
__device__ void fht_lines(float* S, int ls, int es, int L, int N, float2* X, float2* Y, const float* sct) {
  const int half = L / 2, tot = half * N;
  for (int idx = threadIdx.x; idx < tot; idx += T) {
    const int p = idx / N, j = idx - p * N;
    X[idx] = make_float2(S[(2 * p) * ls + j * es], S[(2 * p + 1) * ls + j * es]);
  }
  __syncthreads();
  float2* src = X;
  float2* dst = Y;
  int s = 1, rem = N;
  const float h3 = 0.86602540378443864676f;   // sin(2 pi / 3)
  while (rem > 1) {
    const int r = rem % 3 == 0 ? 3 : 2;
    const int n = N / s, m = n / r;            // this pass: sub-length n, butterflies m x s per line
    const int per = m * s;
    for (int idx = threadIdx.x; idx < half * per; idx += T) {
      const int line = idx / per, b = idx - line * per;
      const int pp = b / s, q = b - pp * s;
      const float2* x = src + line * N + q + s * pp;
      float2* y = dst + line * N + q + s * r * pp;
      if (r == 2) {
        const float2 a0 = x[0], a1 = x[s * m];
        y[0] = make_float2(a0.x + a1.x, a0.y + a1.y);
        y[s] = cmul(make_float2(a0.x - a1.x, a0.y - a1.y), twiddle(sct, (pp * s) % N, N));
      } else {
        const float2 a0 = x[0], a1 = x[s * m], a2 = x[2 * s * m];
        const float2 bsum = make_float2(a1.x + a2.x, a1.y + a2.y), d = make_float2(a1.x - a2.x, a1.y - a2.y);
        const float2 c = make_float2(a0.x - 0.5f * bsum.x, a0.y - 0.5f * bsum.y);
        y[0] = make_float2(a0.x + bsum.x, a0.y + bsum.y);
        // a0 + a1 w + a2 w^2 (w = e^{-2 pi i / 3}) = c - i h3 d, and its conjugate pair
        y[s] = cmul(make_float2(c.x + h3 * d.y, c.y - h3 * d.x), twiddle(sct, (pp * s) % N, N));
        y[2 * s] = cmul(make_float2(c.x - h3 * d.y, c.y + h3 * d.x), twiddle(sct, (2 * pp * s) % N, N));
      }
    }
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
    s *= r;
    rem /= r;
  }
  for (int idx = threadIdx.x; idx < tot; idx += T) {
    const int p = idx / N, k = idx - p * N;
    const float2 zk = src[p * N + k], zm = src[p * N + (k ? N - k : 0)];
    // F1 = (zk + conj zm) / 2, F2 = -i (zk - conj zm) / 2
    const float f1r = 0.5f * (zk.x + zm.x), f1i = 0.5f * (zk.y - zm.y);
    const float f2r = 0.5f * (zk.y + zm.y), f2i = -0.5f * (zk.x - zm.x);
    S[(2 * p) * ls + k * es] = f1r - f1i;
    S[(2 * p + 1) * ls + k * es] = f2r - f2i;
  }
  __syncthreads();
}

// The planned kernel's copy of the front kernel's sub-step coefficients (the
// multiplier reads them for every orbit); the regrid rows stay in the plan.
template <class SH>
__device__ __forceinline__ void plan_coeffs(SH& sh, const BatchPlan* pl, int l) {
  for (int q = threadIdx.x; q < l; q += SH::kT) {
    sh.pa[q][0] = pl->pa[q][0];
    sh.pa[q][1] = pl->pa[q][1];
    sh.pb[q] = pl->pb[q];
  }
}

// One filter's epoch in one CTA (size class C).  kOut: the single-filter
// kernel (helpers called from several places out of line).  kPlan: the
// planned transform kernel of a batch (time update only; the measurement
// update, moments, frame decision, sub-step coefficients and regrid rows come
// from the front kernel through job.plan).
template <int P, bool kOut, bool kPlan = false, int C = 128>
__device__ void fused2d(const FusedView& job, uint8_t* smem) {
  using SM = Smem<P, C, kPlan>;
  using SH = SharedT<kPlan ? SM::threads : kThreads, C, !kPlan>;
  constexpr int kThreads = SH::kT, kSStr = SH::kStr, kGroups = kThreads / 128;
  constexpr int kNV = C / kGroups / 4;          // float4 accumulator columns per thread
  // columns [c0, c0 + ncol) of an accumulator of nout columns (a multiple of
  // 16) held by column group cg: whole groups of 8, so that every row segment
  // is a run of 16-byte operand stores (nout = 48 over 4 groups: 16 + 16 + 16 + 0)
  auto cols = [&](int nout, int g, int& c0, int& ncol) {
    const int per = ((nout >> 3) + kGroups - 1) / kGroups * 8;
    c0 = g * per;
    ncol = nout - c0 < per ? (nout > c0 ? nout - c0 : 0) : per;
  };
  constexpr bool kSina = SM::sina;      // staging tile inside the A region
  constexpr bool kAlias = SM::alias;    // staging tile in the W region
  static_assert(!kSina || SM::items * kThreads * 8 >= C * C, "in-place conversion items");
  // only FP16 operands carry a scale (op_scale is 1 otherwise), so only they
  // need the block maxima of the stage outputs
  constexpr bool kScaled = P == PMF_PREC_FP16X3;
  __shared__ SH sh;
  if (!job.do_meas && !job.do_time) return;   // nothing requested for this filter
  if constexpr (kPlan) {
    if (!job.plan->ok) return;                 // degenerate measurement update: no time update
  }
  DevState* st = job.st;
  FrameState& fs = sh.fs;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, cg = tid >> 7;     // TMEM lane and column group of this thread
  const int N0 = job.N0, N1 = job.N1;
  uint8_t* A = smem + SM::offA;
  uint8_t* W = smem + SM::offW;
  float* S = (float*)(smem + SM::offS);
  const uint32_t mb_mma = su32(&sh.mbar_mma), mb_tma = su32(&sh.mbar_tma);
  uint32_t ph_mma = 0, ph_tma = 0;
  const float sw = P == PMF_PREC_FP16X3 ? 16384.0f : 1.0f;   // scale of the matrix operands
  // the axis tables and the matrices I_a: from shared memory, or (planned
  // kernel) from the axis tables and the plan's rows in global memory
  auto sct = [&](int a) -> const float* {
    if constexpr (kPlan) return job.sctab[a];
    else return sh.sct[a];
  };
  // staging tile -> A planes by the whole block (in place in the sina layout)
  auto to_operand = [&](int nr, int nc, float sc) {
    if constexpr (kSina) stage_to_operand_inplace<P, C, SM::items, kThreads>(A, S, nr, nc, sc);
    else if constexpr (kOut) stage_to_operand_out<P, C>(A, S, nr, nc, sc, threadIdx.x, kThreads);
    else stage_to_operand<P, C>(A, S, nr, nc, sc, threadIdx.x, kThreads);
  };
  auto build_I = [&](int a, int Nm, int realign_, uint8_t* Wd) {
    if constexpr (kPlan) build_interp<P, C, 128>(job.plan->rows[a], Wd, Nm, job.sctab[a], sw, realign_, threadIdx.x, kThreads);
    else if constexpr (kOut) build_interp_out<P, C, C>(sh.rows[a], Wd, Nm, sh.sct[a], sw, realign_, threadIdx.x, kThreads);
    else build_interp<P, C, C>(sh.rows[a], Wd, Nm, sh.sct[a], sw, realign_, threadIdx.x, kThreads);
  };
  constexpr int kFsWords = sizeof(FrameState) / 8;

  for (int i = tid; i < kFsWords; i += kThreads)
    ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  if (job.do_time) {
    if constexpr (!kPlan) {
      const int words = tc_words(job.tc);   // up to the sub-step rows this update uses
      for (int i = tid; i < words; i += kThreads)
        ((unsigned long long*)&sh.tc)[i] = ((const unsigned long long*)job.tc)[i];
    }
    if (tid == 0) sh.realign_mode = job.tc->realign_mode;
    if constexpr (!kPlan)
      for (int a = 0; a < 2; ++a) {
        const int n = 2 * (2 * (a ? N1 : N0) + 1);
        for (int i = tid; i < n; i += kThreads) sh.sct[a][i] = job.sctab[a][i];
      }
  }
  if (job.do_meas) {
    for (int i = tid; i < (int)(sizeof(MeasParams) / 8); i += kThreads)
      ((unsigned long long*)&sh.mp)[i] = ((const unsigned long long*)job.mp)[i];
    __syncthreads();
    if (tid < PMF_MAX_NZ) sh.mp.z[tid] = job.z[tid];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_mma));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_tma));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh.abort = 0;
    sh.degenerate = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = sh.tmem;
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  // ---- weights -> staging rows j0, columns j1 (bulk copies, one per row) ----
  const int cur = fs.cur;
  const float* in = cur ? job.buf1 : job.buf0;
  float* out = cur ? job.buf0 : job.buf1;
  const int q1 = N1 / 4, np4 = N0 * q1;
  if (job.do_time && warp == 2 && (tid & 31) < 2) {
    // the Hartley planes of both axes are needed after the measurement update
    const int a = tid & 1, Nm = a ? N1 : N0;
    prefetch_l2(job.hart[a], (uint32_t)Nm * (uint32_t)(Lay<P, C>::rowblk / 8) * Fmt<P>::planes);
  }
  if (warp == 1) {
    // rows are N1 * 4 bytes (a multiple of 64) at 16-byte aligned addresses
    if (tid == 32) expect_tx(mb_tma, (uint32_t)(N0 * N1 * 4));
    __syncwarp();
    for (int r = tid - 32; r < N0; r += 32)
      bulk_load(su32(S + r * kSStr), in + (size_t)r * N1, (uint32_t)(N1 * 4), mb_tma);
  }
  float smax = 0.0f;      // max |weight| (operand scale of the first GEMM)
  float sa_first = 1.0f;  // scale of the R1 operand
  int realign = 0, l = 0, exact = 0;
  // Planned kernel, separable regrid: the front kernel left the max of the
  // weights it wrote, so the pscale goes into the R1 operand scale instead of
  // a scaling pass over the tile (fold); with W free (no alias) the plan's
  // coefficients and rows and the matrix I1 are set up while the weights
  // arrive (early).
  bool fold = false, early = false;
  float wps = 1.0f;   // pscale folded into the R1 operand
  if constexpr (kPlan) {
    fold = job.plan->wmax >= 0.0f && !fs.realign;
    early = fold && !kAlias;   // W is free while the weights arrive
    if (early) {
      plan_coeffs(sh, job.plan, fs.l);
      build_I(1, N1, 0, W);
    }
  }

  // ---- measurement update (eq. filt) ----
  if (!kPlan && job.do_meas) {
    if (tid == 0) {
      const MeasParams& mp = sh.mp;
      const double c0 = fs.c[0], c1 = fs.c[1];
      sh.mc[0] = (float)c0;
      sh.mc[1] = (float)c1;
      for (int i = 0; i < 4; ++i) sh.mM[i] = (float)fs.M[i];
      for (int i = 0; i < mp.nz * mp.nz; ++i) sh.mRinv[i] = (float)mp.Rinv[i];
      if (mp.kind == PMF_MEAS_LINEAR) {
        for (int i = 0; i < mp.nz; ++i) {
          sh.mr0[i] = (float)(mp.z[i] - (mp.H[i * 2] * c0 + mp.H[i * 2 + 1] * c1));
          for (int b = 0; b < 2; ++b) sh.mH[i * 2 + b] = (float)mp.H[i * 2 + b];
        }
      } else {
        const double cn = sqrt(c0 * c0 + c1 * c1);
        sh.mcn = (float)cn;
        sh.mr0[0] = (float)(mp.z[0] - cn);
      }
    }
    __syncthreads();
    // exponents into the (still free) W region while the weights arrive (the
    // A region when the weights are staged in W)
    const MeasK mk = meas_k(sh);
    // t = r q1 + c/4 < 2^12: (t + 1/2) / q1 is at least 1/(2 q1) from an
    // integer, so the float product truncates to r exactly
    const float rq1 = 1.0f / (float)q1;
    float4* E = (float4*)(kAlias ? A : W);
    float emin = INFINITY;
    for (int t = tid; t < np4; t += kThreads) {
      const int r = (int)(((float)t + 0.5f) * rq1), c = (t - r * q1) * 4;
      const float u0 = r - 0.5f * (N0 - 1), u1 = c - 0.5f * (N1 - 1);
      const float4 e = make_float4(meas_e(mk, u0, u1), meas_e(mk, u0, u1 + 1.0f), meas_e(mk, u0, u1 + 2.0f),
                                   meas_e(mk, u0, u1 + 3.0f));
      E[t] = e;
      emin = fminf(emin, fminf(fminf(e.x, e.y), fminf(e.z, e.w)));
    }
    emin = block_min(sh, emin, 0);
    // the batch front kernel's shift for a linear measurement (same steps as
    // there; the shift cancels in the normalisation)
    if (mk.kind == PMF_MEAS_LINEAR) {
      float shift;
      if (linear_eshift(mk, 0.5f * (N0 - 1), 0.5f * (N1 - 1), &shift)) emin = shift;
    }
    if (__syncthreads_or(!mbar_wait(mb_tma, ph_tma))) {
      if (tid == 0) fs.status = PMF_ERR_TIMEOUT;
      goto done;
    }
    ph_tma ^= 1;
    const float ps = (float)fs.pscale;
    Moments mo;
    mo.zero();
    // a thread keeps one group of four columns (the step is a multiple of q1)
    // and sums its rows in float32 per column; one double-float add per slot
    const int tmax = (kThreads / q1) * q1;
    if (tid < tmax) {
      float ca[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cb[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int t = tid; t < np4; t += tmax) {
        const int r = (int)(((float)t + 0.5f) * rq1), c = (t - r * q1) * 4;
        const float u0 = r - 0.5f * (N0 - 1);
        float4 x = *(const float4*)(S + r * kSStr + c);
        const float4 e = E[t];
        x.x = (x.x * ps) * __expf(emin - e.x);
        x.y = (x.y * ps) * __expf(emin - e.y);
        x.z = (x.z * ps) * __expf(emin - e.z);
        x.w = (x.w * ps) * __expf(emin - e.w);
        *(float4*)(S + r * kSStr + c) = x;
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float xu = xs[i] * u0;
          ca[i] += xs[i];
          cb[i] += xu;
          cc[i] = fmaf(xu, u0, cc[i]);
        }
        smax = amax4(smax, x);
      }
      mo.add_cols4(ca, cb, cc, (tid % q1) * 4 - 0.5f * (N1 - 1));
    }
    if constexpr (kOut) block_moments_out(sh, mo);
    else block_moments(sh, mo);
  } else {
    if (__syncthreads_or(!mbar_wait(mb_tma, ph_tma))) {
      if (tid == 0) fs.status = PMF_ERR_TIMEOUT;
      goto done;
    }
    ph_tma ^= 1;
    const float ps = (float)fs.pscale;
    if (fold) {
      smax = job.plan->wmax * ps;   // = the max of the scaled weights (rounding is monotone)
      wps = ps;
    } else {
      for (int t = tid; t < np4; t += kThreads) {
        const int r = t / q1, c = (t % q1) * 4;
        float4 x = *(const float4*)(S + r * kSStr + c);
        x.x *= ps;
        x.y *= ps;
        x.z *= ps;
        x.w *= ps;
        *(float4*)(S + r * kSStr + c) = x;
        smax = amax4(smax, x);
      }
    }
  }
  {
    // Thread 0 finalises the moments and (time update) computes the frame in
    // float64 while warps 1.. convert the staged weights into the R1 operand,
    // which needs neither.  (With fold, every thread has the weights it reads
    // from its own wait on the copies, and smax is the same in all of them.)
    const float sa0 = fold ? op_scale<P>(smax) : op_scale<P>(block_max(sh, smax, 1));
    if (warp == 0 && kPlan) {
      // the front kernel decided the frame: pending frame and trace factor
      const BatchPlan* pl = job.plan;
      if (tid < 24) sh.pend[tid] = pl->pend[tid];
      if (tid == 0) {
        sh.g = pl->g;
        sh.gsc = pl->gsc;
      }
      __syncwarp();
    } else if (warp == 0) {
      bool ok = true;
      if (job.do_meas) {
        if constexpr (kOut) ok = finalize_warp_out(&fs, sh.tot, 0, nullptr);
        else ok = finalize_warp<2>(&fs, sh.tot, 0, nullptr);
        if (tid == 0) {
          if (!ok) {
            sh.degenerate = 1;
          } else {
            sh.ps = (float)fs.pscale;   // the staged weights times ps are normalised
            fs.pscale = 1.0;
            fs.S0 = 1.0 / fs.V;
          }
        }
        __syncwarp();
      }
      if constexpr (!kPlan) if (ok && job.do_time) {
        frame_warp<2>(sh.tc, &fs, sh.pend, sh.Mpi);
        if (tid == 0) {
          sh.g = (float)fs.g;
          sh.gsc = (float)(fs.g / ((double)N0 * (double)N1));
        }
      }
    } else if (job.do_time && !kSina) {
      // (in the sina layout the tile is converted in place once the regrid
      // is known, by the whole block: a re-alignment reads it first)
      if constexpr (kOut) stage_to_operand_out<P, C>(A, S, N0, N1, sa0, tid - 32, kThreads - 32);
      else stage_to_operand<P, C>(A, S, N0, N1, sa0 * wps, tid - 32, kThreads - 32);
    }
    __syncthreads();
    if (sh.degenerate) goto done;
    if (!job.do_time) {
      const float ps = sh.ps;
      for (int t = tid; t < np4; t += kThreads) {
        const int r = t / q1, c = (t % q1) * 4;
        float4 x = *(const float4*)(S + r * kSStr + c);
        x.x *= ps;
        x.y *= ps;
        x.z *= ps;
        x.w *= ps;
        *(float4*)(out + (size_t)r * N1 + c) = x;
      }
      if (tid == 0) fs.cur = cur ^ 1;
      goto done;
    }
    sa_first = sa0;
  }

  {
    // ---- sub-step coefficients, regrid rows of both axes (or re-alignment) ----
    realign = fs.realign;
    l = fs.l;
    exact = fs.exact;
    if constexpr (kPlan) {
      if (!early) plan_coeffs(sh, job.plan, l);
    } else {
      for (int q = tid; q < l; q += kThreads) {
        double pa[4], pb[6];
        frame_substep<2>(sh.tc, sh.Mpi, q, pa, pb);
        sh.pa[q][0] = (float)pa[0];
        sh.pa[q][1] = (float)pa[1];
        sh.pb[q] = (float)pb[0];
      }
    }
    if (realign && sh.realign_mode == PMF_REALIGN_SHEAR) {
      // band-limited re-alignment in place on the staging tile
      smax = shear_stage(sh, S, (float*)(kSina ? W : A), N0, N1, sct(0), sct(1));   // scratch beside the tile
      sa_first = op_scale<P>(block_max(sh, smax, 0));
      to_operand(N0, N1, sa_first);
    } else if (realign) {
      // multilinear re-alignment: gather into the (free) W region, or the A
      // region when the staging tile lives in W, copy back
      float* G = (float*)(kAlias ? A : W);
      const int npts = N0 * N1;
      for (int p = tid; p < npts; p += kThreads) {
        const int r = p / N1, c = p - r * N1;
        const double u0 = r - 0.5 * (N0 - 1), u1 = c - 0.5 * (N1 - 1);
        // old-grid index coordinates in float64 (positions span +-N/2 nodes)
        const double z0 = fma(fs.B[0], u0, fma(fs.B[1], u1, fs.b[0] + 0.5 * (N0 - 1)));
        const double z1 = fma(fs.B[2], u0, fma(fs.B[3], u1, fs.b[1] + 0.5 * (N1 - 1)));
        const double f0 = floor(z0), f1 = floor(z1);
        const float w0 = (float)(z0 - f0), w1 = (float)(z1 - f1);
        const int i0 = (int)fmax(fmin(f0, 1e6), -1e6), i1 = (int)fmax(fmin(f1, 1e6), -1e6);
        float s = 0.0f;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int a = i0 + (cc & 1), b = i1 + (cc >> 1);
          const float wt = ((cc & 1) ? w0 : 1.0f - w0) * ((cc >> 1) ? w1 : 1.0f - w1);
          if (a >= 0 && a < N0 && b >= 0 && b < N1) s += wt * S[a * kSStr + b];
        }
        G[p] = s;
      }
      __syncthreads();
      smax = 0.0f;
      for (int p = tid; p < npts; p += kThreads) {
        const int r = p / N1, c = p - r * N1;
        S[r * kSStr + c] = G[p];
        smax = fmaxf(smax, fabsf(G[p]));
      }
      sa_first = op_scale<P>(block_max(sh, smax, 0));
      to_operand(N0, N1, sa_first);
    } else {
      // axis 1 by the first half of the block, axis 0 by the second
      const int a = tid < kThreads / 2 ? 1 : 0;
      const int t0 = tid - (a ? 0 : kThreads / 2);
      if constexpr (kPlan) {
        // the rows stay in the plan
      } else if constexpr (kOut) {
        regrid_rows_out(sh.rows[a], fs.rs[a], fs.rd[a], a ? N1 : N0, t0, kThreads / 2);
      } else {
        regrid_rows(sh.rows[a], fs.rs[a], fs.rd[a], a ? N1 : N0, t0, kThreads / 2);
      }
    }
    __syncthreads();
    // the sina layout converts the staged weights now (separable regrid)
    if constexpr (kSina)
      if (!realign) to_operand(N0, N1, sa_first * wps);
  }

  {
    // ---- the matrix I1; the R1 operand is already written ----
    float sa = sa_first;
    if (!early) build_I(1, N1, realign, W);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_after_sync();
      if constexpr (kOut) issue_stage_out<P, C>(tmem, su32(A), 0, su32(W), N1, N1, mb_mma);
      else issue_stage<P, C, C>(tmem, su32(A), 0, su32(W), N1, N1, mb_mma);
    }
    float inv_scale = 1.0f / (sa * sw);

    if (!kSina && !kAlias && job.fft) {
      // FFT form: the regrid of each axis stays a tensor-core GEMM whose
      // epilogue writes float32 to the staging tile; the four Hartley
      // transforms run in shared memory (fht_lines, scratch in W and A).
      float2* X = (float2*)W;
      float2* Y = (float2*)A;
      for (int g = 0; g < 2; ++g) {
        // g = 0: R1 (lanes j0, columns k1); g = 1: R0 (lanes k1, columns j0)
        const bool okw = mbar_wait(mb_mma, ph_mma);
        ph_mma ^= 1;
        if (__syncthreads_or(!okw)) {
          if (tid == 0) sh.abort = 1;
          break;
        }
        tc_after_sync();
        const int nlane = g ? N1 : N0, nout = g ? N0 : N1;
        int c0, ncol;
        cols(nout, cg, c0, ncol);
        float4 v[8];
        tmem_ld_cols(tlane + c0, ncol, v);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (4 * j < ncol && row < nlane) {
            const float4 x = v[j];
            *(float4*)(S + row * kSStr + c0 + 4 * j) =
                make_float4(x.x * inv_scale, x.y * inv_scale, x.z * inv_scale, x.w * inv_scale);
          }
        tc_before_sync();
        __syncthreads();
        if (g == 0) {
          // F1 along axis 1 (rows of the tile), then the operand of R0 (read MN-major)
          fht_lines<kThreads>(S, kSStr, 1, N0, N1, X, Y, sct(1));
          if constexpr (kScaled) sa = op_scale<P>(block_max(sh, stage_max<kThreads, C>(S, N0, N1), 0));
          if constexpr (P == PMF_PREC_TF32) {
            const int q4 = N1 / 4;
            for (int t = tid; t < N0 * q4; t += kThreads) {
              const int r = t % N0, c = (t / N0) * 4;
              store4_t<C>(A, r, c, *(const float4*)(S + r * kSStr + c), sa);
            }
          } else {
            stage_to_operand<P, C>(A, S, N0, N1, sa, tid, kThreads);
          }
          build_I(0, N0, realign, W);
          fence_async_smem();
          __syncthreads();
          if (tid == 0) {
            tc_after_sync();
            issue_stage<P, C, C>(tmem, su32(A), P != PMF_PREC_TF32, su32(W), N0, N0, mb_mma);
          }
          inv_scale = 1.0f / (sa * sw);
        }
      }
      if (!sh.abort) {
        // F0 along axis 0 (rows of the tile T[k1][.]), the multiplier, V0, then
        // V1 along axis 1 (columns of the tile)
        fht_lines<kThreads>(S, kSStr, 1, N1, N0, X, Y, sct(0));
        psi_stage(sh, S, N0, N1, l, exact);
        __syncthreads();
        fht_lines<kThreads>(S, kSStr, 1, N1, N0, X, Y, sct(0));
        fht_lines<kThreads>(S, 1, kSStr, N0, N1, X, Y, sct(1));
        // final weights: tile [j1][j0] -> row j0 of the output, moments
        Moments mo;
        mo.zero();
        const int q4 = N1 / 4;
        for (int t = tid; t < N0 * q4; t += kThreads) {
          const int j0 = t / q4, j1 = (t - j0 * q4) * 4;
          const float4 x = make_float4(S[j1 * kSStr + j0], S[(j1 + 1) * kSStr + j0], S[(j1 + 2) * kSStr + j0],
                                       S[(j1 + 3) * kSStr + j0]);
          *(float4*)(out + (size_t)j0 * N1 + j1) = x;
          const float u0 = j0 - 0.5f * (N0 - 1), u1 = j1 - 0.5f * (N1 - 1);
          const float a0 = x.x + x.y + x.z + x.w;
          const float a1 = x.y + 2.0f * x.z + 3.0f * x.w;
          const float a2 = x.y + 4.0f * x.z + 9.0f * x.w;
          mo.add_row(a0, fmaf(u1, a0, a1), fmaf(u1, fmaf(u1, a0, 2.0f * a1), a2), u0);
        }
        block_moments(sh, mo);
      }
    } else {
    // Stages after R1: F1, R0, F0, V0, V1.  Epilogue of GEMM `stage` (0 = R1)
    // writes the operand of GEMM stage+1.
    for (int stage = 0; stage < 6; ++stage) {
      const bool ok = mbar_wait(mb_mma, ph_mma);
      ph_mma ^= 1;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) sh.abort = 1;
        break;
      }
      tc_after_sync();
      // matrix of the next GEMM: F1 <- H1, R0 <- I0 (built below), F0 <- H0,
      // V0 keeps H0, V1 <- H1.  The MMA that read W has completed, and the
      // epilogue does not touch W, so the copy runs behind the epilogue.
      int mat = -1;
      if (stage == 0 || stage == 4) mat = 1;
      if (stage == 2) mat = 0;
      // the spectrum goes to the staging tile, which shares W in the alias
      // layout: H0 again for V0 once the tile has been read (below)
      if (kAlias && stage == 3) mat = 0;
      if (tid == 0 && mat >= 0 && !(kAlias && stage == 3)) {
        const int Nm = mat == 0 ? N0 : N1;
        const uint32_t pbytes = (uint32_t)Nm * (uint32_t)(Lay<P, C>::rowblk / 8);
        expect_tx(mb_tma, pbytes * Fmt<P>::planes);
        for (int pl = 0; pl < Fmt<P>::planes; ++pl)
          bulk_load(su32(W) + pl * Lay<P, C>::wplane, job.hart[mat] + (size_t)pl * pbytes, pbytes, mb_tma);
      }
      // accumulator of GEMM `stage`: valid lanes and columns
      const int nlane = (stage == 0 || stage == 1 || stage == 5) ? N0 : N1;
      const int nout = (stage <= 1 || stage == 5) ? N1 : N0;
      int c0, ncol;   // this thread's columns
      cols(nout, cg, c0, ncol);
      const bool lane_ok = row < nlane;
      float4 v[kNV];
      if constexpr (kNV == 8) {
        tmem_ld_cols(tlane + c0, ncol, v);
      } else if constexpr (kNV == 4) {
        tmem_ld_cols4(tlane + c0, ncol, v);
      } else {
        // up to 48 columns: 32 + 16
        float4 va[8], vb[4];
        tmem_ld_cols(tlane + c0, ncol < 32 ? ncol : 32, va);
        tmem_ld_cols4(tlane + c0 + 32, ncol > 32 ? ncol - 32 : 0, vb);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = va[j];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[8 + j] = vb[j];
      }
#pragma unroll
      for (int j = 0; j < kNV; ++j) {
        v[j].x *= inv_scale;
        v[j].y *= inv_scale;
        v[j].z *= inv_scale;
        v[j].w *= inv_scale;
      }
      if (stage == 5) {
        // final weights: row j0 = lane, columns j1, straight to HBM (each
        // thread writes its contiguous, 16-byte aligned row segment), and moments
        Moments mo;
        mo.zero();
        const float u0 = row - 0.5f * (N0 - 1);
        float* orow = out + (size_t)row * N1 + c0;
        float ra = 0.0f, rb = 0.0f, rc = 0.0f;   // this row segment: sum x, x u1, x u1^2
#pragma unroll
        for (int j = 0; j < kNV; ++j)
          if (4 * j < ncol && lane_ok) {
            *(float4*)(orow + 4 * j) = v[j];
            const float4 x = v[j];
            const float u1 = (c0 + 4 * j) - 0.5f * (N1 - 1);
            const float a0 = x.x + x.y + x.z + x.w;
            const float a1 = x.y + 2.0f * x.z + 3.0f * x.w;
            const float a2 = x.y + 4.0f * x.z + 9.0f * x.w;
            ra += a0;
            rb += fmaf(u1, a0, a1);
            rc += fmaf(u1, fmaf(u1, a0, 2.0f * a1), a2);
          }
        mo.add_row(ra, rb, rc, u0);
        tc_before_sync();
        if constexpr (kOut) block_moments_out(sh, mo);
        else block_moments(sh, mo);
        break;
      }
      if (stage == 3) {
        // F0 finished: spectrum T[k1][k0] -> staging, multiplier, operand of V0
#pragma unroll
        for (int j = 0; j < kNV; ++j)   // valid lanes only: the staging tile has C rows
          if (4 * j < ncol && lane_ok) *(float4*)(S + row * kSStr + c0 + 4 * j) = v[j];
        tc_before_sync();
        __syncthreads();
        psi_stage(sh, S, N0, N1, l, exact);
        __syncthreads();
        if constexpr (kScaled) sa = op_scale<P>(block_max(sh, stage_max<kThreads, C>(S, N1, N0), stage & 1));
        to_operand(N1, N0, sa);
      } else {
        if constexpr (kScaled) {
          float m = 0.0f;
#pragma unroll
          for (int j = 0; j < kNV; ++j) m = amax4(m, v[j]);
          sa = op_scale<P>(block_max(sh, lane_ok ? m : 0.0f, stage & 1));
        }
        // R0 and V1 read this operand MN-major; TF32 gets it written transposed
        const bool tr = P == PMF_PREC_TF32 && (stage == 1 || stage == 4);
        if (tr) {
          // transposed, lanes become columns: a lane >= C would land in the
          // next row block of the size-64 layout, so invalid lanes are skipped
#pragma unroll
          for (int j = 0; j < kNV; ++j)
            if (4 * j < ncol && lane_ok) store4_t<C>(A, row, c0 + 4 * j, v[j], sa);
        } else if (C == 128 || row < C) {
          // the planes keep C rows: lanes >= C (garbage) are not stored; ncol
          // is a multiple of 8, so the float4 columns pair up
#pragma unroll
          for (int j = 0; j < kNV; j += 2)
            if (4 * j < ncol) store8<P, C, false, C>(A, row, c0 + 4 * j, v[j], v[j + 1], sa);
        }
        tc_before_sync();
      }
      if (stage == 1) {
        __syncthreads();
        build_I(0, N0, realign, W);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_after_sync();
        bool ok2 = true;
        if (kAlias && stage == 3) {
          const uint32_t pbytes = (uint32_t)N0 * (uint32_t)(Lay<P, C>::rowblk / 8);
          expect_tx(mb_tma, pbytes * Fmt<P>::planes);
          for (int pl = 0; pl < Fmt<P>::planes; ++pl)
            bulk_load(su32(W) + pl * Lay<P, C>::wplane, job.hart[0] + (size_t)pl * pbytes, pbytes, mb_tma);
        }
        if (mat >= 0) ok2 = mbar_wait(mb_tma, ph_tma);
        if (!ok2) {
          sh.abort = 1;
        } else {
          // stage+1: F1 (K-major), R0 (MN), F0 (K), V0 (K), V1 (MN)
          const int a_mn = (P != PMF_PREC_TF32) && (stage == 1 || stage == 4);
          const int nn = (stage == 0 || stage == 4) ? N1 : N0;
          if constexpr (kOut) issue_stage_out<P, C>(tmem, su32(A), a_mn, su32(W), nn, nn, mb_mma);
          else issue_stage<P, C, C>(tmem, su32(A), a_mn, su32(W), nn, nn, mb_mma);
        }
      }
      if (mat >= 0) ph_tma ^= 1;
      inv_scale = 1.0f / (sa * sw);
      __syncthreads();
      if (sh.abort) break;
    }
    }   // GEMM form
    if (sh.abort) {
      if (tid == 0) fs.status = PMF_ERR_TIMEOUT;
      goto done;
    }

    // ---- normalisation on the advanced frame ----
    if (warp == 0) {
      bool ok;
      if constexpr (kOut) ok = finalize_warp_out(&fs, sh.tot, 1, sh.pend);
      else ok = finalize_warp<2>(&fs, sh.tot, 1, sh.pend);
      if (ok && tid == 0) fs.cur = cur ^ 1;
    }
  }

done:
  tc_before_sync();
  __syncthreads();
  for (int i = tid; i < kFsWords; i += kThreads)
    ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) k_fused2d(const __grid_constant__ FusedJob job) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const FusedView v{job.st, job.buf0, job.buf1, {job.hart[0], job.hart[1]}, {job.sctab[0], job.sctab[1]},
                    job.N0, job.N1, job.do_meas, job.do_time, &job.mp, job.mp.z, &job.tc, nullptr, job.fft};
  fused2d<P, true>(v, smem);
}

// Front kernel of a batched epoch (one CTA per filter, no operand tiles, so
// several CTAs share an SM and their float64 latency chains overlap): the
// measurement update (eq. filt) streamed through registers from the current
// weight buffer into the other one, the moments, the float64 regrid decision
// of the time update, its sub-step coefficients and the regrid rows of both
// axes, handed to the planned transform kernel through the filter's plan.
// The steps are those of the fused kernel (the exponents are recomputed
// instead of stored).
constexpr int kFrontThreads = 128;   // four warps, 48 registers: ten CTAs (filters) share an SM

__global__ void __launch_bounds__(kFrontThreads, 10) k_front2d(const FilterSlot* __restrict__ slots,
                                                              const StepItem* __restrict__ items,
                                                              const TimeConsts* __restrict__ tcs) {
  __shared__ SharedT<kFrontThreads, 128, true, false> sh;
  constexpr int kT = kFrontThreads;
  const StepItem& it = items[blockIdx.x];
  const FilterSlot& sl = slots[it.slot];
  const int do_meas = it.flags & 1, do_time = (it.flags >> 1) & 1;
  BatchPlan* plan = (BatchPlan*)sl.plan;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!do_meas && !do_time) {
    if (tid == 0) plan->ok = 0;
    return;
  }
  DevState* st = sl.st;
  FrameState& fs = sh.fs;
  const int N0 = sl.N0, N1 = sl.N1;
  constexpr int kFsWords = sizeof(FrameState) / 8;
  for (int i = tid; i < kFsWords; i += kT) ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  if (do_time) {
    const TimeConsts* tc = tcs ? tcs + blockIdx.x : sl.tc;
    const int words = tc_words(tc);
    for (int i = tid; i < words; i += kT) ((unsigned long long*)&sh.tc)[i] = ((const unsigned long long*)tc)[i];
  }
  if (do_meas)
    for (int i = tid; i < (int)(sizeof(MeasParams) / 8); i += kT)
      ((unsigned long long*)&sh.mp)[i] = ((const unsigned long long*)sl.mp)[i];
  if (tid == 0) {
    sh.degenerate = 0;
    sh.wmax_bits = 0;
  }
  __syncthreads();
  if (do_meas && tid < PMF_MAX_NZ) sh.mp.z[tid] = it.z[tid];
  __syncthreads();
  const int cur = fs.cur;
  const float* in = cur ? sl.buf1 : sl.buf0;
  float* out = cur ? sl.buf0 : sl.buf1;
  const int q1 = N1 / 4, np4 = N0 * q1;
  const float rq1 = 1.0f / (float)q1;
  if (do_meas) {
    if (tid == 0) {
      const MeasParams& mp = sh.mp;
      const double c0 = fs.c[0], c1 = fs.c[1];
      sh.mc[0] = (float)c0;
      sh.mc[1] = (float)c1;
      for (int i = 0; i < 4; ++i) sh.mM[i] = (float)fs.M[i];
      for (int i = 0; i < mp.nz * mp.nz; ++i) sh.mRinv[i] = (float)mp.Rinv[i];
      if (mp.kind == PMF_MEAS_LINEAR) {
        for (int i = 0; i < mp.nz; ++i) {
          sh.mr0[i] = (float)(mp.z[i] - (mp.H[i * 2] * c0 + mp.H[i * 2 + 1] * c1));
          for (int b = 0; b < 2; ++b) sh.mH[i * 2 + b] = (float)mp.H[i * 2 + b];
        }
      } else {
        const double cn = sqrt(c0 * c0 + c1 * c1);
        sh.mcn = (float)cn;
        sh.mr0[0] = (float)(mp.z[0] - cn);
      }
    }
    __syncthreads();
    const MeasK mk = meas_k(sh);
    float emin = INFINITY;
    // a linear measurement takes its exponent shift from the box minimum of
    // the quadratic; otherwise (or for a too sharp one) a pass over the grid
    if (!(mk.kind == PMF_MEAS_LINEAR && linear_eshift(mk, 0.5f * (N0 - 1), 0.5f * (N1 - 1), &emin))) {
      emin = INFINITY;
      for (int t = tid; t < np4; t += kT) {
        const int r = (int)(((float)t + 0.5f) * rq1), c = (t - r * q1) * 4;
        const float u0 = r - 0.5f * (N0 - 1), u1 = c - 0.5f * (N1 - 1);
        emin = fminf(emin, fminf(fminf(meas_e(mk, u0, u1), meas_e(mk, u0, u1 + 1.0f)),
                                 fminf(meas_e(mk, u0, u1 + 2.0f), meas_e(mk, u0, u1 + 3.0f))));
      }
      emin = block_min(sh, emin, 0);
    }
    const float ps = (float)fs.pscale;
    Moments mo;
    mo.zero();
    float wmax = 0.0f;
    const int tmax = (kT / q1) * q1;
    if (tid < tmax) {
      // float32 column sums over at most 16 rows, then one double-float add per slot
      float ca[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cb[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      int rows = 0;
      for (int t = tid; t < np4; t += tmax) {
        const int r = (int)(((float)t + 0.5f) * rq1), c = (t - r * q1) * 4;
        const float u0 = r - 0.5f * (N0 - 1), u1 = c - 0.5f * (N1 - 1);
        float4 x = *(const float4*)(in + (size_t)r * N1 + c);
        x.x = (x.x * ps) * __expf(emin - meas_e(mk, u0, u1));
        x.y = (x.y * ps) * __expf(emin - meas_e(mk, u0, u1 + 1.0f));
        x.z = (x.z * ps) * __expf(emin - meas_e(mk, u0, u1 + 2.0f));
        x.w = (x.w * ps) * __expf(emin - meas_e(mk, u0, u1 + 3.0f));
        *(float4*)(out + (size_t)r * N1 + c) = x;
        wmax = amax4(wmax, x);
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float xu = xs[i] * u0;
          ca[i] += xs[i];
          cb[i] += xu;
          cc[i] = fmaf(xu, u0, cc[i]);
        }
        if (++rows == 16) {
          mo.add_cols4(ca, cb, cc, (tid % q1) * 4 - 0.5f * (N1 - 1));
#pragma unroll
          for (int i = 0; i < 4; ++i) ca[i] = cb[i] = cc[i] = 0.0f;
          rows = 0;
        }
      }
      mo.add_cols4(ca, cb, cc, (tid % q1) * 4 - 0.5f * (N1 - 1));
    }
    block_moments(sh, mo);
    // non-negative floats order as their bit patterns: one shared atomic per warp
    for (int o = 16; o; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if ((tid & 31) == 0) atomicMax(&sh.wmax_bits, __float_as_int(wmax));
  }
  if (warp == 0) {
    bool ok = true;
    if (do_meas) {
      ok = finalize_warp<2>(&fs, sh.tot, 0, nullptr);
      if (tid == 0) {
        if (!ok) {
          sh.degenerate = 1;
        } else {
          sh.ps = (float)fs.pscale;   // the new weights times ps are normalised
          fs.pscale = 1.0;
          fs.S0 = 1.0 / fs.V;
          fs.cur = cur ^ 1;           // they live in the other buffer now
        }
      }
      __syncwarp();
    }
    if (ok && do_time) {
      frame_warp<2>(sh.tc, &fs, sh.pend, sh.Mpi);
      if (tid < 24) plan->pend[tid] = sh.pend[tid];
      if (tid == 0) {
        plan->g = (float)fs.g;
        plan->gsc = (float)(fs.g / ((double)N0 * (double)N1));
      }
    }
  }
  __syncthreads();
  if (tid == 0) plan->wmax = do_meas ? __int_as_float(sh.wmax_bits) : -1.0f;
  if (sh.degenerate) {
    if (tid == 0) plan->ok = 0;
  } else if (!do_time) {
    // measurement only: normalise the new weights in place
    const float ps = sh.ps;
    for (int t = tid; t < np4; t += kT) {
      const int r = t / q1, c = (t % q1) * 4;
      float4 x = *(const float4*)(out + (size_t)r * N1 + c);
      x.x *= ps;
      x.y *= ps;
      x.z *= ps;
      x.w *= ps;
      *(float4*)(out + (size_t)r * N1 + c) = x;
    }
    if (tid == 0) plan->ok = 0;
  } else {
    // sub-step coefficients and, for a separable regrid, the regrid rows
    const int l = fs.l;
    for (int q = tid; q < l; q += kT) {
      double pa[4], pb[6];
      frame_substep<2>(sh.tc, sh.Mpi, q, pa, pb);
      plan->pa[q][0] = (float)pa[0];
      plan->pa[q][1] = (float)pa[1];
      plan->pb[q] = (float)pb[0];
    }
    if (!fs.realign) {
      const int a = tid < kT / 2 ? 1 : 0;
      regrid_rows(plan->rows[a], fs.rs[a], fs.rd[a], a ? N1 : N0, tid - (a ? 0 : kT / 2), kT / 2);
    }
    if (tid == 0) plan->ok = 1;
  }
  __syncthreads();
  for (int i = tid; i < kFsWords; i += kT) ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
}

// CTAs per SM of the planned kernel of class C: shared memory (dynamic, static
// and the 1 KiB the hardware keeps per CTA, of 228 KiB per SM) and TMEM (128
// of 512 columns per CTA).  The launch bound holds the registers to it.
template <int P, int C>
constexpr int planned_ctas() {
  constexpr int per = Smem<P, C>::bytes + (int)sizeof(SharedT<Smem<P, C>::threads, C, false>) + 1024;
  constexpr int by_smem = 228 * 1024 / per;
  return by_smem < 4 ? by_smem : 4;
}

// Planned transform kernel of a batched epoch (size class C): the time update
// of the filters whose front kernel ran it, from the weights and plan it left.
template <int P, int C>
__global__ void __launch_bounds__(Smem<P, C>::threads, planned_ctas<P, C>())
    k_fused2d_planned(const FilterSlot* __restrict__ slots, const StepItem* __restrict__ items,
                      const TimeConsts* __restrict__ tcs) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const StepItem& it = items[blockIdx.x];
  const FilterSlot& sl = slots[it.slot];
  const FusedView v{sl.st, sl.buf0, sl.buf1, {sl.hart[0], sl.hart[1]}, {sl.sctab[0], sl.sctab[1]},
                    sl.N0, sl.N1, 0, (it.flags >> 1) & 1, sl.mp, it.z,
                    tcs ? tcs + blockIdx.x : sl.tc, (const BatchPlan*)sl.plan, sl.fft};
  fused2d<P, false, true, C>(v, smem);
}

// Moments and status words of the listed filters (read before any is cleared:
// a filter may be listed twice).
__global__ void k_batch_gather(const DevState* __restrict__ st, const int* __restrict__ ids, int k,
                               double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const FrameState& f = st[ids[i]].f;
    double* o = out + (size_t)i * 8;
    o[0] = f.mean[0];
    o[1] = f.mean[1];
    for (int j = 0; j < 4; ++j) o[2 + j] = f.cov[j];
    o[6] = (double)f.status;
    o[7] = 0.0;
  }
}

__global__ void k_batch_clear(DevState* __restrict__ st, const int* __restrict__ ids, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) st[ids[i]].f.status = 0;
}

// Prior weights exp(-1/2 (x - m0)^T P0^{-1} (x - m0)) on the initial frame (float32 storage).
__global__ void k_prior_f32(Dims d, const DevState* st, const double* aux, float* X) {
  const int n = d.nx;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d.P;
       p += (long long)gridDim.x * blockDim.x) {
    int j[MAXN];
    long long t = p;
    for (int m = n - 1; m >= 0; --m) { j[m] = (int)(t % d.N[m]); t /= d.N[m]; }
    double dx[MAXN];
    for (int a = 0; a < n; ++a) {
      double x = st->f.c[a];
      for (int b = 0; b < n; ++b) x += st->f.M[a * n + b] * (j[b] - 0.5 * (d.N[b] - 1));
      dx[a] = x - aux[kAuxM0 + a];
    }
    double q = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) q += dx[a] * aux[a * n + b] * dx[b];
    X[p] = (float)exp(-0.5 * q);
  }
}

// Host: f(std::integral_constant<int, P>) for the tensor-core format P of a precision.
template <class F>
void with_format(int precision, F&& f) {
  switch (precision) {
    case PMF_PREC_FP16X3: f(std::integral_constant<int, PMF_PREC_FP16X3>{}); break;
    case PMF_PREC_BF16X3: f(std::integral_constant<int, PMF_PREC_BF16X3>{}); break;
    case PMF_PREC_BF16X6: f(std::integral_constant<int, PMF_PREC_BF16X6>{}); break;
    default: f(std::integral_constant<int, PMF_PREC_TF32>{}); break;
  }
}

void launch_fused(int precision, const FusedJob& job, cudaStream_t s) {
  with_format(precision, [&](auto fmt) {
    constexpr int P = decltype(fmt)::value;
    k_fused2d<P><<<1, kThreads, Smem<P, 128, false>::bytes, s>>>(job);
  });
}

template <int P>
void set_smem_limits() {
  cudaFuncSetAttribute(k_fused2d<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<P, 128, false>::bytes);
  cudaFuncSetAttribute(k_fused2d_planned<P, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<P, 128>::bytes);
  cudaFuncSetAttribute(k_fused2d_planned<P, 96>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<P, 96>::bytes);
  cudaFuncSetAttribute(k_fused2d_planned<P, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<P, 64>::bytes);
}

// Host: split 16-bit (or float32) planes of a matrix in the operand layout.
void split_planes(const std::vector<double>& Mt, int rows, int cols, int prec, double scale,
                  std::vector<uint8_t>& out, int cls) {
  const int esz = prec == PMF_PREC_TF32 ? 4 : 2;
  const int epc = 16 / esz, rowblk = (cls / epc) * 128;
  const size_t plane = (size_t)rows / 8 * rowblk;
  const int np = prec == PMF_PREC_TF32 ? 1 : prec == PMF_PREC_BF16X6 ? 3 : 2;
  out.assign(plane * np, 0);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) {
      const size_t off = (size_t)(r / 8) * rowblk + (c / epc) * 128 + (r % 8) * 16 + (c % epc) * esz;
      const double x = Mt[(size_t)r * cols + c] * scale;
      if (prec == PMF_PREC_TF32) {
        float f = (float)x;
        std::memcpy(&out[off], &f, 4);
      } else if (prec == PMF_PREC_BF16X3 || prec == PMF_PREC_BF16X6) {
        // pieces of the float64 value: hi, then the remainders
        __nv_bfloat16 pc[3];
        double r = x;
        for (int i = 0; i < np; ++i) {
          pc[i] = __float2bfloat16_rn((float)r);
          r -= (double)__bfloat162float(pc[i]);
          std::memcpy(&out[i * plane + off], &pc[i], 2);
        }
      } else {
        __half hi = __float2half_rn((float)x);
        __half lo = __float2half_rn((float)(x - (double)__half2float(hi)));
        std::memcpy(&out[off], &hi, 2);
        std::memcpy(&out[plane + off], &lo, 2);
      }
    }
}

}  // namespace

int tc_supported(const pmf_config* cfg, std::string* why) {
  if (cfg->nx != 2 && cfg->nx != 3) {
    *why = "the tensor-core path handles n_x = 2 (fused) and n_x = 3 (per-axis pipelines)";
    return PMF_ERR_UNSUPPORTED;
  }
  for (int a = 0; a < cfg->nx; ++a)
    if (cfg->N[a] % 16 || cfg->N[a] < 16 || cfg->N[a] > 128) {
      *why = "the fused tensor-core kernel needs N multiple of 16 in [16, 128]";
      return PMF_ERR_UNSUPPORTED;
    }
  if (cfg->precision != PMF_PREC_FP16X3 && cfg->precision != PMF_PREC_BF16X3 &&
      cfg->precision != PMF_PREC_TF32 && !(cfg->precision == PMF_PREC_BF16X6 && cfg->nx == 2)) {
    *why = "the tensor-core kernels support FP16X3, BF16X3 and TF32 (and BF16X6 for n_x = 2)";
    return PMF_ERR_UNSUPPORTED;
  }
  return PMF_OK;
}

int tc_build_axis_table(int N, int precision, void** dev, size_t* hart_bytes, int cls) {
  if ((cls != 128 && cls != 96 && cls != 64) || N > cls) return PMF_ERR_ARG;
  const double scale = precision == PMF_PREC_FP16X3 ? 16384.0 : 1.0;
  std::vector<double> H((size_t)N * N);
  const double w = 6.283185307179586476925286766559 / N;
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j) {
      const long long r = ((long long)k * j) % N;
      H[(size_t)k * N + j] = std::cos(w * r) + std::sin(w * r);
    }
  std::vector<uint8_t> planes;
  split_planes(H, N, N, precision, scale, planes, cls);
  std::vector<float> tab(2 * (2 * N + 1));
  for (int m = -N; m <= N; ++m) {
    const double ang = 3.14159265358979323846 * m / N;
    tab[2 * (m + N)] = (float)std::cos(ang);
    tab[2 * (m + N) + 1] = (float)std::sin(ang);
  }
  const size_t hb = planes.size(), tb = tab.size() * sizeof(float);
  *dev = nullptr;
  if (cudaMalloc(dev, hb + tb) != cudaSuccess) return PMF_ERR_OOM;
  *hart_bytes = hb;
  if (cudaMemcpy(*dev, planes.data(), hb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((uint8_t*)*dev + hb, tab.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess)
    return PMF_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    for (int p : {PMF_PREC_FP16X3, PMF_PREC_BF16X3, PMF_PREC_BF16X6, PMF_PREC_TF32})
      with_format(p, [](auto fmt) { set_smem_limits<decltype(fmt)::value>(); });
    attr = true;
  }
  return PMF_OK;
}

size_t tc_axis_table_bytes(int N, int precision, int cls) {
  const size_t plane = (size_t)N / 8 * (precision == PMF_PREC_TF32 ? 32 : 16) * cls;
  const int np = precision == PMF_PREC_TF32 ? 1 : precision == PMF_PREC_BF16X6 ? 3 : 2;
  return plane * np + 2 * (2 * N + 1) * sizeof(float);
}

int tc_build_tables(const pmf_config* cfg, TcTables* t, std::string* why) {
  std::memset(t, 0, sizeof(*t));
  t->prec = cfg->precision;
  for (int a = 0; a < cfg->nx; ++a) {
    const int rc = tc_build_axis_table(cfg->N[a], cfg->precision, &t->hart[a], &t->hart_bytes[a]);
    if (rc) {
      *why = "transform tables";
      return rc;
    }
  }
  return PMF_OK;
}

void tc_free_tables(TcTables* t) {
  for (int a = 0; a < MAXN; ++a) {
    cudaFree(t->hart[a]);
    t->hart[a] = nullptr;
  }
}

// One warp waits (bounded) on a shared-memory mbarrier expecting one arrival;
// with arrive the arrival precedes the wait.  out: PMF_OK or PMF_ERR_TIMEOUT.
__global__ void k_wait_probe(long long polls, int arrive, int* out) {
  __shared__ uint64_t bar;
  const uint32_t mb = su32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncwarp();
  if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
  __syncwarp();
  const bool ok = mbar_wait(mb, 0, polls);
  if (threadIdx.x == 0) *out = ok ? PMF_OK : PMF_ERR_TIMEOUT;
}

int tc_wait_probe(long long polls, int arrive, cudaStream_t s) {
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return PMF_ERR_CUDA;
  int h = -1;
  k_wait_probe<<<1, 32, 0, s>>>(polls, arrive, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  return e == cudaSuccess ? h : PMF_ERR_CUDA;
}

int tc_prior(const Dims& d, DevState* st, const double* prior_aux, float* X, double* partials,
             cudaStream_t s) {
  long long blocks = (d.P + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_prior_f32<<<(int)blocks, 256, 0, s>>>(d, st, prior_aux, X);
  launch_moments_f32(d, st, X, partials, s);
  return 3;
}

int tc_step(const Dims& d, const pmf_config& cfg, const TcTables* t, const MeasParams* mp,
            const TimeConsts* tcs, DevState* st, float* b0, float* b1, cudaStream_t s) {
  FusedJob job{};
  job.st = st;
  job.buf0 = b0;
  job.buf1 = b1;
  job.N0 = cfg.N[0];
  job.N1 = cfg.N[1];
  for (int a = 0; a < 2; ++a) {
    job.hart[a] = (const uint8_t*)t->hart[a];
    job.sctab[a] = (const float*)((const uint8_t*)t->hart[a] + t->hart_bytes[a]);
  }
  job.do_meas = mp != nullptr;
  job.do_time = tcs != nullptr;
  job.fft = t->fft;
  if (mp) job.mp = *mp;
  if (tcs) job.tc = *tcs;
  if (!job.do_meas && !job.do_time) return 0;
  launch_fused(cfg.precision, job, s);
  return 1;
}

size_t tc_plan_bytes() { return sizeof(BatchPlan); }

namespace {
template <int P>
void launch_planned(const FilterSlot* slots, const StepItem* items, int k, int k128, int k96, cudaStream_t s,
                    const TimeConsts* tcs, cudaStream_t s2) {
  if (k128 > 0)
    k_fused2d_planned<P, 128><<<k128, Smem<P, 128>::threads, Smem<P, 128>::bytes, s>>>(slots, items, tcs);
  if (k96 > 0)
    k_fused2d_planned<P, 96><<<k96, Smem<P, 96>::threads, Smem<P, 96>::bytes, s2>>>(
        slots, items + k128, tcs ? tcs + k128 : nullptr);
  const int k64 = k - k128 - k96;
  if (k64 > 0)
    k_fused2d_planned<P, 64><<<k64, Smem<P, 64>::threads, Smem<P, 64>::bytes, s2>>>(
        slots, items + k128 + k96, tcs ? tcs + k128 + k96 : nullptr);
}
}  // namespace

int tc_batch_epoch(int precision, const FilterSlot* slots, const StepItem* items, int k, int k128, int k96,
                   cudaStream_t s, const TimeConsts* tcs, cudaStream_t s2, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  if (k <= 0) return 0;
  k_front2d<<<k, kFrontThreads, 0, s>>>(slots, items, tcs);
  const bool fork = s2 && ev_fork && ev_join && k128 > 0 && k > k128;
  if (fork) {
    cudaEventRecord(ev_fork, s);
    cudaStreamWaitEvent(s2, ev_fork, 0);
  }
  cudaStream_t t = fork ? s2 : s;
  with_format(precision, [&](auto fmt) { launch_planned<decltype(fmt)::value>(slots, items, k, k128, k96, s, tcs, t); });
  if (fork) {
    cudaEventRecord(ev_join, s2);
    cudaStreamWaitEvent(s, ev_join, 0);
  }
  return 1 + (k128 > 0) + (k96 > 0) + (k - k128 - k96 > 0);
}

// ---- form of the 2-D Hartley transforms: tensor-core GEMM or shared-memory FFT
bool tc2_fft_ok(int N0, int N1, int precision) {
  if (precision == PMF_PREC_BF16X6) return false;
  auto ok = [](int N) {
    while (N % 3 == 0) N /= 3;
    return N >= 2 && (N & (N - 1)) == 0;
  };
  return ok(N0) && ok(N1);
}

namespace {

std::mutex g_tune2_mu;
// (N0, N1, precision) -> (form, GEMM us, FFT us)
std::map<std::tuple<int, int, int>, std::tuple<int, double, double>> g_tune2;
bool g_tune2_loaded = false;

std::string tune2_path() {
  Dl_info info;
  if (!dladdr((void*)&tc2_fft_ok, &info) || !info.dli_fname) return "";
  std::string p = info.dli_fname;
  const size_t slash = p.rfind('/');
  return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/autotune_2d.json";
}

// {"2d:N0x N1:p": {"form": f, "gemm_us": g, "fft_us": t}, ...}
void tune2_load() {
  g_tune2_loaded = true;
  const std::string p = tune2_path();
  FILE* f = p.empty() ? nullptr : std::fopen(p.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int a = 0, b = 0, prec = 0, form = -1;
    double tg = 0.0, tf = 0.0;
    const char* q = std::strstr(line, "\"2d:");
    if (q && std::sscanf(q, "\"2d:%dx%d:%d\": {\"form\": %d, \"gemm_us\": %lf, \"fft_us\": %lf", &a, &b, &prec, &form,
                         &tg, &tf) == 6 &&
        (form == 0 || form == 1))
      g_tune2[std::make_tuple(a, b, prec)] = std::make_tuple(form, tg, tf);
  }
  std::fclose(f);
}

void tune2_save() {
  const std::string p = tune2_path();
  FILE* f = p.empty() ? nullptr : std::fopen(p.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : g_tune2)
    std::fprintf(f, "  \"2d:%dx%d:%d\": {\"form\": %d, \"gemm_us\": %.3f, \"fft_us\": %.3f}%s\n",
                 std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<0>(kv.second),
                 std::get<1>(kv.second), std::get<2>(kv.second), ++i < g_tune2.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
}

// Mean time of one epoch (measurement + time update) of a scratch N0 x N1
// filter in the fused kernel, in the given form.
double time_form2(int N0, int N1, int prec, int fft, cudaStream_t s) {
  pmf_config c{};
  c.nx = 2;
  c.N[0] = N0;
  c.N[1] = N1;
  const double A[4] = {0.0, 1.0, -1.0, -0.2};
  for (int i = 0; i < 4; ++i) c.A[i] = A[i];
  c.Q[0] = 0.1;
  c.Q[3] = 0.3;
  c.P0[0] = c.P0[3] = 0.25;
  c.span_sigma = 6.0;
  c.dt_sub = 0.01;
  c.realign_rho = 0.5;
  c.precision = prec;
  pmf_meas m{};
  m.kind = PMF_MEAS_LINEAR;
  m.nz = 2;
  m.z[0] = 0.05;
  m.z[1] = -0.05;
  m.R[0] = m.R[3] = 0.01;
  m.H[0] = m.H[3] = 1.0;
  std::string why;
  FusedJob job{};
  if (meas_params(2, &m, &job.mp, &why) || time_consts(c, 0.05, &job.tc, &why)) return -1.0;
  TcTables t{};
  if (tc_build_tables(&c, &t, &why) != PMF_OK) {
    tc_free_tables(&t);
    return -1.0;
  }
  const DevState h = initial_state(c);
  const size_t P = (size_t)N0 * N1;
  std::vector<float> w(2 * P, 0.0f);
  for (int i = 0; i < N0; ++i)
    for (int j = 0; j < N1; ++j) {
      const double u = (i - 0.5 * (N0 - 1)) / (N0 / 12.0), v = (j - 0.5 * (N1 - 1)) / (N1 / 12.0);
      w[(size_t)i * N1 + j] = (float)std::exp(-0.5 * (u * u + v * v));
    }
  DevState* st = nullptr;
  float* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double us = -1.0;
  if (cudaMalloc(&st, sizeof(DevState)) == cudaSuccess && cudaMalloc(&buf, sizeof(float) * 2 * P) == cudaSuccess &&
      cudaMemcpy(buf, w.data(), sizeof(float) * 2 * P, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    job.st = st;
    job.buf0 = buf;
    job.buf1 = buf + P;
    job.N0 = N0;
    job.N1 = N1;
    for (int a = 0; a < 2; ++a) {
      job.hart[a] = (const uint8_t*)t.hart[a];
      job.sctab[a] = (const float*)((const uint8_t*)t.hart[a] + t.hart_bytes[a]);
    }
    job.do_meas = 1;
    job.do_time = 1;
    job.fft = fft;
    auto launch = [&]() { launch_fused(prec, job, s); };
    constexpr int kReps = 20;
    float ms = 0.0f;
    // every epoch starts from the same state and weights
    for (int i = 0; i < 3 + kReps; ++i) {
      if (i == 3) cudaEventRecord(e0, s);
      cudaMemcpyAsync(st, &h, sizeof(DevState), cudaMemcpyHostToDevice, s);
      launch();
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        cudaGetLastError() == cudaSuccess)
      us = 1e3 * ms / kReps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(st);
  cudaFree(buf);
  tc_free_tables(&t);
  return us;
}

}  // namespace

int tc2_form(const pmf_config* cfg, cudaStream_t s) {
  if (cfg->nx != 2 || !tc2_fft_ok(cfg->N[0], cfg->N[1], cfg->precision) || cfg->transform == PMF_TRANSFORM_GEMM)
    return 0;
  if (cfg->transform == PMF_TRANSFORM_FFT) return 1;
  if (const char* form = std::getenv("PMF_2D_FORM")) {   // explicit choice, no tuning
    if (!std::strcmp(form, "fft")) return 1;
    if (!std::strcmp(form, "gemm")) return 0;
  }
  const auto key = std::make_tuple(cfg->N[0], cfg->N[1], cfg->precision);
  std::lock_guard<std::mutex> g(g_tune2_mu);
  if (!g_tune2_loaded) tune2_load();
  auto it = g_tune2.find(key);
  if (it != g_tune2.end()) return std::get<0>(it->second);
  const double tg = time_form2(cfg->N[0], cfg->N[1], cfg->precision, 0, s);
  const double tf = time_form2(cfg->N[0], cfg->N[1], cfg->precision, 1, s);
  const int form = (tf > 0.0 && tg > 0.0 && tf < tg) ? 1 : 0;
  g_tune2[key] = std::make_tuple(form, tg, tf);
  tune2_save();
  return form;
}

int tc_batch_gather(DevState* st, const int* ids, int k, double* out, cudaStream_t s) {
  if (k <= 0) return 0;
  const int blocks = (k + 255) / 256;
  k_batch_gather<<<blocks, 256, 0, s>>>(st, ids, k, out);
  k_batch_clear<<<blocks, 256, 0, s>>>(st, ids, k);
  return 2;
}

}  // namespace pmf
