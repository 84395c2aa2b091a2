// Tensor-core path for 3-D grids (N0, N1, N2 multiples of 16, at most 128):
// the grid lives in HBM/L2 and each time update runs three on-chip pipelines.
//
//   meas   M1 exponent minimum, M2 likelihood multiply + moment partials,
//          F  moments, normaliser, frame (float64), sub-step coefficients,
//             regrid rows of the three axes
//   time   [realign gather + copy-back when the frame is re-aligned; when it
//             is kept, the folded forward matrices W_a = H_a I_a instead]
//          A  per slice j0: regrid + Hartley along axes 2 and 1, one GEMM per
//             axis with W_a (H_a after a re-alignment) -> T
//          B  per tile of 128 lines along axis 0, closed under sign flips
//             ({k1, -k1} x (C u -C)): regrid + Hartley along axis 0, the 3-D
//             diffusion multiplier with the separable-to-3-D parity fix-up on
//             8-point orbits (Sec. V-B steps 2-4), inverse along axis 0 -> T
//          C  per slice: inverse along axes 2 and 1, moment partials -> weights
//          F2 moments, normaliser, frame commit
//
// GEMM stages, operand layouts and split formats are those of the 2-D fused
// kernel (pmf_tcops.cuh).  Every CTA scales its own operands.
#include <cmath>
#include <cstring>
#include <vector>

#include "pmf_device.cuh"
#include "pmf_kernels.cuh"
#include "pmf_tc.cuh"
#include "pmf_tcops.cuh"

namespace pmf {

namespace {

constexpr int kT = 512;
constexpr int kOffA = 0, kOffW = 65536, kOffS = 131072;
constexpr int kSStr = 132;
constexpr int kSmem = kOffS + 128 * kSStr * 4;
constexpr uint32_t kTmemCols = 128;

struct Geo3 {
  int N[3];
  long long P;
};

// Per-update scalars written by the frame kernel for the time-update kernels.
struct Update3 {
  float pa[MAXL][3];
  float pb[MAXL][3];
  int l, exact, realign, skip;   // skip: the measurement update was degenerate
  float gsc;                 // trace factor / (N0 N1 N2)
  RegridRows rows[3];        // regrid rows per axis
  double shear[25];          // band-limited re-alignment passes (shear3_setup layout)
  unsigned int wmax[3];      // float bits of max |W_a| of the folded forward matrices
};

struct Job3 {
  DevState* st;
  float* buf0;
  float* buf1;
  const uint8_t* hart[3];
  const float* sctab[3];
  Geo3 g;
  DF* partials;              // per-CTA moment partials (double-float, 16 slots each)
  unsigned int* emin_bits;   // float bits of the exponent minimum
  Update3* up;               // device
  double* pend;              // pending frame (device)
  float* fold;               // folded forward matrices W_a = H_a I_a: [3][128][128], rows k, columns j
  int precision;
  int flags;                 // this epoch: bit 0 measurement update, bit 1 time update
  int chunks;                // axis-0 line tiles: chunks of 32 k2 per k1
  int mblocks;               // CTAs of the measurement kernels
  MeasParams mp;             // measurement of this epoch (z filled)
  TimeConsts tc;             // constants of this epoch's time update
};

// One batched launch sequence: jobs and, per kernel kind, the first CTA of
// each job (n + 1 entries per kind; a job may own no CTA of a kind).
enum { kKindMeas = 0, kKindPoints = 1, kKindSlices = 2, kKindLines = 3, kKindShear = 4, kKinds = 5 };
struct Batch3 {
  const Job3* jobs;
  const int* first;          // [kind * (n + 1) + j]
  int n;
  Job3 one;                  // n == 1: the job itself, in the kernel parameters
};

__device__ __forceinline__ const Job3& job_at(const Batch3& b, int j) { return b.n == 1 ? b.one : b.jobs[j]; }

// Job owning CTA blk of a kind (largest j with first[j] <= blk), the CTA's
// index within the job and the job's CTA count.
__device__ __forceinline__ int find_job(const Batch3& b, int kind, int blk, int* local, int* count) {
  if (b.n == 1) {
    *local = blk;
    *count = gridDim.x;
    return 0;
  }
  const int* f = b.first + kind * (b.n + 1);
  int lo = 0, hi = b.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (f[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  *local = blk - f[lo];
  *count = f[lo + 1] - f[lo];
  return lo;
}

struct Smem3 {
  uint64_t mbar_mma, mbar_tma;
  uint32_t tmem;
  int abort;
  float redf[2][16];
  DF redd[16][6];
  float redw[16][10];   // per-warp float32 moment sums of the measurement kernel
};

__device__ __forceinline__ float block_max3(Smem3& sh, float v, int slot) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh.redf[slot][threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.0f;
#pragma unroll
  for (int w = 0; w < kT / 32; ++w) m = fmaxf(m, sh.redf[slot][w]);
  return m;
}

// Block sum of six double-float moment sums; thread 0 writes them (double-float)
// to out.
__device__ void block_partials3(Smem3& sh, const DF* s, DF* out) {
  DF a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = s[i];
    for (int o = 16; o; o >>= 1) {
      DF b{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
      a[i] = df_add(a[i], b);
    }
  }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < 6; ++i) sh.redd[threadIdx.x >> 5][i] = a[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    DF v[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      v[i] = threadIdx.x < kT / 32 ? sh.redd[threadIdx.x][i] : DF{0.0f, 0.0f};
      for (int o = 16; o; o >>= 1) {
        DF b{__shfl_xor_sync(0xffffffffu, v[i].hi, o), __shfl_xor_sync(0xffffffffu, v[i].lo, o)};
        v[i] = df_add(v[i], b);
      }
    }
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < 6; ++i) out[i] = v[i];
  }
}

// --- tensor-core plumbing shared by the three pipelines -----------------------
struct Pipe {
  uint32_t tmem, tlane, mb_mma, mb_tma, ph_mma, ph_tma;
};

__device__ void pipe_init(Smem3& sh, Pipe& p) {
  const int warp = threadIdx.x >> 5;
  p.mb_mma = su32(&sh.mbar_mma);
  p.mb_tma = su32(&sh.mbar_tma);
  p.ph_mma = p.ph_tma = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(p.mb_mma));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(p.mb_tma));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  p.tmem = sh.tmem;
  p.tlane = p.tmem + ((uint32_t)((warp & 3) * 32) << 16);
}

__device__ void pipe_done(Smem3& sh, const Pipe& p) {
  tc_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(p.tmem), "r"(kTmemCols));
}

// After the operand and matrix of a GEMM are in shared memory (generic stores
// fenced by the caller's __syncthreads): optionally TMA-load the Hartley planes
// of size N into W, then issue the GEMM (thread 0).  Returns false on timeout.
template <int P>
__device__ bool pipe_issue(Smem3& sh, Pipe& p, uint8_t* A, uint8_t* W, const uint8_t* hart, int Nh, int a_mn,
                           int nout, int K) {
  if (threadIdx.x == 0) {
    tc_after_sync();
    bool ok = true;
    if (hart) {
      const uint32_t pbytes = (uint32_t)Nh * (uint32_t)(Fmt<P>::rowblk / 8);
      expect_tx(p.mb_tma, pbytes * Fmt<P>::planes);
      for (int pl = 0; pl < Fmt<P>::planes; ++pl)
        bulk_load(su32(W) + pl * kPlane, hart + (size_t)pl * pbytes, pbytes, p.mb_tma);
      ok = mbar_wait(p.mb_tma, p.ph_tma);
    }
    if (ok) issue_stage<P>(p.tmem, su32(A), a_mn, su32(W), nout, K, p.mb_mma);
    else sh.abort = 1;
  }
  if (hart) p.ph_tma ^= 1;
  return true;
}

// Wait for the GEMM; false (block-uniform) on timeout.
__device__ bool pipe_wait(Smem3& sh, Pipe& p) {
  const bool ok = mbar_wait(p.mb_mma, p.ph_mma);
  p.ph_mma ^= 1;
  const bool bad = __syncthreads_or(!ok || sh.abort);
  tc_after_sync();
  return !bad;
}

// Accumulator (lanes < nlane valid, nout columns) -> next operand with a fresh
// scale; `tr` writes it transposed (TF32 operands read K-major only).
// Returns the operand scale.
template <int P>
__device__ float acc_to_operand(Smem3& sh, const Pipe& p, uint8_t* A, int nlane, int nout, float inv_scale,
                                bool tr, int slot) {
  const int row = threadIdx.x & 127, cg = threadIdx.x >> 7;
  const int ncol = nout / 4, c0 = cg * ncol;
  float m = 0.0f;
  for (int c = 0; c < ncol; c += 4) m = amax4(m, tmem_ld4(p.tlane + c0 + c));
  const float sa = op_scale<P>(block_max3(sh, row < nlane ? m * inv_scale : 0.0f, slot));
  for (int c = 0; c < ncol; c += 4) {
    float4 v = tmem_ld4(p.tlane + c0 + c);
    v.x *= inv_scale;
    v.y *= inv_scale;
    v.z *= inv_scale;
    v.w *= inv_scale;
    if (tr)
      store4_t(A, row, c0 + c, v, sa);
    else
      store4<P>(A, row, c0 + c, v, sa);
  }
  tc_before_sync();
  return sa;
}

// Accumulator -> staging tile (true scale).
__device__ void acc_to_stage(const Pipe& p, float* S, int nout, float inv_scale) {
  const int row = threadIdx.x & 127, cg = threadIdx.x >> 7;
  const int ncol = nout / 4, c0 = cg * ncol;
  for (int c = 0; c < ncol; c += 4) {
    float4 v = tmem_ld4(p.tlane + c0 + c);
    v.x *= inv_scale;
    v.y *= inv_scale;
    v.z *= inv_scale;
    v.w *= inv_scale;
    *(float4*)(S + row * kSStr + c0 + c) = v;
  }
  tc_before_sync();
}

template <int P>
__device__ void stage_to_op(uint8_t* A, const float* S, int nr, int nc, float s) {
  const int q4 = nc / 4;
  for (int t = threadIdx.x; t < nr * q4; t += kT) {
    const int r = t % nr, c = (t / nr) * 4;
    store4<P>(A, r, c, *(const float4*)(S + r * kSStr + c), s);
  }
}

__device__ float stage_absmax(const float* S, int nr, int nc) {
  const int q4 = nc / 4;
  float m = 0.0f;
  for (int t = threadIdx.x; t < nr * q4; t += kT) {
    const int r = t % nr, c = (t / nr) * 4;
    m = amax4(m, *(const float4*)(S + r * kSStr + c));
  }
  return m;
}

// =========================== measurement update ==============================
struct Meas3 {
  int kind, nz;
  float Rinv[9];
  float M[9];
  float r0[3];      // linear: z - H c; bearing: wrap(z1 - atan2(c2, c1)), z2 - c3
  float H[9];
  float c0, c1, cc; // bearing: centre components, |c_{1:2}|^2
};

__device__ __forceinline__ float wrapf(float r) {
  // at an exact +-pi boundary either branch gives the same squared residual
  const float two_pi = 6.28318530717958647692f, pi = 3.14159265358979323846f;
  const float inv_two_pi = 0.15915494309189533577f;
  return r - two_pi * ceilf((r - pi) * inv_two_pi);
}

// 1/2 r^T R^{-1} r, residual relative to the frame centre (d = M u):
// linear r = r0 - H d; bearing: atan2(c + d) - atan2(c) = atan2(c x d, |c|^2 + c.d).
__device__ __forceinline__ float meas_e3(const Meas3& m, float u0, float u1, float u2) {
  const float d0 = m.M[0] * u0 + m.M[1] * u1 + m.M[2] * u2;
  const float d1 = m.M[3] * u0 + m.M[4] * u1 + m.M[5] * u2;
  const float d2 = m.M[6] * u0 + m.M[7] * u1 + m.M[8] * u2;
  float r[3];
  if (m.kind == PMF_MEAS_LINEAR) {
    for (int i = 0; i < m.nz; ++i) r[i] = m.r0[i] - (m.H[i * 3] * d0 + m.H[i * 3 + 1] * d1 + m.H[i * 3 + 2] * d2);
  } else {
    const float dth = atan2f(m.c0 * d1 - m.c1 * d0, m.cc + m.c0 * d0 + m.c1 * d1);
    r[0] = wrapf(m.r0[0] - dth);
    r[1] = m.r0[1] - d2;
  }
  float e = 0.0f;
  for (int i = 0; i < m.nz; ++i)
    for (int k = 0; k < m.nz; ++k) e += r[i] * m.Rinv[i * m.nz + k] * r[k];
  return 0.5f * e;
}

// Frame-relative measurement constants of a 3-D filter, formed by the 32
// lanes of one warp (lane e < 9 one
// entry of M, R^-1 and H, lanes < nz one residual at the centre): one
// float64 step per lane instead of a serial chain in one thread while the
// rest of the CTA waits.
__device__ void meas_consts_warp(const MeasParams& mp, const FrameState& fs, Meas3& m) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    m.kind = mp.kind;
    m.nz = mp.nz;
  }
  if (lane < 9) {
    m.M[lane] = (float)fs.M[lane];
    if (lane < mp.nz * mp.nz) m.Rinv[lane] = (float)mp.Rinv[lane];
  }
  if (mp.kind == PMF_MEAS_LINEAR) {
    if (lane < 9 && lane < mp.nz * 3) m.H[lane] = (float)mp.H[lane];
    if (lane < mp.nz) {
      const double h = fma(mp.H[lane * 3], fs.c[0], fma(mp.H[lane * 3 + 1], fs.c[1], mp.H[lane * 3 + 2] * fs.c[2]));
      m.r0[lane] = (float)(mp.z[lane] - h);
    }
  } else if (lane == 0) {
    // angle and squared norm of the centre were formed when the frame was committed
    double r = mp.z[0] - fs.hc[0];
    const double two_pi = 6.283185307179586476925286766559, pi = 3.14159265358979323846;
    r -= two_pi * ceil((r - pi) * (1.0 / two_pi));
    m.r0[0] = (float)r;
  } else if (lane == 1) {
    m.r0[1] = (float)(mp.z[1] - fs.c[2]);
  } else if (lane == 2) {
    m.c0 = (float)fs.c[0];
  } else if (lane == 3) {
    m.c1 = (float)fs.c[1];
  } else if (lane == 4) {
    m.cc = (float)fs.hc[1];
  }
}

// Point index -> (j0, j1, j2); 32-bit arithmetic (P <= 128^3 < 2^31).
__device__ __forceinline__ void unflat3(const Geo3& g, long long p, int* j) {
  const int i = (int)p, t = i / g.N[2];
  j[2] = i - t * g.N[2];
  j[1] = t % g.N[1];
  j[0] = t / g.N[1];
}

__global__ void __launch_bounds__(kT) k_meas_min3(const __grid_constant__ Batch3 b) {
  __shared__ Meas3 m;
  __shared__ float red[kT / 32];
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindMeas, blockIdx.x, &blk, &cnt));
  const MeasParams& mp = job.mp;
  if (threadIdx.x < 32) meas_consts_warp(mp, job.st->f, m);
  __syncthreads();
  const Geo3& g = job.g;
  float e = INFINITY;
  for (long long q = blk * (long long)kT + threadIdx.x; q < g.P / 4; q += (long long)cnt * kT) {
    int j[3];
    unflat3(g, q * 4, j);
    const float u0 = j[0] - 0.5f * (g.N[0] - 1), u1 = j[1] - 0.5f * (g.N[1] - 1), u2 = j[2] - 0.5f * (g.N[2] - 1);
    for (int k = 0; k < 4; ++k) e = fminf(e, meas_e3(m, u0, u1, u2 + k));
  }
  for (int o = 16; o; o >>= 1) e = fminf(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = INFINITY;
    for (int w = 0; w < kT / 32; ++w) v = fminf(v, red[w]);
    if (v < INFINITY) atomicMin(job.emin_bits, __float_as_uint(fmaxf(v, 0.0f)));
  }
}

// Likelihood multiply (into the other buffer) and moment partials per CTA.
__global__ void __launch_bounds__(kT) k_meas_apply3(const __grid_constant__ Batch3 b) {
  __shared__ Meas3 m;
  __shared__ Smem3 sh;
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindMeas, blockIdx.x, &blk, &cnt));
  const MeasParams& mp = job.mp;
  if (threadIdx.x < 32) meas_consts_warp(mp, job.st->f, m);
  __syncthreads();
  const Geo3& g = job.g;
  const int cur = job.st->f.cur;
  const float* in = cur ? job.buf1 : job.buf0;
  float* out = cur ? job.buf0 : job.buf1;
  const float ps = (float)job.st->f.pscale;
  const float emin = __uint_as_float(*job.emin_bits);
  // the ten moment sums of this thread's points in float32 (a few quads)
  float f[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) f[i] = 0.0f;
  for (long long q = blk * (long long)kT + threadIdx.x; q < g.P / 4; q += (long long)cnt * kT) {
    int j[3];
    unflat3(g, q * 4, j);
    const float u0 = j[0] - 0.5f * (g.N[0] - 1), u1 = j[1] - 0.5f * (g.N[1] - 1), u2 = j[2] - 0.5f * (g.N[2] - 1);
    float4 x = *(const float4*)(in + q * 4);
    x.x *= ps * __expf(emin - meas_e3(m, u0, u1, u2));
    x.y *= ps * __expf(emin - meas_e3(m, u0, u1, u2 + 1.0f));
    x.z *= ps * __expf(emin - meas_e3(m, u0, u1, u2 + 2.0f));
    x.w *= ps * __expf(emin - meas_e3(m, u0, u1, u2 + 3.0f));
    *(float4*)(out + q * 4) = x;
    // four points along axis 2 at (u0, u1, u2 .. u2 + 3)
    const float a0 = x.x + x.y + x.z + x.w;
    const float a1 = x.y + 2.0f * x.z + 3.0f * x.w;
    const float a2 = x.y + 4.0f * x.z + 9.0f * x.w;
    const float b2 = fmaf(u2, a0, a1);
    f[0] += a0;                                       // S0
    f[1] = fmaf(a0, u0, f[1]);                        // S1_0
    f[2] = fmaf(a0, u1, f[2]);                        // S1_1
    f[3] += b2;                                       // S1_2
    f[4] = fmaf(a0 * u0, u0, f[4]);                   // S2_00
    f[5] = fmaf(a0 * u0, u1, f[5]);                   // S2_01
    f[6] = fmaf(b2, u0, f[6]);                        // S2_02
    f[7] = fmaf(a0 * u1, u1, f[7]);                   // S2_11
    f[8] = fmaf(b2, u1, f[8]);                        // S2_12
    f[9] += fmaf(u2, fmaf(u2, a0, 2.0f * a1), a2);    // S2_22
  }
  // a warp's sums by a float32 tree (at most a few hundred points, so the
  // tree's rounding stays near 5 ulp), then double-float across the warps:
  // slots S0, S1[0..2], S2_00, S2_01 | S2_02, S2_11, S2_12, S2_22
#pragma unroll
  for (int i = 0; i < 10; ++i)
    for (int o = 16; o; o >>= 1) f[i] += __shfl_xor_sync(0xffffffffu, f[i], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 10; ++i) sh.redw[warp][i] = f[i];
  __syncthreads();
  if (warp == 0) {
    DF* out = job.partials + (size_t)blk * 16;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      DF v{lane < kT / 32 ? sh.redw[lane][i] : 0.0f, 0.0f};
      for (int o = kT / 64; o; o >>= 1) {
        DF b{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, b);
      }
      if (lane == 0) out[i] = v;
    }
  }
}

// Sum the per-CTA partials (16 double-float slots each: S0, S1[0..2], S2_00,
// S2_01 | S2_02, S2_11, S2_12, S2_22, ...) into tot = {S0, S1[3], S2[6]}:
// double-float throughout, lanes 0..9 of warp 0 convert the totals to float64.
__device__ void sum_partials3(const DF* part, int nb, double* tot, DF (*red)[10] /* smem [kT/32] */) {
  DF a[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) a[i] = DF{0.0f, 0.0f};
  for (int b = threadIdx.x; b < nb; b += kT) {
    const DF* p = part + (size_t)b * 16;
#pragma unroll
    for (int i = 0; i < 10; ++i) a[i] = df_add(a[i], p[i]);
  }
#pragma unroll
  for (int i = 0; i < 10; ++i)
    for (int o = 16; o; o >>= 1) {
      DF q{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
      a[i] = df_add(a[i], q);
    }
  const int lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 10; ++i) red[threadIdx.x >> 5][i] = a[i];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      a[i] = lane < kT / 32 ? red[lane][i] : DF{0.0f, 0.0f};
      for (int o = kT / 64; o; o >>= 1) {
        DF q{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
        a[i] = df_add(a[i], q);
      }
    }
    DF mine = a[0];
#pragma unroll
    for (int i = 1; i < 10; ++i)
      if (lane == i) mine = a[i];
    if (lane < 10) tot[lane] = (double)mine.hi + (double)mine.lo;
    __syncwarp();
  }
}

// Moments after the measurement update; then (time update) the frame, the
// sub-step coefficients and the regrid rows of all axes.
__global__ void __launch_bounds__(kT) k_frame3(const __grid_constant__ Batch3 b) {
  const Job3& job = job_at(b, blockIdx.x);
  const TimeConsts& tc = job.tc;
  const int nb = (job.flags & 1) ? job.mblocks : 0;
  const int do_meas = job.flags & 1, do_time = (job.flags >> 1) & 1;
  __shared__ FrameState fs;
  __shared__ double tot[10];
  __shared__ DF red[kT / 32][10];
  __shared__ double Mpi[9];
  __shared__ int ok;
  DevState* st = job.st;
  constexpr int kW = sizeof(FrameState) / 8;
  for (int i = threadIdx.x; i < kW; i += kT) ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  __syncthreads();
  if (do_meas) sum_partials3(job.partials, nb, tot, red);
  if (threadIdx.x < 32) {
    bool good = true;
    if (do_meas) {
      good = finalize_warp<3>(&fs, tot, 0, nullptr);
      if (good && threadIdx.x == 0) fs.cur ^= 1;   // the multiplied weights are in the other buffer
      __syncwarp();
    }
    if (good && do_time) frame_warp<3>(tc, &fs, job.pend, Mpi);
    if (threadIdx.x == 0) ok = good;
  }
  __syncthreads();
  if (threadIdx.x == 0) job.up->skip = !(ok && do_time);
  if (ok && do_time) {
    Update3* up = job.up;
    const int l = fs.l;
    for (int q = threadIdx.x; q < l; q += kT) {
      double pa[4], pb[6];
      frame_substep<3>(tc, Mpi, q, pa, pb);
      for (int a = 0; a < 3; ++a) {
        up->pa[q][a] = (float)pa[a];
        up->pb[q][a] = (float)pb[a];
      }
    }
    if (threadIdx.x == 0) {
      up->l = l;
      up->exact = fs.exact;
      up->realign = fs.realign;
      up->gsc = (float)(fs.g / ((double)job.g.N[0] * job.g.N[1] * job.g.N[2]));
      up->shear[24] = 0.0;
      for (int a = 0; a < 3; ++a) up->wmax[a] = 0u;
      if (fs.realign && tc.realign_mode == PMF_REALIGN_SHEAR && !shear3_setup(fs, up->shear))
        fs.status = PMF_ERR_DEGENERATE;
    }
    if (!fs.realign)
      for (int a = 0; a < 3; ++a) regrid_rows(up->rows[a], fs.rs[a], fs.rd[a], job.g.N[a], threadIdx.x, kT);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kW; i += kT) ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
  if (threadIdx.x == 0) *job.emin_bits = 0x7f7f7f7fu;   // re-armed for the next measurement update
}

// Folded forward matrices of a kept frame: W_a[k][j] = sum_n H_a[k][n] I_a[n][j]
// with H_a the unnormalised Hartley matrix cas(2 pi k n / N) and I_a the
// periodic-sinc regrid matrix of eq. interFreq (rows: new nodes n, columns:
// old nodes j), so the slice and tile kernels apply the regrid and the
// forward transform of an axis as one GEMM.  A unit is (axis, 8 rows k); the
// four 128-thread groups of the CTA sum quarters of n for column j (float32),
// and the unit's max |W| goes to wmax[a] (the operand scale of the consumers).
constexpr int kFoldRows = 8;

__device__ __forceinline__ int fold_units(const Geo3& g) {
  return (g.N[0] + kFoldRows - 1) / kFoldRows + (g.N[1] + kFoldRows - 1) / kFoldRows +
         (g.N[2] + kFoldRows - 1) / kFoldRows;
}

__device__ void fold_unit(const Job3& job, int u) {
  __shared__ float hs[kFoldRows][128];
  __shared__ float part[4][kFoldRows][128];
  __shared__ float bmax[kT / 32];
  __shared__ RegridRows rows;
  int a = 0;
  while (a < 2 && u >= (job.g.N[a] + kFoldRows - 1) / kFoldRows) {
    u -= (job.g.N[a] + kFoldRows - 1) / kFoldRows;
    ++a;
  }
  const int N = job.g.N[a], k0 = u * kFoldRows;
  const float* sct = job.sctab[a];
  {
    // the axis' regrid row parameters, read by every thread for every n
    const unsigned int* src = (const unsigned int*)&job.up->rows[a];
    unsigned int* dst = (unsigned int*)&rows;
    for (int i = threadIdx.x; i < (int)(sizeof(RegridRows) / 4); i += kT) dst[i] = src[i];
  }
  // H rows k0 .. k0 + kFoldRows - 1 from the (cos, sin)(pi m / N) table: cas(2 pi r / N), r = k n mod N
  for (int t = threadIdx.x; t < kFoldRows * N; t += kT) {
    const int kr = t / N, n = t - kr * N, k = k0 + kr;
    float h = 0.0f;
    if (k < N) {
      const int r = (k * n) % N, m = 2 * r <= N ? 2 * r : 2 * r - 2 * N;
      h = sct[2 * (m + N)] + sct[2 * (m + N) + 1];
    }
    hs[kr][n] = h;
  }
  __syncthreads();
  const int grp = threadIdx.x >> 7, j = threadIdx.x & 127;
  const int q = (N + 3) / 4, nb = grp * q, ne = min(N, nb + q);
  float acc[kFoldRows];
#pragma unroll
  for (int r = 0; r < kFoldRows; ++r) acc[r] = 0.0f;
  if (j < N)
    for (int n = nb; n < ne; ++n) {
      const float x = interp_value(regrid_row(rows, n), j, N, sct);
#pragma unroll
      for (int r = 0; r < kFoldRows; ++r) acc[r] = fmaf(hs[r][n], x, acc[r]);
    }
#pragma unroll
  for (int r = 0; r < kFoldRows; ++r) part[grp][r][j] = acc[r];
  __syncthreads();
  float m = 0.0f;
  float* dst = job.fold + (size_t)a * 128 * 128;
  for (int t = threadIdx.x; t < kFoldRows * 128; t += kT) {
    const int kr = t >> 7, jj = t & 127, k = k0 + kr;
    if (k < N && jj < N) {
      const float w = (part[0][kr][jj] + part[1][kr][jj]) + (part[2][kr][jj] + part[3][kr][jj]);
      dst[k * 128 + jj] = w;
      m = fmaxf(m, fabsf(w));
    }
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) bmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int w = 0; w < kT / 32; ++w) v = fmaxf(v, bmax[w]);
    atomicMax(&job.up->wmax[a], __float_as_uint(v));
  }
  __syncthreads();   // the shared arrays are reused by the CTA's next unit
}

// Folded matrix of axis a into the W planes, scaled by a power of two (16-bit
// float: max |W| into [2^14, 2^15), the exponent capped as for the data
// operands); returns the scale.  Consecutive threads take consecutive rows.
template <int P>
__device__ float load_fold(const Job3& job, int a, uint8_t* W) {
  const int N = job.g.N[a];
  float sc = 1.0f;
  if (P == PMF_PREC_FP16X3) {
    const float wmax = __uint_as_float(job.up->wmax[a]);
    if (wmax > 0.0f && wmax < INFINITY) {
      int e;
      frexpf(wmax, &e);
      sc = ldexpf(1.0f, min(15 - e, 100));
    }
  }
  const float* src = job.fold + (size_t)a * 128 * 128;
  const int q4 = N / 4;
  for (int t = threadIdx.x; t < N * q4; t += kT) {
    const int n = t % N, c = (t / N) * 4;
    store4<P>(W, n, c, *(const float4*)(src + n * 128 + c), sc);
  }
  return sc;
}

// Multilinear re-alignment (only when the frame kernel decided it): gather
// buf[cur] -> buf[cur^1] with pscale folded in; k_copy3 copies it back.  When
// the frame was kept, the CTAs form the folded forward matrices instead.
__global__ void __launch_bounds__(kT) k_realign3(const __grid_constant__ Batch3 b) {
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindPoints, blockIdx.x, &blk, &cnt));
  const FrameState& f = job.st->f;
  if (job.up->skip) return;
  if (!job.up->realign) {
    const int units = fold_units(job.g);
    for (int u = blk; u < units; u += cnt) fold_unit(job, u);
    return;
  }
  if (job.tc.realign_mode == PMF_REALIGN_SHEAR) return;
  const Geo3& g = job.g;
  const float* in = f.cur ? job.buf1 : job.buf0;
  float* out = f.cur ? job.buf0 : job.buf1;
  const float ps = (float)f.pscale;
  for (long long p = blk * (long long)kT + threadIdx.x; p < g.P; p += (long long)cnt * kT) {
    int j[3];
    unflat3(g, p, j);
    double z[3];
    int fl[3];
    float w[3];
    for (int a = 0; a < 3; ++a) {
      double uo = f.b[a];
      for (int b = 0; b < 3; ++b) uo = fma(f.B[a * 3 + b], j[b] - 0.5 * (g.N[b] - 1), uo);
      z[a] = uo + 0.5 * (g.N[a] - 1);
      const double fz = floor(z[a]);
      fl[a] = (int)fmax(fmin(fz, 1e6), -1e6);
      w[a] = (float)(z[a] - fz);
    }
    float s = 0.0f;
    for (int c = 0; c < 8; ++c) {
      float wt = 1.0f;
      long long off = 0;
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        const int bit = (c >> a) & 1, i = fl[a] + bit;
        wt *= bit ? w[a] : 1.0f - w[a];
        ok = ok && i >= 0 && i < g.N[a];
        off = off * g.N[a] + (ok ? i : 0);
      }
      if (ok) s += wt * in[off];
    }
    out[p] = ps * s;
  }
}

__global__ void __launch_bounds__(kT) k_copy3(const __grid_constant__ Batch3 b) {
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindPoints, blockIdx.x, &blk, &cnt));
  const FrameState& f = job.st->f;
  if (job.up->skip || !job.up->realign) return;
  const float* src = f.cur ? job.buf0 : job.buf1;
  float* dst = f.cur ? job.buf1 : job.buf0;
  for (long long p = blk * (long long)kT + threadIdx.x; p < job.g.P; p += (long long)cnt * kT)
    dst[p] = src[p];
}

// Band-limited re-alignment (shear mode), one of three line-wise passes: one
// CTA per line along the pass's axis (the job owns N0 N1 N2 / min N CTAs; the
// surplus exits).  Per line the DFT coefficients (float32, exact twiddle
// indices), then the trigonometric interpolant (eq. interFreq) at the line's
// positions alpha . u_S + beta . w_T + gamma (float64 positions, float32
// evaluation by a recurrence from e^{2 pi i x / N}); positions outside the old
// box give 0.  Buffers: pass 0 buf[cur] -> buf[cur ^ 1], pass 1 back, pass 2
// buf[cur] -> buf[cur ^ 1] with pscale (k_copy3 then copies it back).
constexpr int kShearT = 128;   // threads per line CTA (N <= 128)

__global__ void __launch_bounds__(kShearT) k_shear3p(const __grid_constant__ Batch3 b, int pass) {
  __shared__ float fl[128], cs[128], sn[128], Xr[65], Xi[65];
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindShear, blockIdx.x, &blk, &cnt));
  const Update3* up = job.up;
  if (up->skip || !up->realign || up->shear[24] == 0.0) return;
  const FrameState& f = job.st->f;
  const double* pc = up->shear + 8 * pass;
  const int a = (int)pc[0];
  const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
  const int N = job.g.N[a], H = N / 2, N1 = job.g.N[o1], N2 = job.g.N[o2];
  if (blk >= N1 * N2) return;
  const int i1 = blk / N2, i2 = blk % N2;
  const long long stride[3] = {(long long)job.g.N[1] * job.g.N[2], job.g.N[2], 1};
  const long long base = i1 * stride[o1] + i2 * stride[o2], sa = stride[a];
  float* bc = f.cur ? job.buf1 : job.buf0;
  float* bn = f.cur ? job.buf0 : job.buf1;
  const float* in = pass == 1 ? bn : bc;
  float* out = pass == 1 ? bc : bn;
  for (int t = threadIdx.x; t < N; t += kShearT) {
    fl[t] = in[base + t * sa];
    sincospif(2.0f * (float)t / (float)N, &sn[t], &cs[t]);
  }
  __syncthreads();
  for (int sidx = threadIdx.x; sidx <= H; sidx += kShearT) {
    float re = 0.0f, im = 0.0f;
    int r = 0;
    for (int j = 0; j < N; ++j) {
      re = fmaf(fl[j], cs[r], re);
      im = fmaf(-fl[j], sn[r], im);
      r += sidx;
      if (r >= N) r -= N;
    }
    Xr[sidx] = re / (float)N;
    Xi[sidx] = im / (float)N;
  }
  __syncthreads();
  const double offset = pc[4] + pc[1 + o1] * (i1 - 0.5 * (N1 - 1)) + pc[1 + o2] * (i2 - 0.5 * (N2 - 1));
  const float ps = pass == 2 ? (float)f.pscale : 1.0f;
  for (int t = threadIdx.x; t < N; t += kShearT) {
    const double pos = offset + pc[1 + a] * (t - 0.5 * (N - 1));
    float v = 0.0f;
    if (fabs(pos) <= 0.5 * N) {
      const double x = pos + 0.5 * (N - 1);
      float sx, cx;
      sincospif((float)(2.0 * x / N), &sx, &cx);
      float zr = 1.0f, zi = 0.0f;   // e^{2 pi i s x / N}
      v = Xr[0];
      for (int k = 1; k < H; ++k) {
        const float nr = zr * cx - zi * sx;
        zi = zr * sx + zi * cx;
        zr = nr;
        v += 2.0f * (Xr[k] * zr - Xi[k] * zi);
      }
      v += Xr[H] * cospif((float)x);
    }
    out[base + t * sa] = ps * v;
  }
}

// =========================== pipeline A (slices) =============================
// Slice j0 of buf[cur] (rows j1, columns j2) -> regrid + Hartley along axis 2,
// then axis 1 (one GEMM each) -> T[j0][k1][k2] in buf[cur^1].
template <int P>
__global__ void __launch_bounds__(kT, 1) k_slices_fwd(const __grid_constant__ Batch3 b) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Smem3 sh;
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindSlices, blockIdx.x, &blk, &cnt));
  uint8_t* A = smem + kOffA;
  uint8_t* W = smem + kOffW;
  float* S = (float*)(smem + kOffS);
  const FrameState& f = job.st->f;
  const Update3* up = job.up;
  const int N1 = job.g.N[1], N2 = job.g.N[2];
  const int j0 = blk;
  if (up->skip) return;
  const int realign = up->realign;
  const float* in = f.cur ? job.buf1 : job.buf0;
  float* out = f.cur ? job.buf0 : job.buf1;
  const float ps = realign ? 1.0f : (float)f.pscale;   // the re-aligned copy already carries it
  const float sw = P == PMF_PREC_FP16X3 ? 16384.0f : 1.0f;
  Pipe p;
  pipe_init(sh, p);
  const float* src = in + (size_t)j0 * N1 * N2;
  const int q2 = N2 / 4;
  float m = 0.0f;
  for (int t = threadIdx.x; t < N1 * q2; t += kT) {
    const int r = t / q2, c = (t % q2) * 4;
    float4 x = *(const float4*)(src + (size_t)r * N2 + c);
    x.x *= ps;
    x.y *= ps;
    x.z *= ps;
    x.w *= ps;
    *(float4*)(S + r * kSStr + c) = x;
    m = amax4(m, x);
  }
  float sa = op_scale<P>(block_max3(sh, m, 0));
  stage_to_op<P>(A, S, N1, N2, sa);
  // regrid and transform of an axis in one GEMM: the folded matrix of a kept
  // frame, the Hartley matrix after a re-alignment (the gather moved the weights)
  float wsc = realign ? sw : load_fold<P>(job, 2, W);
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, realign ? job.hart[2] : nullptr, N2, 0, N2, N2);   // F2 (regrid folded in)
  float inv = 1.0f / (sa * wsc);
  if (!pipe_wait(sh, p)) goto fail;
  sa = acc_to_operand<P>(sh, p, A, N1, N2, inv, P == PMF_PREC_TF32, 0);     // [j1][k2]: MN-major next
  wsc = realign ? sw : load_fold<P>(job, 1, W);
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, realign ? job.hart[1] : nullptr, N1, P != PMF_PREC_TF32, N1, N1);   // F1: lanes k2
  inv = 1.0f / (sa * wsc);
  if (!pipe_wait(sh, p)) goto fail;
  {
    // T[j0][k1][k2]: lane k2, column k1 (consecutive lanes: consecutive addresses)
    const int row = threadIdx.x & 127, cg = threadIdx.x >> 7;
    const int ncol = N1 / 4, c0 = cg * ncol;
    float* dst = out + (size_t)j0 * N1 * N2;
    for (int c = 0; c < ncol; c += 4) {
      const float4 v = tmem_ld4(p.tlane + c0 + c);
      if (row < N2) {
        dst[(size_t)(c0 + c + 0) * N2 + row] = v.x * inv;
        dst[(size_t)(c0 + c + 1) * N2 + row] = v.y * inv;
        dst[(size_t)(c0 + c + 2) * N2 + row] = v.z * inv;
        dst[(size_t)(c0 + c + 3) * N2 + row] = v.w * inv;
      }
    }
  }
  pipe_done(sh, p);
  return;
fail:
  if (threadIdx.x == 0) job.st->f.status = PMF_ERR_TIMEOUT;
  pipe_done(sh, p);
}

// ======================= pipeline B (axis-0 line tiles) ======================
// Tile (k1, chunk): lines {k1, -k1} x (C u -C) with C = [32 chunk, 32 chunk + 32)
// intersected with [0, N2/2]; line index s1 * 64 + i (k2 = C[i]) and
// s1 * 64 + 32 + i (k2 = -C[i]).
template <int P>
__global__ void __launch_bounds__(kT, 1) k_lines_axis0(const __grid_constant__ Batch3 b) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Smem3 sh;
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindLines, blockIdx.x, &blk, &cnt));
  const int chunks = job.chunks;
  __shared__ int lk1[128], lk2[128];
  __shared__ unsigned char lwr[128];   // line written back (the first copy of a self-mirrored line)
  __shared__ float spa[MAXL][3], spb[MAXL][3];
  uint8_t* A = smem + kOffA;
  uint8_t* W = smem + kOffW;
  float* S = (float*)(smem + kOffS);
  const FrameState& f = job.st->f;
  const Update3* up = job.up;
  const int N0 = job.g.N[0], N1 = job.g.N[1], N2 = job.g.N[2];
  const int k1 = blk / chunks, chunk = blk % chunks;
  const int cbeg = 32 * chunk, cend = min(32 * chunk + 32, N2 / 2 + 1), nc = cend - cbeg;
  if (up->skip) return;
  const int realign = up->realign;
  float* T = f.cur ? job.buf0 : job.buf1;   // written by the slice kernel
  const size_t plane = (size_t)N1 * N2;
  const float sw = P == PMF_PREC_FP16X3 ? 16384.0f : 1.0f;
  for (int L = threadIdx.x; L < 128; L += kT) {
    const int s1 = L >> 6, i = L & 31, mir = (L >> 5) & 1;
    const int kk1 = s1 ? (N1 - k1) % N1 : k1;
    const int c = cbeg + i;
    lk1[L] = kk1;
    lk2[L] = i < nc ? (mir ? (N2 - c) % N2 : c) : -1;
    // k1 = -k1 (0, N1/2) or k2 = -k2 (0, N2/2): the tile holds the line twice;
    // the two copies agree only up to rounding, so one of them is written back
    lwr[L] = i < nc && !(s1 && kk1 == k1) && !(mir && (N2 - c) % N2 == c);
  }
  Pipe p;
  pipe_init(sh, p);
  // gather the lines: S[line][j0]
  float m = 0.0f;
  for (int t = threadIdx.x; t < 128 * (N0 / 4); t += kT) {
    const int L = t & 127, q = t >> 7;
    float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (lk2[L] >= 0) {
      const float* src = T + (size_t)lk1[L] * N2 + lk2[L];
      x.x = src[(size_t)(4 * q + 0) * plane];
      x.y = src[(size_t)(4 * q + 1) * plane];
      x.z = src[(size_t)(4 * q + 2) * plane];
      x.w = src[(size_t)(4 * q + 3) * plane];
    }
    *(float4*)(S + L * kSStr + 4 * q) = x;
    m = amax4(m, x);
  }
  float sa = op_scale<P>(block_max3(sh, m, 0));
  stage_to_op<P>(A, S, 128, N0, sa);
  const float wsc = realign ? sw : load_fold<P>(job, 0, W);
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, realign ? job.hart[0] : nullptr, N0, 0, N0, N0);   // F0 (regrid folded in)
  float inv = 1.0f / (sa * wsc);
  if (!pipe_wait(sh, p)) goto fail;
  acc_to_stage(p, S, N0, inv);
  __syncthreads();
  {
    // diffusion multiplier on 8-point orbits (+-k0, +-k1, +-k2); bit 0 of a
    // sign pattern flips k0, bit 1 k1, bit 2 k2
    const float two_pi = 6.28318530717958647692f;
    const int H0 = N0 / 2 + 1;
    const int l = up->l, exact = up->exact;
    const float gsc = up->gsc;
    for (int q = threadIdx.x; q < l * 3; q += kT) {
      spa[q / 3][q % 3] = up->pa[q / 3][q % 3];
      spb[q / 3][q % 3] = up->pb[q / 3][q % 3];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < H0 * nc; o += kT) {
      const int k0 = o % H0, i = o / H0;
      const int col[2] = {k0, (N0 - k0) % N0};
      float Sv[8], Ps[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int L = ((s >> 1) & 1) * 64 + ((s >> 2) & 1) * 32 + i;
        Sv[s] = S[L * kSStr + col[s & 1]];
      }
      // Over the orbit the squared wavenumbers are fixed and a flipped index
      // negates the first-derivative coefficient (zero at 0 and N/2), so the
      // sub-step exponent of pattern s is E + s01 X01 + s02 X02 + s12 X12 with
      // s_ab = sigma_a sigma_b: four distinct values (s and s ^ 7 agree), formed
      // from one read of the sub-step coefficients.  Magnitudes from pattern 0.
      {
        const int a0 = k0, a1 = lk1[i], a2 = lk2[i];
        const int w0 = a0 < N0 / 2 ? a0 : a0 - N0, w1 = a1 < N1 / 2 ? a1 : a1 - N1, w2 = a2 < N2 / 2 ? a2 : a2 - N2;
        const float q0 = two_pi * w0 / N0, q1 = two_pi * w1 / N1, q2 = two_pi * w2 / N2;
        const float t0 = (2 * a0 == N0) ? 0.0f : q0, t1 = (2 * a1 == N1) ? 0.0f : q1, t2 = (2 * a2 == N2) ? 0.0f : q2;
        const float q00 = q0 * q0, q11 = q1 * q1, q22 = q2 * q2, c01 = t0 * t1, c02 = t0 * t2, c12 = t1 * t2;
        float den[4] = {1.0f, 1.0f, 1.0f, 1.0f}, ex[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int qq = 0; qq < l; ++qq) {
          const float E = spa[qq][0] * q00 + spa[qq][1] * q11 + spa[qq][2] * q22;
          const float x01 = spb[qq][0] * c01, x02 = spb[qq][1] * c02, x12 = spb[qq][2] * c12;
          // patterns 0 (no flip), 1 (k0), 2 (k1), 3 (k0 and k1)
          const float e[4] = {E + x01 + x02 + x12, E - x01 - x02 + x12, E - x01 + x02 - x12, E + x01 - x02 - x12};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            den[h] *= 1.0f + e[h];
            ex[h] += e[h];
          }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int h = s < 4 ? s : s ^ 7;
          Ps[s] = exact ? expf(-ex[h]) : __frcp_rn(den[h]);
        }
      }
      float Tb[8], Pe[8], Tp[8];
#pragma unroll
      for (int B = 0; B < 8; ++B) {
        float tb = 0.0f, pe = 0.0f;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const float chi = (__popc(B & s) & 1) ? -1.0f : 1.0f;
          tb += chi * Sv[s];
          pe += chi * Ps[s];
        }
        Tb[B] = 0.125f * tb;
        Pe[B] = 0.125f * pe;
      }
#pragma unroll
      for (int C = 0; C < 8; ++C) {
        float acc = 0.0f;
#pragma unroll
        for (int E = 0; E < 8; ++E) {
          const int pe = __popc(E);
          if (pe & 1) continue;
          const int sg = ((pe >> 1) + __popc(E & C)) & 1;
          acc += (sg ? -1.0f : 1.0f) * Pe[E] * Tb[E ^ C];
        }
        Tp[C] = acc * gsc;
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        float v = 0.0f;
#pragma unroll
        for (int C = 0; C < 8; ++C) v += ((__popc(C & s) & 1) ? -1.0f : 1.0f) * Tp[C];
        Sv[s] = v;
      }
      // duplicate lines/columns of self-mirrored frequencies receive equal values
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int L = ((s >> 1) & 1) * 64 + ((s >> 2) & 1) * 32 + i;
        S[L * kSStr + col[s & 1]] = Sv[s];
      }
    }
  }
  __syncthreads();
  sa = op_scale<P>(block_max3(sh, stage_absmax(S, 128, N0), 1));
  stage_to_op<P>(A, S, 128, N0, sa);
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, realign ? nullptr : job.hart[0], N0, 0, N0, N0);   // V0 (H0 resident if re-aligned)
  inv = 1.0f / (sa * sw);
  if (!pipe_wait(sh, p)) goto fail;
  {
    const int row = threadIdx.x & 127, cg = threadIdx.x >> 7;
    const int ncol = N0 / 4, c0 = cg * ncol;
    const bool ok = lwr[row] != 0;
    float* dst = T + (size_t)lk1[row] * N2 + (ok ? lk2[row] : 0);
    for (int c = 0; c < ncol; c += 4) {
      const float4 v = tmem_ld4(p.tlane + c0 + c);
      if (ok) {
        dst[(size_t)(c0 + c + 0) * plane] = v.x * inv;
        dst[(size_t)(c0 + c + 1) * plane] = v.y * inv;
        dst[(size_t)(c0 + c + 2) * plane] = v.z * inv;
        dst[(size_t)(c0 + c + 3) * plane] = v.w * inv;
      }
    }
  }
  pipe_done(sh, p);
  return;
fail:
  if (threadIdx.x == 0) job.st->f.status = PMF_ERR_TIMEOUT;
  pipe_done(sh, p);
}

// ======================= pipeline C (inverse slices) =========================
// T[j0][k1][k2] (rows k1, columns k2) -> inverse along axis 2, then axis 1 ->
// weights[j0][j1][j2] in buf[cur]; moment partials per CTA.
template <int P>
__global__ void __launch_bounds__(kT, 1) k_slices_inv(const __grid_constant__ Batch3 b) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Smem3 sh;
  int blk, cnt;
  const Job3& job = job_at(b, find_job(b, kKindSlices, blockIdx.x, &blk, &cnt));
  uint8_t* A = smem + kOffA;
  uint8_t* W = smem + kOffW;
  float* S = (float*)(smem + kOffS);
  const FrameState& f = job.st->f;
  const int N0 = job.g.N[0], N1 = job.g.N[1], N2 = job.g.N[2];
  const int j0 = blk;
  if (job.up->skip) return;
  const float* T = f.cur ? job.buf0 : job.buf1;
  float* out = f.cur ? job.buf1 : job.buf0;
  const float sw = P == PMF_PREC_FP16X3 ? 16384.0f : 1.0f;
  Pipe p;
  pipe_init(sh, p);
  const float* src = T + (size_t)j0 * N1 * N2;
  const int q2 = N2 / 4;
  float m = 0.0f;
  for (int t = threadIdx.x; t < N1 * q2; t += kT) {
    const int r = t / q2, c = (t % q2) * 4;
    const float4 x = *(const float4*)(src + (size_t)r * N2 + c);
    *(float4*)(S + r * kSStr + c) = x;
    m = amax4(m, x);
  }
  float sa = op_scale<P>(block_max3(sh, m, 0));
  stage_to_op<P>(A, S, N1, N2, sa);
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, job.hart[2], N2, 0, N2, N2);                   // V2: lanes k1, cols j2
  float inv = 1.0f / (sa * sw);
  if (!pipe_wait(sh, p)) goto fail;
  sa = acc_to_operand<P>(sh, p, A, N1, N2, inv, P == PMF_PREC_TF32, 1);     // [k1][j2]: MN-major next
  fence_async_smem();
  __syncthreads();
  pipe_issue<P>(sh, p, A, W, job.hart[1], N1, P != PMF_PREC_TF32, N1, N1);  // V1: lanes j2, cols j1
  inv = 1.0f / (sa * sw);
  if (!pipe_wait(sh, p)) goto fail;
  {
    const int row = threadIdx.x & 127, cg = threadIdx.x >> 7;
    const int ncol = N1 / 4, c0 = cg * ncol;
    float* dst = out + (size_t)j0 * N1 * N2;
    const float u0 = j0 - 0.5f * (N0 - 1), u2 = row - 0.5f * (N2 - 1);
    DF s[6];
    for (int i = 0; i < 6; ++i) s[i] = DF{0.0f, 0.0f};
    DF s2[4];
    for (int i = 0; i < 4; ++i) s2[i] = DF{0.0f, 0.0f};
    for (int c = 0; c < ncol; c += 4) {
      float4 v = tmem_ld4(p.tlane + c0 + c);
      v.x *= inv;
      v.y *= inv;
      v.z *= inv;
      v.w *= inv;
      if (row < N2) {
        const int j1 = c0 + c;
        dst[(size_t)(j1 + 0) * N2 + row] = v.x;
        dst[(size_t)(j1 + 1) * N2 + row] = v.y;
        dst[(size_t)(j1 + 2) * N2 + row] = v.z;
        dst[(size_t)(j1 + 3) * N2 + row] = v.w;
        // four points along axis 1 at (u0, u1 .. u1 + 3, u2)
        const float u1 = j1 - 0.5f * (N1 - 1);
        const float a0 = v.x + v.y + v.z + v.w;
        const float a1 = v.y + 2.0f * v.z + 3.0f * v.w;
        const float a2 = v.y + 4.0f * v.z + 9.0f * v.w;
        const float b1 = fmaf(u1, a0, a1);
        s[0] = df_add1(s[0], a0);
        s[1] = df_add1(s[1], a0 * u0);
        s[2] = df_add1(s[2], b1);
        s[3] = df_add1(s[3], a0 * u2);
        s[4] = df_add1(s[4], a0 * u0 * u0);
        s[5] = df_add1(s[5], b1 * u0);
        s2[0] = df_add1(s2[0], a0 * u0 * u2);                              // S2_02
        s2[1] = df_add1(s2[1], fmaf(u1, fmaf(u1, a0, 2.0f * a1), a2));     // S2_11
        s2[2] = df_add1(s2[2], b1 * u2);                                   // S2_12
        s2[3] = df_add1(s2[3], a0 * u2 * u2);                              // S2_22
      }
    }
    tc_before_sync();
    DF* part = job.partials + (size_t)j0 * 16;
    block_partials3(sh, s, part);
    __syncthreads();
    DF t4[6] = {s2[0], s2[1], s2[2], s2[3], DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
    block_partials3(sh, t4, part + 6);
  }
  pipe_done(sh, p);
  return;
fail:
  if (threadIdx.x == 0) job.st->f.status = PMF_ERR_TIMEOUT;
  pipe_done(sh, p);
}

// Moments of the new weights, normaliser and frame commit (one CTA).
__global__ void __launch_bounds__(kT) k_commit3(const __grid_constant__ Batch3 b) {
  const Job3& job = job_at(b, blockIdx.x);
  const int nb = job.g.N[0];
  __shared__ FrameState fs;
  __shared__ double tot[10];
  __shared__ DF red[kT / 32][10];
  DevState* st = job.st;
  if (job.up->skip) return;
  constexpr int kW = sizeof(FrameState) / 8;
  for (int i = threadIdx.x; i < kW; i += kT) ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  __syncthreads();
  sum_partials3(job.partials, nb, tot, red);
  if (threadIdx.x < 32 && finalize_warp<3>(&fs, tot, 1, job.pend) && threadIdx.x == 0) {
    fs.hc[0] = atan2(fs.c[1], fs.c[0]);
    fs.hc[1] = fs.c[0] * fs.c[0] + fs.c[1] * fs.c[1];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kW; i += kT) ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
}

}  // namespace

// ------------------------------- host side ----------------------------------
struct Tc3State {
  Update3* up = nullptr;
  double* pend = nullptr;
  DF* partials = nullptr;
  unsigned int* emin = nullptr;
  float* fold = nullptr;  // folded forward matrices, 3 x 128 x 128
  Tc3Stage stage[2];    // single-filter launches alternate between two stagings
  int parity = 0;
};

int tc3_alloc(void** handle) {
  Tc3State* s = new (std::nothrow) Tc3State();
  if (!s) return PMF_ERR_OOM;
  if (cudaMalloc(&s->up, sizeof(Update3)) != cudaSuccess || cudaMalloc(&s->pend, 32 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s->partials, 16 * 4096 * sizeof(DF)) != cudaSuccess ||
      cudaMalloc(&s->emin, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&s->fold, 3 * 128 * 128 * sizeof(float)) != cudaSuccess ||
      cudaMemset(s->emin, 0x7f, sizeof(unsigned int)) != cudaSuccess) {
    tc3_free(s);
    return PMF_ERR_OOM;
  }
  static bool attr = false;
  if (!attr) {
#define PMF_SET(k) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)
    PMF_SET(k_slices_fwd<PMF_PREC_FP16X3>);
    PMF_SET(k_slices_fwd<PMF_PREC_BF16X3>);
    PMF_SET(k_slices_fwd<PMF_PREC_TF32>);
    PMF_SET(k_lines_axis0<PMF_PREC_FP16X3>);
    PMF_SET(k_lines_axis0<PMF_PREC_BF16X3>);
    PMF_SET(k_lines_axis0<PMF_PREC_TF32>);
    PMF_SET(k_slices_inv<PMF_PREC_FP16X3>);
    PMF_SET(k_slices_inv<PMF_PREC_BF16X3>);
    PMF_SET(k_slices_inv<PMF_PREC_TF32>);
#undef PMF_SET
    attr = true;
  }
  *handle = s;
  return PMF_OK;
}

size_t tc3_state_bytes() {
  return sizeof(Update3) + 32 * sizeof(double) + 16 * 4096 * sizeof(DF) + sizeof(unsigned int) +
         3 * 128 * 128 * sizeof(float) + 2 * (sizeof(Job3) + (kKinds + 1) * 2 * sizeof(int));
}

void tc3_free(void* handle) {
  Tc3State* s = (Tc3State*)handle;
  if (!s) return;
  cudaFree(s->up);
  cudaFree(s->pend);
  cudaFree(s->partials);
  cudaFree(s->emin);
  cudaFree(s->fold);
  tc3_stage_free(&s->stage[0]);
  tc3_stage_free(&s->stage[1]);
  delete s;
}

int tc3_stage_reserve(Tc3Stage* g, int n) {
  if (g->ev && cudaEventSynchronize(g->ev) != cudaSuccess) return PMF_ERR_CUDA;
  if (n <= g->cap) return PMF_OK;
  cudaFreeHost(g->h_jobs);
  cudaFreeHost(g->h_first);
  cudaFree(g->d_jobs);
  cudaFree(g->d_first);
  *g = Tc3Stage{nullptr, nullptr, nullptr, nullptr, 0, g->ev};
  const int cap = n < 16 ? 16 : n;
  const size_t fb = sizeof(int) * kKinds * (size_t)(cap + 1);
  if (cudaMallocHost(&g->h_jobs, sizeof(Job3) * cap) != cudaSuccess || cudaMallocHost(&g->h_first, fb) != cudaSuccess ||
      cudaMalloc(&g->d_jobs, sizeof(Job3) * cap) != cudaSuccess || cudaMalloc(&g->d_first, fb) != cudaSuccess)
    return PMF_ERR_OOM;
  if (!g->ev && cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess) return PMF_ERR_CUDA;
  g->cap = cap;
  return PMF_OK;
}

void tc3_stage_free(Tc3Stage* g) {
  cudaFreeHost(g->h_jobs);
  cudaFreeHost(g->h_first);
  cudaFree(g->d_jobs);
  cudaFree(g->d_first);
  if (g->ev) cudaEventDestroy(g->ev);
  *g = Tc3Stage{};
}

namespace {

// CTAs of the measurement kernels of one filter: one per SM at most, so that
// each thread takes a few quads (the block reductions and the frame kernel's
// sum over the per-CTA partials are paid per CTA)
int meas_blocks(long long P) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
      nsm = 128;
  }
  return (int)std::min<long long>(std::min(nsm, 1024), (P / 4 + kT - 1) / kT);
}

template <int P>
void launch_pipes(const Batch3& b, const int* tot, cudaStream_t s) {
  k_slices_fwd<P><<<tot[kKindSlices], kT, kSmem, s>>>(b);
  k_lines_axis0<P><<<tot[kKindLines], kT, kSmem, s>>>(b);
  k_slices_inv<P><<<tot[kKindSlices], kT, kSmem, s>>>(b);
}

}  // namespace

int tc3_batch(const Tc3Item* items, int n, int precision, Tc3Stage* g, cudaStream_t s) {
  if (n <= 0) return 0;
  static thread_local Batch3 b;      // n == 1: built here, passed by value
  Job3* jobs = &b.one;
  int one_first[kKinds * 2];
  int* first = one_first;
  if (n > 1) {
    const int rc = tc3_stage_reserve(g, n);
    if (rc) return -rc;
    jobs = (Job3*)g->h_jobs;
    first = g->h_first;
  }
  int tot[kKinds] = {0, 0, 0, 0, 0};
  for (int k = 0; k < kKinds; ++k) first[k * (n + 1)] = 0;
  for (int i = 0; i < n; ++i) {
    const Tc3Item& it = items[i];
    const Tc3State* h = (const Tc3State*)it.handle;
    Job3& job = jobs[i];
    job.st = it.st;
    job.buf0 = it.b0;
    job.buf1 = it.b1;
    for (int a = 0; a < 3; ++a) {
      job.hart[a] = (const uint8_t*)it.t->hart[a];
      job.sctab[a] = (const float*)((const uint8_t*)it.t->hart[a] + it.t->hart_bytes[a]);
      job.g.N[a] = it.d.N[a];
    }
    job.g.P = it.d.P;
    job.partials = h->partials;
    job.emin_bits = h->emin;
    job.up = h->up;
    job.pend = h->pend;
    job.fold = h->fold;
    job.precision = precision;
    job.flags = (it.mp ? 1 : 0) | (it.tc ? 2 : 0);
    job.chunks = (it.d.N[2] / 2 + 1 + 31) / 32;
    job.mblocks = it.mp ? meas_blocks(it.d.P) : 0;
    if (it.mp) job.mp = *it.mp;
    if (it.tc) job.tc = *it.tc;
    const int nmin = std::min(it.d.N[0], std::min(it.d.N[1], it.d.N[2]));
    const bool shear = it.tc && it.tc->realign_mode == PMF_REALIGN_SHEAR;
    const int cnt[kKinds] = {it.mp ? meas_blocks(it.d.P) : 0,
                             it.tc ? (int)std::min<long long>(304, (it.d.P + kT - 1) / kT) : 0,
                             it.tc ? it.d.N[0] : 0, it.tc ? (it.d.N[1] / 2 + 1) * job.chunks : 0,
                             shear ? (int)(it.d.P / nmin) : 0};
    for (int k = 0; k < kKinds; ++k) {
      tot[k] += cnt[k];
      first[k * (n + 1) + i + 1] = tot[k];
    }
  }
  b.n = n;
  b.jobs = nullptr;
  b.first = nullptr;
  if (n > 1) {
    if (cudaMemcpyAsync(g->d_jobs, g->h_jobs, sizeof(Job3) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(g->d_first, g->h_first, sizeof(int) * kKinds * (n + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaEventRecord(g->ev, s) != cudaSuccess)
      return -PMF_ERR_CUDA;
    b.jobs = (const Job3*)g->d_jobs;
    b.first = g->d_first;
  }
  int launches = 0;
  if (tot[kKindMeas]) {
    k_meas_min3<<<tot[kKindMeas], kT, 0, s>>>(b);
    k_meas_apply3<<<tot[kKindMeas], kT, 0, s>>>(b);
    launches += 2;
  }
  k_frame3<<<n, kT, 0, s>>>(b);
  ++launches;
  if (tot[kKindSlices]) {
    k_realign3<<<tot[kKindPoints], kT, 0, s>>>(b);
    if (tot[kKindShear]) {
      for (int pass = 0; pass < 3; ++pass) k_shear3p<<<tot[kKindShear], kShearT, 0, s>>>(b, pass);
      launches += 3;
    }
    k_copy3<<<tot[kKindPoints], kT, 0, s>>>(b);
    if (precision == PMF_PREC_FP16X3) launch_pipes<PMF_PREC_FP16X3>(b, tot, s);
    else if (precision == PMF_PREC_BF16X3) launch_pipes<PMF_PREC_BF16X3>(b, tot, s);
    else launch_pipes<PMF_PREC_TF32>(b, tot, s);
    launches += 5;
  }
  k_commit3<<<n, kT, 0, s>>>(b);
  return launches + 1;
}

int tc3_step(void* handle, const Dims& d, const pmf_config& cfg, const TcTables* t, const MeasParams* mp,
             const TimeConsts* tcs, DevState* st, float* b0, float* b1, cudaStream_t s) {
  Tc3State* h = (Tc3State*)handle;
  if (!mp && !tcs) return 0;
  const Tc3Item it{handle, d, t, mp, tcs, st, b0, b1};
  Tc3Stage* g = &h->stage[h->parity];
  h->parity ^= 1;
  const int r = tc3_batch(&it, 1, cfg.precision, g, s);
  return r < 0 ? 0 : r;
}

}  // namespace pmf
