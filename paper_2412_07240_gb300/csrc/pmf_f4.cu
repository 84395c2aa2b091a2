// Float32 path for n_x = 4 grids (the coordinated-turn workload of Sec. VI and
// any other four-dimensional filter).  The weights live in float32; the
// per-axis transforms along axes 0 and 1 are tensor-core contractions (split
// FP16, FP32 accumulation), those along axes 2 and 3 float32 contractions of
// shared-memory slabs; the frame arithmetic, the regrid matrices, the
// measurement exponents and the moment sums keep float64-class accuracy.
//
// Per time update (Sec. V-B algorithm on the moving grid, eq. gridMov):
//   frame        regrid decision and sub-step coefficients (float64, shared
//                with the float64 path)
//   tables       W_a = H_a I_a per axis: the trigonometric regrid (eq.
//                interFreq) folded into the forward Hartley transform, float64,
//                rounded to float32
//   realign      multilinear re-alignment (or scaled copy) of the weights
//   slab23       W_3 and W_2 on (j0, j1) slabs in shared memory (one pass)
//   fwd 1, fwd 0 W_a along axis a (k_f4_axis_tc)
//   psi          diffusion multiplier and trace factor over 16-point sign-flip
//                orbits (the separable-to-4-D Hartley parity fix-up)
//   inv 0, inv 1 inverse Hartley transform along axes 0 and 1 (step 5)
//   slab23       inverse along axes 2 and 3, with the moment sums of the result
//   finalize     normaliser and moments (double-float sums, float64 frame; step 6)
// Per measurement update (eq. filt): exponent parts and their minimum, then
// the likelihood multiply with the moment sums, then the finalisation.
#include <cmath>
#include <vector>

#include "pmf_f4.cuh"
#include "pmf_device.cuh"
#include "pmf_grid.cuh"
#include "pmf_kernels.cuh"
#include "pmf_model.cuh"
#include "pmf_tcops.cuh"

namespace pmf {
namespace {

constexpr int kMaxN4 = 64;

__host__ __device__ inline int kpad(int N) { return (N + 7) & ~7; }


// ---- double-float helpers ---------------------------------------------------
__device__ __forceinline__ DF df_of(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}
// a b, with the product of the high parts exact (fma) and the cross terms rounded
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float h = p + e;
  return DF{h, e - (h - p)};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// ---- measurement update, pass 1 -------------------------------------------
// Terrain altitude (Sec. VI): base + sum_i amp_i sin(phi_i), phi_i = kx_i x_0 +
// ky_i x_2 + ph_i with x = c + M u, so phi_i = theta_i + sum_a g_ia u_a with
// theta_i = kx_i c_0 + ky_i c_2 + ph_i and g_ia = kx_i M_0a + ky_i M_2a, and
// e^{i phi_i} is a product of per-axis factors.  k_f4_meas_tab forms the
// factors (float64); k_f4_meas_e takes one block per (j0, j1) slab, multiplies
// the factors of axes 0-2 into a table over j2 (float64, then double-float),
// holds the axis-3 factors as double-float, and forms a point's altitude
// residual r = (z - base) - sum_i Im(t2_i t3_i) in double-float (~2^-44
// relative); the mixture exponents follow from r - mu_g in float32.  The
// exponent is kept as its smaller component m_lo and the gap |m_1 - m_2|
// (e = m_lo - log(1 + e^-gap)); other measurement kinds store e itself
// (float64, rounded) with an infinite gap.
//
// Phase tables (one block per wave i): tab[i][a][j] = e^{i g_ia u_j}, with
// amp_i e^{i theta_i} folded into axis 0.
__global__ void k_f4_meas_tab(Dims d, MeasParams mp, const DevState* st, double2* tab) {
  const int i = blockIdx.x;
  const double* c = st->f.c;
  const double* M = st->f.M;
  const double kx = mp.p[4 * i + 1], ky = mp.p[4 * i + 2];
  const double theta = kx * c[0] + ky * c[2] + mp.p[4 * i + 3];
  for (int t = threadIdx.x; t < 4 * kMaxN4; t += blockDim.x) {
    const int a = t / kMaxN4, j = t % kMaxN4;
    if (j >= d.N[a]) continue;
    const double g = kx * M[a] + ky * M[8 + a];
    const double ph = g * (j - 0.5 * (d.N[a] - 1)) + (a == 0 ? theta : 0.0);
    double sn, cs;
    sincos(ph, &sn, &cs);
    const double amp = a == 0 ? mp.p[4 * i] : 1.0;
    tab[(i * 4 + a) * kMaxN4 + j] = make_double2(amp * cs, amp * sn);
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_f4_meas_e(Dims d, MeasParams mp, DevState* st, const double2* tab, float* lo_out,
                            float* gap_out) {
  __shared__ float4 t2[4][kMaxN4], t3[4][kMaxN4];   // (re.hi, re.lo, im.hi, im.lo)
  __shared__ float wmin[32];
  const int N2 = d.N[2], N3 = d.N[3];
  const int j0 = blockIdx.x / d.N[1], j1 = blockIdx.x % d.N[1];
  const double u0 = j0 - 0.5 * (d.N[0] - 1), u1 = j1 - 0.5 * (d.N[1] - 1);
  const double* c = st->f.c;
  const double* M = st->f.M;
  const bool terrain = mp.kind == PMF_MEAS_TERRAIN_GM;
  if (terrain) {
    // t2: amp_i e^{i(theta + g_0 u_0 + g_1 u_1 + g_2 u_2)} over j2, t3: e^{i g_3 u_3}
    for (int t = threadIdx.x; t < 4 * (N2 + N3); t += blockDim.x) {
      const int i = t / (N2 + N3), r = t % (N2 + N3);
      const double2* ti = tab + i * 4 * kMaxN4;
      double2 v;
      if (r < N2) v = cmul(cmul(ti[j0], ti[kMaxN4 + j1]), ti[2 * kMaxN4 + r]);
      else v = ti[3 * kMaxN4 + r - N2];
      const DF re = df_of(v.x), im = df_of(v.y);
      (r < N2 ? t2[i][r] : t3[i][r - N2]) = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
  }
  const DF zb = df_of(mp.z[0] - mp.p[16]);
  const DF mu1 = df_of(mp.gm[4]), mu2 = df_of(mp.gm[5]);
  const float g0 = (float)mp.gm[0], g1 = (float)mp.gm[1], g2 = (float)mp.gm[2], g3 = (float)mp.gm[3];
  const int p0 = blockIdx.x * N2 * N3;
  float emin = INFINITY;
  for (int t = threadIdx.x; t < N2 * N3; t += blockDim.x) {
    const int j2 = t / N3, j3 = t % N3;
    float lo, gap;
    if (terrain) {
      DF h{0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 a = t2[i][j2], b = t3[i][j3];
        // amp_i sin(phi_i) = Im(a b) = a.re b.im + a.im b.re
        h = df_add(h, df_add(df_mul(DF{a.x, a.y}, DF{b.z, b.w}), df_mul(DF{a.z, a.w}, DF{b.x, b.y})));
      }
      const DF rr = df_add(zb, df_neg(h));
      const DF e1 = df_add(rr, df_neg(mu1)), e2 = df_add(rr, df_neg(mu2));
      const float d1 = e1.hi + e1.lo, d2 = e2.hi + e2.lo;
      const float m1 = fmaf(d1 * d1, g0, g2), m2 = fmaf(d2 * d2, g1, g3);
      lo = fminf(m1, m2);
      gap = fabsf(m1 - m2);
    } else {
      const double u[4] = {u0, u1, j2 - 0.5 * (N2 - 1), j3 - 0.5 * (N3 - 1)};
      double x[4];
      for (int a = 0; a < 4; ++a) {
        x[a] = c[a];
        for (int b = 0; b < 4; ++b) x[a] += M[a * 4 + b] * u[b];
      }
      lo = (float)meas_exponent_f64(mp, x);
      gap = INFINITY;
    }
    lo_out[p0 + t] = lo;
    gap_out[p0 + t] = gap;
    emin = fminf(emin, lo);
  }
  for (int o = 16; o; o >>= 1) emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = emin;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) emin = fminf(emin, wmin[w]);
    // every exponent is >= 0 (Gaussian forms; mixture constants shifted on the
    // host), so the bit patterns order like the values
    atomicMin(&st->emin_bits, (unsigned long long)__double_as_longlong((double)emin));
  }
}

// Double-float moment sums of one thread in the tot_S2 layout for n_x = 4:
// {S0, S1[4], S2[10]}, accumulated line by line.
struct Mom4 {
  DF s[kMomentSlots];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < kMomentSlots; ++i) s[i] = DF{0.0f, 0.0f};
  }
  // One line along axis 3 at (u0, u1, u2): its float32 sums s0 = sum v,
  // s1 = sum v u3, s2 = sum v u3^2 spread over the 15 slots.
  __device__ __forceinline__ void add_line(float s0, float s1, float s2, float u0, float u1, float u2) {
    const float u[3] = {u0, u1, u2};
    s[0] = df_add1(s[0], s0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float su = s0 * u[a];
      s[1 + a] = df_add1(s[1 + a], su);
#pragma unroll
      for (int b = a; b < 3; ++b) s[tot_S2(4, a, b)] = df_add1(s[tot_S2(4, a, b)], su * u[b]);
      s[tot_S2(4, a, 3)] = df_add1(s[tot_S2(4, a, 3)], s1 * u[a]);
    }
    s[4] = df_add1(s[4], s1);
    s[tot_S2(4, 3, 3)] = df_add1(s[tot_S2(4, 3, 3)], s2);
  }
};

// Block sum of the double-float moment sums into double-float partials
// (float2 {hi, lo} per slot), summed again in double-float by k_f4_finalize.
__device__ void mom4_block(Mom4& m, float2* out) {
  __shared__ DF red[32][kMomentSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < kMomentSlots; ++i)
    for (int o = 16; o; o >>= 1) {
      DF b{__shfl_xor_sync(0xffffffffu, m.s[i].hi, o), __shfl_xor_sync(0xffffffffu, m.s[i].lo, o)};
      m.s[i] = df_add(m.s[i], b);
    }
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < kMomentSlots; ++i) red[warp][i] = m.s[i];
  __syncthreads();
  if (warp == 0 && lane < kMomentSlots) {
    DF t = red[0][lane];
    for (int w = 1; w < nw; ++w) t = df_add(t, red[w][lane]);
    out[lane] = make_float2(t.hi, t.lo);
  }
}

// Normaliser and moments of the n_x = 4 weights from the blocks' double-float
// partials: the cross-block sums stay in double-float (float32 arithmetic;
// GB300 issues float64 at 1/64 of the float32 rate and this runs on one SM),
// the 15 totals become float64, and warp 0 finalises (finalize_warp, one
// matrix entry per lane) on a shared copy of the frame state.
__global__ void __launch_bounds__(256) k_f4_finalize(DevState* st, const float2* partials, int nblocks, int flip,
                                                     int use_pending, const double* pend) {
  __shared__ DF red[8][kMomentSlots];
  __shared__ double tot[kMomentSlots];
  __shared__ FrameState fs;
  constexpr int kWords = sizeof(FrameState) / 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DF acc[kMomentSlots];
#pragma unroll
  for (int i = 0; i < kMomentSlots; ++i) acc[i] = DF{0.0f, 0.0f};
  for (int b = tid; b < nblocks; b += 256)
#pragma unroll
    for (int i = 0; i < kMomentSlots; ++i) {
      const float2 v = partials[b * kMomentSlots + i];
      acc[i] = df_add(acc[i], DF{v.x, v.y});
    }
#pragma unroll
  for (int i = 0; i < kMomentSlots; ++i)
    for (int o = 16; o; o >>= 1) {
      DF b{__shfl_xor_sync(0xffffffffu, acc[i].hi, o), __shfl_xor_sync(0xffffffffu, acc[i].lo, o)};
      acc[i] = df_add(acc[i], b);
    }
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < kMomentSlots; ++i) red[warp][i] = acc[i];
  for (int i = tid; i < kWords; i += 256) ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  __syncthreads();
  if (warp == 0 && lane < kMomentSlots) {
    DF t = red[0][lane];
    for (int w = 1; w < 8; ++w) t = df_add(t, red[w][lane]);
    tot[lane] = (double)t.hi + (double)t.lo;
  }
  __syncthreads();
  if (warp != 0) return;
  const bool ok = finalize_warp<4>(&fs, tot, use_pending, pend);
  if (ok && lane == 0) fs.cur ^= flip;
  __syncwarp();
  for (int i = lane; i < kWords; i += 32) ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
}

// Moment kernels: a block takes kLinesM lines along axis 3, four threads per
// line (points j3 = q, q + 4, ...); a thread sums its points in float32 and adds
// the 15 slot contributions of its part of the line in double-float.
constexpr int kLinesM = 64;
constexpr int kMomThreads = 4 * kLinesM;

__device__ __forceinline__ void line_u(const Dims& d, int ln, float* u) {
  const int j2 = ln % d.N[2], r = ln / d.N[2];
  u[0] = (r / d.N[1]) - 0.5f * (d.N[0] - 1);
  u[1] = (r % d.N[1]) - 0.5f * (d.N[1] - 1);
  u[2] = j2 - 0.5f * (d.N[2] - 1);
}

// ---- measurement update, pass 2: likelihood multiply and moment sums ----
__global__ void __launch_bounds__(kMomThreads) k_f4_meas_apply(Dims d, DevState* st, const float* lo,
                                                               const float* gap, float* b0, float* b1,
                                                               double* partials) {
  const int cur = st->f.cur;
  const float* in = cur ? b1 : b0;
  float* out = cur ? b0 : b1;
  const double emin = __longlong_as_double((long long)st->emin_bits);
  const float ps = (float)st->f.pscale;
  const int N3 = d.N[3], lines = (int)d.P / N3;
  const float h3 = 0.5f * (N3 - 1);
  const int ln = blockIdx.x * kLinesM + threadIdx.x / 4, q = threadIdx.x % 4;
  Mom4 m;
  m.zero();
  if (ln < lines) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    for (int j = q; j < N3; j += 4) {
      const int p = ln * N3 + j;
      const float f = expf((float)(emin - (double)lo[p])) * (1.0f + expf(-gap[p]));
      const float v = (in[p] * ps) * f;
      out[p] = v;
      const float u3 = j - h3, vu = v * u3;
      s0 += v;
      s1 += vu;
      s2 = fmaf(vu, u3, s2);
    }
    float u[3];
    line_u(d, ln, u);
    m.add_line(s0, s1, s2, u[0], u[1], u[2]);
  }
  mom4_block(m, (float2*)partials + blockIdx.x * kMomentSlots);
}

// ---- time update ------------------------------------------------------------
// W_a^T (row j, column k, k padded to a multiple of 8 with zeros) of the fused
// regrid + forward transform W_a = H_a I_a, formed in float64.  I_a is the
// periodic-sinc regrid matrix of eq. interFreq (identity when the frame was
// re-aligned): I[q, j] = sin(pi v) cos(pi v / N) / (N sin(pi v / N)), v = y_q -
// u_j, y_q = rs_a + rd_a u_q, zero rows where |y_q| > N / 2.  One block per
// (j, axis): the column I[., j] in shared memory, then one thread per k.
__global__ void k_f4_tables(Dims d, const DevState* st, const F4Tables t) {
  __shared__ double col[kMaxN4];
  const int a = blockIdx.y, N = d.N[a], j = blockIdx.x;
  if (j >= N) return;
  const double half = 0.5 * (N - 1);
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    double v;
    if (st->f.realign) {
      v = q == j ? 1.0 : 0.0;
    } else {
      const double y = st->f.rs[a] + st->f.rd[a] * (q - half);
      if (fabs(y) > 0.5 * N) {
        v = 0.0;
      } else {
        const double x = y - (j - half);
        v = x == 0.0 ? 1.0 : sinpi(x) * cospi(x / N) / (N * sinpi(x / N));
      }
    }
    col[q] = v;
  }
  __syncthreads();
  const int Kp = kpad(N);
  for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
    double sum = 0.0;
    if (k < N)
      for (int q = 0; q < N; ++q) sum = fma(t.hfwd[a][k * N + q], col[q], sum);
    t.wfwd[a][j * Kp + k] = (float)sum;
  }
}

// Multilinear re-alignment of the weights onto the new frame (u_old = B u_new
// + b, 16 corners; nodes outside the old box contribute 0), or the scaled copy
// when the frame was not re-aligned.  Reads buf[cur], writes buf[cur ^ 1].
// A block takes kLinesR lines along axis 3: the old-index position of each
// line's first node is formed once in float64 and held as double-float, a
// node adds B_a3 j3 in double-float (exact product of the high part), and the
// integer part and the fraction of the position come from that sum (~1e-12
// node); the corner weights and sums are float32.
constexpr int kLinesRMax = 128;   // lines per block iteration: 512 / N3 (two passes of 256 threads)

__global__ void __launch_bounds__(256) k_f4_realign(Dims d, const DevState* st, float* b0, float* b1,
                                                    int shear) {
  __shared__ DF zl[kLinesRMax][4];
  const int cur = st->f.cur;
  const float* in = cur ? b1 : b0;
  float* out = cur ? b0 : b1;
  const float ps = (float)st->f.pscale;
  const int P = (int)d.P, N3 = d.N[3];
  if (st->f.realign && shear) return;   // the band-limited passes fill the re-aligned frame
  if (!st->f.realign) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) out[p] = ps * in[p];
    return;
  }
  const int lines = P / N3, kLinesR = min(kLinesRMax, 512 / N3);
  const int N0 = d.N[0], N1 = d.N[1], N2 = d.N[2];
  DF B3[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) B3[a] = df_of(st->f.B[a * 4 + 3]);
  for (int l0 = blockIdx.x * kLinesR; l0 < lines; l0 += gridDim.x * kLinesR) {
    for (int it = threadIdx.x; it < kLinesR * 4; it += blockDim.x) {
      const int li = it >> 2, a = it & 3, ln = l0 + li;
      if (ln < lines) {
        const int j2 = ln % N2, j1 = (ln / N2) % N1, j0 = ln / (N2 * N1);
        double z = st->f.b[a] + 0.5 * ((a == 0 ? N0 : a == 1 ? N1 : a == 2 ? N2 : N3) - 1);
        z = fma(st->f.B[a * 4 + 0], j0 - 0.5 * (N0 - 1), z);
        z = fma(st->f.B[a * 4 + 1], j1 - 0.5 * (N1 - 1), z);
        z = fma(st->f.B[a * 4 + 2], j2 - 0.5 * (N2 - 1), z);
        z = fma(st->f.B[a * 4 + 3], -0.5 * (N3 - 1), z);
        zl[li][a] = df_of(z);
      }
    }
    __syncthreads();
    const int cnt = min(kLinesR, lines - l0) * N3;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int li = t / N3, j3 = t - li * N3;
      int f[4];
      float w[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const DF b3 = B3[a];
        const float jf = (float)j3;
        const float p = b3.hi * jf;
        const DF z = df_add(zl[li][a], DF{p, fmaf(b3.lo, jf, fmaf(b3.hi, jf, -p))});
        float fl = floorf(z.hi);
        float wa = (z.hi - fl) + z.lo;
        if (wa < 0.0f) {
          wa += 1.0f;
          fl -= 1.0f;
        } else if (wa >= 1.0f) {
          wa -= 1.0f;
          fl += 1.0f;
        }
        f[a] = (int)fmaxf(fminf(fl, 1e6f), -1e6f);
        w[a] = wa;
      }
      float sum = 0.0f;
#pragma unroll
      for (int corner = 0; corner < 16; ++corner) {
        float wt = 1.0f;
        int off = 0;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int bit = (corner >> a) & 1;
          const int i = f[a] + bit;
          wt *= bit ? w[a] : 1.0f - w[a];
          ok = ok && i >= 0 && i < d.N[a];
          off = off * d.N[a] + (ok ? i : 0);
        }
        if (ok) sum = fmaf(wt, in[off], sum);
      }
      out[(l0 + li) * N3 + j3] = ps * sum;
    }
    __syncthreads();
  }
}

// Band-limited re-alignment (shear mode): the four line-wise passes of
// shear4_setup (pmf_device.cuh; pass coefficients in float64, written by
// k_f4_shear_setup), each the trigonometric interpolant (eq. interFreq) of
// every line along the pass's axis at that line's positions: one CTA per line,
// the line's DFT coefficients in float32 from a twiddle table, the positions
// in float64, each power e^{2 pi i k x / N} from the table (k m mod N) and the
// power of a small-angle factor.  Buffers:
// pass 0 buf[cur] -> buf[cur ^ 1], pass 1 back to buf[cur], pass 2 buf[cur] ->
// scratch (the measurement exponents, free during a time update), pass 3
// scratch -> buf[cur ^ 1] with pscale.
__global__ void k_f4_shear_setup(DevState* st, double* pc) {
  if (!st->f.realign) return;
  if (!shear4_setup(st->f, pc)) st->f.status = PMF_ERR_DEGENERATE;
}

constexpr int kShearT4 = 64;

__global__ void __launch_bounds__(kShearT4) k_f4_shear(Dims d, const DevState* st, const double* pc, int pass,
                                                       float* b0, float* b1, float* scratch) {
  __shared__ float fl[kMaxN4], cs[kMaxN4], sn[kMaxN4], Xr[kMaxN4 / 2 + 1], Xi[kMaxN4 / 2 + 1];
  const FrameState& f = st->f;
  if (!f.realign || pc[40] == 0.0) return;
  float* bc = f.cur ? b1 : b0;
  float* bn = f.cur ? b0 : b1;
  const float* in = pass == 0 ? bc : pass == 1 ? bn : pass == 2 ? bc : scratch;
  float* out = pass == 0 ? bn : pass == 1 ? bc : pass == 2 ? scratch : bn;
  const double* q = pc + 10 * pass;
  const int a = (int)q[0];
  int o[3], no = 0;
  for (int m = 0; m < 4; ++m)
    if (m != a) o[no++] = m;
  const int N = d.N[a], H = N / 2;
  const int lines = (int)(d.P / N);
  if ((int)blockIdx.x >= lines) return;
  int stride[4];
  stride[3] = 1;
  for (int m = 2; m >= 0; --m) stride[m] = stride[m + 1] * d.N[m + 1];
  int rest = blockIdx.x, base = 0;
  double offset = q[5];
  for (int k = 2; k >= 0; --k) {
    const int m = o[k], i = rest % d.N[m];
    rest /= d.N[m];
    base += i * stride[m];
    offset += q[1 + m] * (i - 0.5 * (d.N[m] - 1));
  }
  const int sa = stride[a];
  for (int t = threadIdx.x; t < N; t += kShearT4) {
    fl[t] = in[base + t * sa];
    sincospif(2.0f * (float)t / (float)N, &sn[t], &cs[t]);
  }
  __syncthreads();
  for (int sidx = threadIdx.x; sidx <= H; sidx += kShearT4) {
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
  const float ps = pass == 3 ? (float)f.pscale : 1.0f;
  for (int t = threadIdx.x; t < N; t += kShearT4) {
    const double pos = offset + q[1 + a] * (t - 0.5 * (N - 1));
    float v = 0.0f;
    if (fabs(pos) <= 0.5 * N) {
      // x = m + fr (m integer, |fr| <= 1/2): e^{2 pi i k x / N} is the table
      // entry of k m mod N times e^{2 pi i k fr / N}; the small-angle factor's
      // powers by recurrence from one sincospi (no rounded large argument)
      const double x = pos + 0.5 * (N - 1);
      const double mf = rint(x);
      const float fr = (float)(x - mf);
      int m = (int)mf % N;
      if (m < 0) m += N;
      float s1, c1;
      sincospif(2.0f * fr / (float)N, &s1, &c1);
      float wr = 1.0f, wi = 0.0f;   // e^{2 pi i k fr / N}
      int idx = 0;
      v = Xr[0];
      for (int k = 1; k < H; ++k) {
        const float nr = wr * c1 - wi * s1;
        wi = wr * s1 + wi * c1;
        wr = nr;
        idx += m;
        if (idx >= N) idx -= N;
        const float zr = cs[idx] * wr - sn[idx] * wi, zi = sn[idx] * wr + cs[idx] * wi;
        v += 2.0f * (Xr[k] * zr - Xi[k] * zi);
      }
      const float cn = cospif(fr);
      v += Xr[H] * ((((int)mf) & 1) ? -cn : cn);   // cos(pi x)
    }
    out[base + t * sa] = ps * v;
  }
}

// Y = W x_axis X on the float32 grid viewed as [outer][N][inner] (C order),
// on the tensor cores (tcgen05, split FP16, three products per K step): a CTA of 128 threads takes 128 consecutive lines, one
// per thread and TMEM lane.  Each thread loads its line (the loads of a warp
// are runs of consecutive floats for axes 0 and 1), and the tile becomes the A
// operand [128 lines x K] in hi + lo 16-bit planes under a power-of-two tile
// scale; W^T becomes the B operand [Nout x K] likewise (K and Nout padded to
// a multiple of 16 with zeros).  The accumulator goes from TMEM straight to
// the output lines.  The layout is the size-64 operand layout of the fused
// kernels (N <= 64).  Every wait is bounded; a lost completion records
// PMF_ERR_TIMEOUT in the filter's status and skips the stores.
constexpr int kTcLines = 128;
constexpr int kTcSmem = 2 * Lay<PMF_PREC_FP16X3, 64>::plane + 2 * Lay<PMF_PREC_FP16X3, 64>::wplane;

__global__ void __launch_bounds__(kTcLines) k_f4_axis_tc(Dims d, int axis, const float* __restrict__ WT,
                                                         DevState* st, int stage, float* b0, float* b1) {
  constexpr int P = PMF_PREC_FP16X3, C = 64;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float red[2][kTcLines / 32];
  uint8_t* A = smem;
  uint8_t* W = smem + 2 * Lay<P, C>::plane;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = d.N[axis], Kw = kpad(N), K = (N + 15) & ~15;
  int inner = 1;
#pragma unroll
  for (int m = 1; m < 4; ++m)
    if (m > axis) inner *= d.N[m];
  const int lines = (int)d.P / N;
  const int ln = blockIdx.x * kTcLines + tid;
  const bool mine = ln < lines;
  int cbase = 0;
  if (mine) {
    const int o = ln / inner;
    cbase = o * N * inner + (ln - o * inner);
  }
  const int par = (st->f.cur + stage) & 1;
  const float* X = par ? b1 : b0;
  float* Y = par ? b0 : b1;
  const uint32_t mb = su32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // this thread's line, and the largest |x| of the tile and |W^T| of the matrix
  float x[64];
  float mx = 0.0f, mw = 0.0f;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    x[j] = (mine && j < N) ? X[cbase + j * inner] : 0.0f;
    mx = fmaxf(mx, fabsf(x[j]));
  }
  for (int i = tid; i < N * Kw; i += kTcLines) mw = fmaxf(mw, fabsf(WT[i]));
  for (int o = 16; o; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
  }
  if ((tid & 31) == 0) {
    red[0][warp] = mx;
    red[1][warp] = mw;
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  mx = fmaxf(fmaxf(red[0][0], red[0][1]), fmaxf(red[0][2], red[0][3]));
  mw = fmaxf(fmaxf(red[1][0], red[1][1]), fmaxf(red[1][2], red[1][3]));
  const float sa = op_scale<P>(mx), sw = op_scale<P>(mw);
  // A: row = this line, K columns; B: row k (output), column j: W^T[j][k]
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (4 * q < K) store4<P, C>(A, tid, 4 * q, make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]), sa);
  for (int i = tid; i < K * (K / 4); i += kTcLines) {
    const int k = i / (K / 4), j = (i - k * (K / 4)) * 4;
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = (k < N && j + t < N) ? WT[(j + t) * Kw + k] : 0.0f;
    store4<P, C, true>(W, k, j, make_float4(v[0], v[1], v[2], v[3]), sw);
  }
  fence_async_smem();
  __syncthreads();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    tc_after_sync();
    issue_stage<P, C>(tmem, su32(A), 0, su32(W), K, K, mb);
  }
  const bool ok = mbar_wait(mb, 0);
  tc_after_sync();
  if (__syncthreads_or(!ok)) {
    if (tid == 0) st->f.status = PMF_ERR_TIMEOUT;
  } else {
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    const float inv = 1.0f / (sa * sw);
    float4 v[8];
    tmem_ld_cols(lane, K < 32 ? K : 32, v);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float y[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (mine && 4 * q + t < N) Y[cbase + (4 * q + t) * inner] = y[t] * inv;
    }
    if (K > 32) {
      tmem_ld_cols(lane + 32, K - 32, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float y[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (mine && 32 + 4 * q + t < N) Y[cbase + (32 + 4 * q + t) * inner] = y[t] * inv;
      }
    }
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

void launch_axis(const Dims& d, int a, const float* WT, DevState* st, int stage, float* b0, float* b1,
                 cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_f4_axis_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    attr = true;
  }
  const int lines = (int)(d.P / d.N[a]);
  k_f4_axis_tc<<<(lines + kTcLines - 1) / kTcLines, kTcLines, kTcSmem, s>>>(d, a, WT, st, stage, b0, b1);
}

// Both inner axes at once: a block takes kSlabs slabs (j0, j1) of N2 x N3
// contiguous points, applies W3 along axis 3 (rows of a slab) and then W2
// along axis 2 (its columns) in shared memory, and writes the slabs back: one
// pass over the grid for two contractions.  With kMom the moment sums of the
// result (the weights after the inverse transform) are formed from the slabs
// in shared memory (line sums along axis 3, double-float slot totals).
// Reads bufs[(cur+stage)&1], writes the other one.
constexpr int kSlabs = 4;
constexpr int kSlabThreads = 256;

__device__ __forceinline__ void contract_lines(const float* X, float* Y, const float* Ws, int lines, int per,
                                               int sstride, int N, int Kp, int xl, int xj, int yl, int yk) {
  // Y[line][k] = sum_j W[k][j] X[line][j] over lines = (slab, c), line = slab *
  // per + c: element (line, j) of X at slab * sstride + c * xl + j * xj, of Y
  // at slab * sstride + c * yl + k * yk; W^T rows j in Ws (k contiguous, Kp)
  const int groups = (N + 7) / 8;
  for (int it = threadIdx.x; it < lines * groups; it += blockDim.x) {
    const int line = it % lines, k0 = (it / lines) * 8;
    const int sb = line / per, c = line - sb * per;
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0f;
    const float* xr = X + sb * sstride + c * xl;
#pragma unroll 2
    for (int j = 0; j < N; ++j) {
      const float x = xr[j * xj];
      const float4 w0 = *(const float4*)(Ws + j * Kp + k0);
      const float4 w1 = *(const float4*)(Ws + j * Kp + k0 + 4);
      acc[0] = fmaf(w0.x, x, acc[0]);
      acc[1] = fmaf(w0.y, x, acc[1]);
      acc[2] = fmaf(w0.z, x, acc[2]);
      acc[3] = fmaf(w0.w, x, acc[3]);
      acc[4] = fmaf(w1.x, x, acc[4]);
      acc[5] = fmaf(w1.y, x, acc[5]);
      acc[6] = fmaf(w1.z, x, acc[6]);
      acc[7] = fmaf(w1.w, x, acc[7]);
    }
    float* yr = Y + sb * sstride + c * yl;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (k0 + r < N) yr[(k0 + r) * yk] = acc[r];
  }
}

size_t slab_smem(int N2, int N3) {
  return sizeof(float) * (2 * (size_t)kSlabs * N2 * (N3 + 1) + (size_t)N3 * kpad(N3) + (size_t)N2 * kpad(N2));
}

template <bool kMom>
__global__ void __launch_bounds__(kSlabThreads) k_f4_slab23(Dims d, const float* W3T, const float* W2T,
                                                            const DevState* st, int stage, float* b0, float* b1,
                                                            double* partials) {
  extern __shared__ __align__(16) float sm[];
  const int N1 = d.N[1], N2 = d.N[2], N3 = d.N[3];
  const int str = N3 + 1, slab = N2 * str, K3 = kpad(N3), K2 = kpad(N2);
  float* Xs = sm;                               // [kSlabs][N2][N3 + 1]
  float* Ys = Xs + kSlabs * slab;               // [kSlabs][N2][N3 + 1]
  float* W3 = Ys + kSlabs * slab;               // [N3][K3]
  float* W2 = W3 + N3 * K3;                     // [N2][K2]
  const int par = (st->f.cur + stage) & 1;
  const float* X = par ? b1 : b0;
  float* Y = par ? b0 : b1;
  const int nslab = d.N[0] * N1, s0 = blockIdx.x * kSlabs, ns = min(kSlabs, nslab - s0);
  const int tid = threadIdx.x, pts = N2 * N3;
  for (int i = tid; i < N3 * K3; i += kSlabThreads) W3[i] = W3T[i];
  for (int i = tid; i < N2 * K2; i += kSlabThreads) W2[i] = W2T[i];
  for (int sl = 0; sl < ns; ++sl) {
    const float* src = X + (size_t)(s0 + sl) * pts;
    for (int t = tid; t < pts; t += kSlabThreads) {
      const int r = t / N3, c = t - r * N3;
      Xs[sl * slab + r * str + c] = src[t];
    }
  }
  __syncthreads();
  // axis 3: rows (sl, j2) of every slab, X -> Y
  contract_lines(Xs, Ys, W3, ns * N2, N2, slab, N3, K3, str, 1, str, 1);
  __syncthreads();
  // axis 2: columns (sl, k3) of every slab, Y -> X
  contract_lines(Ys, Xs, W2, ns * N3, N3, slab, N2, K2, 1, str, 1, str);
  __syncthreads();
  for (int sl = 0; sl < ns; ++sl) {
    float* dst = Y + (size_t)(s0 + sl) * pts;
    for (int t = tid; t < pts; t += kSlabThreads) {
      const int r = t / N3, c = t - r * N3;
      dst[t] = Xs[sl * slab + r * str + c];
    }
  }
  if constexpr (kMom) {
    Mom4 m;
    m.zero();
    const float h3 = 0.5f * (N3 - 1);
    for (int ln = tid; ln < ns * N2; ln += kSlabThreads) {
      const int sl = ln / N2, r = ln - sl * N2, sg = s0 + sl;
      const float* row = Xs + sl * slab + r * str;
      float a = 0.0f, b = 0.0f, c = 0.0f;
      for (int j = 0; j < N3; ++j) {
        const float v = row[j], u3 = j - h3, vu = v * u3;
        a += v;
        b += vu;
        c = fmaf(vu, u3, c);
      }
      m.add_line(a, b, c, (sg / N1) - 0.5f * (d.N[0] - 1), (sg % N1) - 0.5f * (N1 - 1), r - 0.5f * (N2 - 1));
    }
    mom4_block(m, (float2*)partials + blockIdx.x * kMomentSlots);
  }
}

// Diffusion multiplier and trace factor in the Hartley domain (algorithm
// steps 2-4) for n_x = 4: one thread per orbit {sigma . k} of the 16 sign
// flips.  The separable coefficients S split into parity components T_B (odd
// in the axes of B), the multiplier into its jointly-even components Psi_E,
// and T'_C = sum_{|E| even} (-1)^{|E|/2 + |E & C|} Psi_E T_{E ^ C}.
// Over an orbit |kappa_a| is fixed and the first-derivative coefficients flip
// sign with sigma_a, so a sub-step exponent is E_q + sum_{a<b} sigma_a sigma_b
// X_q,ab: eight distinct values (sigma and -sigma agree), formed from one
// read of the sub-step coefficients.  float32 arithmetic; the coefficients are
// rounded from float64 once per block.
__global__ void __launch_bounds__(128) k_f4_psi(Dims d, const DevState* st, int stage, float* b0,
                                                float* b1) {
  __shared__ float spa[MAXL][4], spb[MAXL][6];
  const int par = (st->f.cur + stage) & 1;
  float* X = par ? b1 : b0;
  const int l = st->f.l, exact = st->f.exact;
  const float g = (float)st->f.g;
  for (int q = threadIdx.x; q < l; q += blockDim.x) {
    for (int a = 0; a < 4; ++a) spa[q][a] = (float)st->pa[q][a];
    for (int a = 0; a < 6; ++a) spb[q][a] = (float)st->pb[q][a];
  }
  __syncthreads();
  int H[4], N[4];
  int reps = 1;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    N[a] = d.N[a];
    H[a] = N[a] / 2 + 1;
    reps *= H[a];
  }
  const float two_pi = 6.28318530717958647692f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < reps; r += gridDim.x * blockDim.x) {
    int k[4];
    int t = r;
#pragma unroll
    for (int a = 3; a >= 0; --a) {
      k[a] = t % H[a];
      t /= H[a];
    }
    float kap2[4], kt[4];
    int kp[4], km[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      kp[a] = k[a];
      km[a] = (N[a] - k[a]) % N[a];
      const int w = k[a] < N[a] / 2 ? k[a] : k[a] - N[a];     // fftshift(-N/2 : N/2-1)
      const float kap = two_pi * (float)w / (float)N[a];
      kap2[a] = kap * kap;
      kt[a] = (2 * k[a] == N[a]) ? 0.0f : kap;                // first derivative: Nyquist omitted
    }
    // eight sign patterns sigma (sigma_3 = +1); pattern s and s ^ 15 share Psi
    float den[8], ex[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      den[s] = 1.0f;
      ex[s] = 0.0f;
    }
    const float c01 = kt[0] * kt[1], c02 = kt[0] * kt[2], c12 = kt[1] * kt[2];
    const float c03 = kt[0] * kt[3], c13 = kt[1] * kt[3], c23 = kt[2] * kt[3];
    for (int q = 0; q < l; ++q) {
      const float E = spa[q][0] * kap2[0] + spa[q][1] * kap2[1] + spa[q][2] * kap2[2] + spa[q][3] * kap2[3];
      const float x01 = spb[q][0] * c01, x02 = spb[q][1] * c02, x12 = spb[q][2] * c12;
      const float x03 = spb[q][3] * c03, x13 = spb[q][4] * c13, x23 = spb[q][5] * c23;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float s0 = (s & 1) ? -1.0f : 1.0f, s1 = (s & 2) ? -1.0f : 1.0f, s2 = (s & 4) ? -1.0f : 1.0f;
        const float e = E + s0 * s1 * x01 + s0 * s2 * x02 + s1 * s2 * x12 + s0 * x03 + s1 * x13 + s2 * x23;
        den[s] *= 1.0f + e;
        ex[s] += e;
      }
    }
    float Psi[16], S[16];
    int idx[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int h = s < 8 ? s : s ^ 15;
      Psi[s] = exact ? expf(-ex[h]) : 1.0f / den[h];
      int off = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) off = off * N[a] + (((s >> a) & 1) ? km[a] : kp[a]);
      idx[s] = off;
      S[s] = X[off];
    }
    float T[16], Pe[16];
#pragma unroll
    for (int B = 0; B < 16; ++B) {
      float tb = 0.0f, pe = 0.0f;
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const bool odd = popc((unsigned)(B & s)) & 1;
        tb += odd ? -S[s] : S[s];
        pe += odd ? -Psi[s] : Psi[s];
      }
      T[B] = tb * (1.0f / 16.0f);
      Pe[B] = pe * (1.0f / 16.0f);
    }
    float Tp[16];
#pragma unroll
    for (int C = 0; C < 16; ++C) {
      float acc = 0.0f;
#pragma unroll
      for (int E = 0; E < 16; ++E) {
        const int pe = popc((unsigned)E);
        if (pe & 1) continue;
        const int sgn = ((pe / 2) + popc((unsigned)(E & C))) & 1;
        acc += sgn ? -Pe[E] * T[E ^ C] : Pe[E] * T[E ^ C];
      }
      Tp[C] = acc * g;
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      float v = 0.0f;
#pragma unroll
      for (int C = 0; C < 16; ++C) v += (popc((unsigned)(C & s)) & 1) ? -Tp[C] : Tp[C];
      X[idx[s]] = v;
    }
  }
}

inline int grid_cap(long long work, int threads, int cap) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b > cap ? cap : b);
}

}  // namespace

int f4_supported(const pmf_config* cfg, std::string* why) {
  if (cfg->nx != 4) {
    *why = "the float32 4-D kernels handle n_x = 4";
    return PMF_ERR_UNSUPPORTED;
  }
  long long P = 1;
  for (int a = 0; a < 4; ++a) {
    if (cfg->N[a] > kMaxN4) {
      *why = "the float32 4-D kernels need N <= 64 per axis";
      return PMF_ERR_UNSUPPORTED;
    }
    P *= cfg->N[a];
  }
  if (P / ((long long)cfg->N[0] * cfg->N[1]) > (1 << 20)) {
    *why = "grid too large for the 4-D kernels";
    return PMF_ERR_UNSUPPORTED;
  }
  return PMF_OK;
}

int f4_alloc(const pmf_config* cfg, F4Tables* t) {
  *t = F4Tables{};
  long long P = 1;
  for (int a = 0; a < 4; ++a) P *= cfg->N[a];
  bool ok = cudaMalloc(&t->mtab, sizeof(double2) * 16 * kMaxN4) == cudaSuccess &&
            cudaMalloc(&t->shear, sizeof(double) * 48) == cudaSuccess &&
            cudaMalloc(&t->lo, sizeof(float) * P) == cudaSuccess &&
            cudaMalloc(&t->gap, sizeof(float) * P) == cudaSuccess;
  for (int a = 0; ok && a < 4; ++a) {
    const int N = cfg->N[a], Kp = kpad(N);
    ok = cudaMalloc(&t->hfwd[a], sizeof(double) * N * N) == cudaSuccess &&
         cudaMalloc(&t->wfwd[a], sizeof(float) * N * Kp) == cudaSuccess &&
         cudaMalloc(&t->winv[a], sizeof(float) * N * Kp) == cudaSuccess;
    if (!ok) break;
    std::vector<double> H((size_t)N * N);
    hartley_host(N, 1.0 / N, H.data());
    ok = cudaMemcpy(t->hfwd[a], H.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice) == cudaSuccess;
    // inverse transform (the Hartley matrix is symmetric): W^T = H, k padded
    hartley_host(N, 1.0, H.data());
    std::vector<float> WT((size_t)N * Kp, 0.0f);
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) WT[(size_t)j * Kp + k] = (float)H[(size_t)k * N + j];
    ok = ok && cudaMemcpy(t->winv[a], WT.data(), sizeof(float) * N * Kp, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (ok) {
    // the axis tiles need at most 64 x (65 + 64) floats = 33 KB (no opt-in)
    const int ssm = (int)slab_smem(kMaxN4, kMaxN4);
    ok = cudaFuncSetAttribute(k_f4_slab23<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_f4_slab23<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm) == cudaSuccess;
  }
  if (!ok) {
    f4_free(t);
    return PMF_ERR_OOM;
  }
  return PMF_OK;
}

void f4_free(F4Tables* t) {
  cudaFree(t->mtab);
  cudaFree(t->shear);
  cudaFree(t->lo);
  cudaFree(t->gap);
  for (int a = 0; a < 4; ++a) {
    cudaFree(t->hfwd[a]);
    cudaFree(t->wfwd[a]);
    cudaFree(t->winv[a]);
  }
  *t = F4Tables{};
}

int f4_meas(const Dims& d, const MeasParams& mp, DevState* st, const F4Tables& t, float* b0, float* b1,
            double* partials, cudaStream_t s) {
  cudaMemsetAsync(&st->emin_bits, 0xff, sizeof(unsigned long long), s);
  int n = 3;
  if (mp.kind == PMF_MEAS_TERRAIN_GM) {
    k_f4_meas_tab<<<4, 128, 0, s>>>(d, mp, st, t.mtab);
    ++n;
  }
  k_f4_meas_e<<<d.N[0] * d.N[1], 256, 0, s>>>(d, mp, st, t.mtab, t.lo, t.gap);
  const int nb = (int)((d.P / d.N[3] + kLinesM - 1) / kLinesM);
  k_f4_meas_apply<<<nb, kMomThreads, 0, s>>>(d, st, t.lo, t.gap, b0, b1, partials);
  k_f4_finalize<<<1, 256, 0, s>>>(st, (const float2*)partials, nb, 1, 0, nullptr);
  return n;
}

int f4_time(const Dims& d, const TimeConsts& tc, DevState* st, const F4Tables& t, float* b0, float* b1,
            double* partials, double* pend, cudaStream_t s) {
  launch_frame(tc, st, pend, s);
  int maxN = 0;
  for (int a = 0; a < 4; ++a) maxN = d.N[a] > maxN ? d.N[a] : maxN;
  k_f4_tables<<<dim3(maxN, 4), 64, 0, s>>>(d, st, t);
  const int shear = tc.realign_mode == PMF_REALIGN_SHEAR;
  k_f4_realign<<<grid_cap(d.P / d.N[3], 512 / d.N[3], 4096), 256, 0, s>>>(d, st, b0, b1, shear);
  if (shear) {
    int Nmin = d.N[0];
    for (int a = 1; a < 4; ++a) Nmin = d.N[a] < Nmin ? d.N[a] : Nmin;
    k_f4_shear_setup<<<1, 1, 0, s>>>(st, t.shear);
    for (int pass = 0; pass < 4; ++pass)
      k_f4_shear<<<(unsigned)(d.P / Nmin), kShearT4, 0, s>>>(d, st, t.shear, pass, b0, b1, t.lo);
  }
  int stage = 1;
  auto axis = [&](int a, const float* WT) { launch_axis(d, a, WT, st, stage++, b0, b1, s); };
  const int nslab = (d.N[0] * d.N[1] + kSlabs - 1) / kSlabs;
  const size_t ssm = slab_smem(d.N[2], d.N[3]);
  k_f4_slab23<false><<<nslab, kSlabThreads, ssm, s>>>(d, t.wfwd[3], t.wfwd[2], st, stage++, b0, b1, nullptr);
  axis(1, t.wfwd[1]);
  axis(0, t.wfwd[0]);
  long long reps = 1;
  for (int a = 0; a < 4; ++a) reps *= d.N[a] / 2 + 1;
  k_f4_psi<<<grid_cap(reps, 128, 4096), 128, 0, s>>>(d, st, stage, b0, b1);
  axis(0, t.winv[0]);
  axis(1, t.winv[1]);
  k_f4_slab23<true><<<nslab, kSlabThreads, ssm, s>>>(d, t.winv[3], t.winv[2], st, stage++, b0, b1, partials);
  k_f4_finalize<<<1, 256, 0, s>>>(st, (const float2*)partials, nslab, stage & 1, 1, pend);
  return 1 + 1 + 1 + 6 + 1 + 1 + (shear ? 5 : 0);
}

}  // namespace pmf
