// One-dimensional filters on the CUDA cores (n_x = 1, N <= 512): one CTA
// carries one filter through an epoch with its grid in shared memory.
//
//   measurement update (eq. filt)   likelihood relative to the frame centre,
//                                   exponent minimum, double-float moments
//   frame (float64, one warp)       regrid decision, sub-step coefficients
//   regrid                          y = I x, periodic-sinc entries generated on the fly
//   forward Hartley                 Y_k = sum_j y_j cas(2 pi k j / N)
//   multiplier                      Psi(k) g / N (Sec. V-B algorithm steps 2-4;
//                                   in 1-D Psi is even and there is no cross term)
//   inverse Hartley                 x'_j = sum_k Y'_k cas(2 pi k j / N)
//   normalisation and moments (step 6), weights written back.
//
// A single 1-D filter's transform is a matrix-vector product, not a GEMM tile:
// the products run in float32 on the CUDA cores with every operand in shared
// memory, and the small footprint lets several filters share an SM.  For N a
// power of two the two Hartley transforms can instead run as a radix-2
// Stockham FFT in shared memory (H_k = Re Z_k - Im Z_k); an autotuner times
// both forms once per N and caches the choice in autotune.json beside the
// library.
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pmf_model.cuh"

#include "pmf_device.cuh"
#include "pmf_tc.cuh"
#include "pmf_tcops.cuh"

namespace pmf {

namespace {

constexpr int kT1 = 256;
constexpr int kMaxN1 = 512;

// What one CTA works on.
struct View1 {
  DevState* st;
  float* buf0;
  float* buf1;
  const float* tab;         // cas(2 pi r / N), r < N, then (cos, sin)(pi m / N), m = -N..N
  int N, do_meas, do_time;
  const MeasParams* mp;
  const double* z;
  const TimeConsts* tc;
  int mode;                 // Hartley transforms: 0 matrix-vector, 1 Stockham FFT (N a power of two)
};

// One filter launched alone: everything by value.
struct Job1 {
  DevState* st;
  float* buf0;
  float* buf1;
  const float* tab;
  int N, do_meas, do_time;
  MeasParams mp;
  TimeConsts tc;
  int mode;
};

struct Shared1 {
  TimeConsts tc;
  MeasParams mp;
  FrameState fs;
  double tot[10];
  double pend[24];
  double Mpi[9];
  DF redm[kT1 / 32][3];
  float redf[kT1 / 32];
  float x[kMaxN1], y[kMaxN1];
  float fre[2][kMaxN1], fim[2][kMaxN1];   // FFT ping-pong buffers
  float cas[kMaxN1];
  float sct[2 * (2 * kMaxN1 + 1)];
  RegridRowsT<kMaxN1> rows;
  float pa[MAXL];
  float gsc, ps;
  float hM[PMF_MAX_NZ], r0[PMF_MAX_NZ], Rinv[PMF_MAX_NZ * PMF_MAX_NZ];
  int degenerate;
};

__device__ __forceinline__ float block_min1(Shared1& sh, float v) {
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh.redf[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = INFINITY;
#pragma unroll
  for (int w = 0; w < kT1 / 32; ++w) m = fminf(m, sh.redf[w]);
  return m;
}

// Block sums of {S0, S1, S2} (double-float) into tot[0], tot[1], tot[4]
// (the remaining slots zero); valid in warp 0 after the call.
__device__ __forceinline__ void block_moments1(Shared1& sh, DF s0, DF s1, DF s2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DF a[3] = {s0, s1, s2};
#pragma unroll
  for (int i = 0; i < 3; ++i)
    for (int o = 16; o; o >>= 1) {
      DF b{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
      a[i] = df_add(a[i], b);
    }
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 3; ++i) sh.redm[warp][i] = a[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a[i] = lane < kT1 / 32 ? sh.redm[lane][i] : DF{0.0f, 0.0f};
      for (int o = kT1 / 64; o; o >>= 1) {
        DF b{__shfl_xor_sync(0xffffffffu, a[i].hi, o), __shfl_xor_sync(0xffffffffu, a[i].lo, o)};
        a[i] = df_add(a[i], b);
      }
    }
    const DF mine = lane == 1 ? a[1] : (lane == 4 ? a[2] : a[0]);
    if (lane == 0 || lane == 1 || lane == 4) sh.tot[lane] = (double)mine.hi + (double)mine.lo;
    else if (lane < 10) sh.tot[lane] = 0.0;
    __syncwarp();
  }
}

// dst[o] = epi(o, sum_j entry(o, j) src[j]) for o < N: P = 2^lp consecutive
// lanes share an output (each sums every P-th term), so small N still uses
// the whole block.  Every thread runs the same number of rounds.
template <class Entry, class Epi>
__device__ __forceinline__ void matvec1(int N, int lp, const float* src, Entry entry, Epi epi) {
  const int P = 1 << lp, total = N << lp;
  for (int base = 0; base < total; base += kT1) {
    const int w = base + threadIdx.x;
    const int o = w >> lp, p = w & (P - 1);
    float s = 0.0f;
    if (w < total) s = entry(o, p, P, src);
    for (int d = P >> 1; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (w < total && p == 0) epi(o, s);
  }
}

// Hartley transform of src (N = 2^lg) by a radix-2 Stockham FFT of the real
// sequence: Z = sum_j y_j e^{-2 pi i j k / N}, stage Ns pairs j and j + N/2,
// twiddle e^{-i pi (j mod Ns) / Ns} from the (cos, sin)(pi m / N) table, and
// writes to (j - t) 2 + t and + Ns (t = j mod Ns); then epi(k, Re Z_k - Im Z_k).
template <class Epi>
__device__ __forceinline__ void fht1(Shared1& sh, const float* src, int N, Epi epi) {
  for (int j = threadIdx.x; j < N; j += kT1) {
    sh.fre[0][j] = src[j];
    sh.fim[0][j] = 0.0f;
  }
  __syncthreads();
  int b = 0;
  for (int Ns = 1; Ns < N; Ns <<= 1) {
    const float* ri = sh.fre[b];
    const float* ii = sh.fim[b];
    float* ro = sh.fre[b ^ 1];
    float* io = sh.fim[b ^ 1];
    const int half = N >> 1, step = N / (2 * Ns);
    for (int j = threadIdx.x; j < half; j += kT1) {
      const int t = j & (Ns - 1), m = 2 * t * step;
      const float c = sh.sct[2 * (m + N)], s = sh.sct[2 * (m + N) + 1];
      const float ar = ri[j], ai = ii[j], br = ri[j + half], bi = ii[j + half];
      const float tr = br * c + bi * s, ti = bi * c - br * s;
      const int o = (j - t) * 2 + t;
      ro[o] = ar + tr;
      io[o] = ai + ti;
      ro[o + Ns] = ar - tr;
      io[o + Ns] = ai - ti;
    }
    b ^= 1;
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N; k += kT1) epi(k, sh.fre[b][k] - sh.fim[b][k]);
}

__device__ void fused1d(const View1& v) {
  __shared__ Shared1 sh;
  if (!v.do_meas && !v.do_time) return;   // nothing requested for this filter
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = v.N;
  DevState* st = v.st;
  FrameState& fs = sh.fs;
  constexpr int kFsWords = sizeof(FrameState) / 8;
  for (int i = tid; i < kFsWords; i += kT1) ((unsigned long long*)&fs)[i] = ((const unsigned long long*)&st->f)[i];
  if (v.do_time) {
    const int words = tc_words(v.tc);   // up to the sub-step rows this update uses
    for (int i = tid; i < words; i += kT1)
      ((unsigned long long*)&sh.tc)[i] = ((const unsigned long long*)v.tc)[i];
    for (int i = tid; i < N; i += kT1) sh.cas[i] = v.tab[i];
    for (int i = tid; i < 2 * (2 * N + 1); i += kT1) sh.sct[i] = v.tab[N + i];
  }
  if (v.do_meas) {
    for (int i = tid; i < (int)(sizeof(MeasParams) / 8); i += kT1)
      ((unsigned long long*)&sh.mp)[i] = ((const unsigned long long*)v.mp)[i];
  }
  if (tid == 0) sh.degenerate = 0;
  __syncthreads();
  if (v.do_meas && tid < PMF_MAX_NZ) sh.mp.z[tid] = v.z[tid];
  const int cur = fs.cur;
  const float* in = cur ? v.buf1 : v.buf0;
  float* out = cur ? v.buf0 : v.buf1;
  {
    const float ps = (float)fs.pscale;
    for (int j = tid; j < N; j += kT1) sh.x[j] = in[j] * ps;
  }
  const float uc = 0.5f * (N - 1);
  int l = 0, exact = 0;

  // ---- measurement update (eq. filt), linear h: r = (z - H c) - (H M) u ----
  if (v.do_meas) {
    __syncthreads();
    if (tid == 0) {
      const MeasParams& mp = sh.mp;
      for (int i = 0; i < mp.nz; ++i) {
        sh.r0[i] = (float)(mp.z[i] - mp.H[i] * fs.c[0]);
        sh.hM[i] = (float)(mp.H[i] * fs.M[0]);
      }
      for (int i = 0; i < mp.nz * mp.nz; ++i) sh.Rinv[i] = (float)mp.Rinv[i];
    }
    __syncthreads();
    const int nz = sh.mp.nz;
    float emin = INFINITY;
    for (int j = tid; j < N; j += kT1) {
      const float u = j - uc;
      float r[PMF_MAX_NZ];
      for (int i = 0; i < nz; ++i) r[i] = sh.r0[i] - sh.hM[i] * u;
      float e = 0.0f;
      for (int i = 0; i < nz; ++i)
        for (int k = 0; k < nz; ++k) e += r[i] * sh.Rinv[i * nz + k] * r[k];
      e *= 0.5f;
      sh.y[j] = e;
      emin = fminf(emin, e);
    }
    emin = block_min1(sh, emin);
    DF s0{0.0f, 0.0f}, s1{0.0f, 0.0f}, s2{0.0f, 0.0f};
    for (int j = tid; j < N; j += kT1) {
      const float u = j - uc;
      const float w = sh.x[j] * __expf(emin - sh.y[j]);
      sh.x[j] = w;
      s0 = df_add1(s0, w);
      s1 = df_add1(s1, w * u);
      s2 = df_add1(s2, w * u * u);
    }
    block_moments1(sh, s0, s1, s2);
  }
  if (warp == 0) {
    bool ok = true;
    if (v.do_meas) {
      ok = finalize_warp<1>(&fs, sh.tot, 0, nullptr);
      if (tid == 0) {
        if (!ok) {
          sh.degenerate = 1;
        } else {
          sh.ps = (float)fs.pscale;   // the posterior weights times ps are normalised
          fs.pscale = 1.0;
          fs.S0 = 1.0 / fs.V;
        }
      }
      __syncwarp();
    }
    if (ok && v.do_time) {
      frame_warp<1>(sh.tc, &fs, sh.pend, sh.Mpi);
      if (tid == 0) sh.gsc = (float)(fs.g / (double)N);
    }
  }
  __syncthreads();
  if (sh.degenerate) goto done;
  if (!v.do_time) {
    for (int j = tid; j < N; j += kT1) out[j] = sh.x[j] * sh.ps;
    if (tid == 0) fs.cur = cur ^ 1;
    goto done;
  }
  {
    // ---- sub-step coefficients and regrid rows (1-D never re-aligns) ----
    l = fs.l;
    exact = fs.exact;
    for (int q = tid; q < l; q += kT1) {
      double pa[4], pb[6];
      frame_substep<1>(sh.tc, sh.Mpi, q, pa, pb);
      sh.pa[q] = (float)pa[0];
    }
    regrid_rows(sh.rows, fs.rs[0], fs.rd[0], N, tid, kT1);
    __syncthreads();
    int lp = 0;
    while ((2 << lp) * N <= kT1 && lp < 5) ++lp;
    // y = I x
    matvec1(
        N, lp, sh.x,
        [&](int o, int p, int P, const float* src) {
          float s = 0.0f;
          for (int j = p; j < N; j += P) s = fmaf(interp_entry(sh.rows, o, j, N, sh.sct), src[j], s);
          return s;
        },
        [&](int o, float s) { sh.y[o] = s; });
    __syncthreads();
    // forward Hartley and the multiplier
    const float w2 = 6.28318530717958647692f / (float)N;
    auto hartley = [&](int o, int p, int P, const float* src) {
      int idx = (o * p) % N;
      const int step = (o * P) % N;
      float s = 0.0f;
      for (int j = p; j < N; j += P) {
        s = fmaf(sh.cas[idx], src[j], s);
        idx += step;
        if (idx >= N) idx -= N;
      }
      return s;
    };
    auto psi = [&](int k, float s) {
      const float kf = w2 * (float)(k < N / 2 ? k : k - N);
      const float q = kf * kf;
      float den = 1.0f, ex = 0.0f;
      for (int qq = 0; qq < l; ++qq) {
        const float e = sh.pa[qq] * q;
        den *= 1.0f + e;
        ex += e;
      }
      sh.x[k] = s * (exact ? expf(-ex) : __frcp_rn(den)) * sh.gsc;
    };
    if (v.mode == 1)
      fht1(sh, sh.y, N, psi);
    else
      matvec1(N, lp, sh.y, hartley, psi);
    __syncthreads();
    // inverse Hartley (its own inverse; 1/N is in gsc)
    auto keep = [&](int j, float s) { sh.y[j] = s; };
    if (v.mode == 1)
      fht1(sh, sh.x, N, keep);
    else
      matvec1(N, lp, sh.x, hartley, keep);
    __syncthreads();
    // ---- write-back, moments and normalisation on the advanced frame ----
    DF s0{0.0f, 0.0f}, s1{0.0f, 0.0f}, s2{0.0f, 0.0f};
    for (int j = tid; j < N; j += kT1) {
      const float w = sh.y[j], u = j - uc;
      out[j] = w;
      s0 = df_add1(s0, w);
      s1 = df_add1(s1, w * u);
      s2 = df_add1(s2, w * u * u);
    }
    block_moments1(sh, s0, s1, s2);
    if (warp == 0 && finalize_warp<1>(&fs, sh.tot, 1, sh.pend) && tid == 0) fs.cur = cur ^ 1;
  }
done:
  __syncthreads();
  for (int i = tid; i < kFsWords; i += kT1) ((unsigned long long*)&st->f)[i] = ((const unsigned long long*)&fs)[i];
}

__global__ void __launch_bounds__(kT1) k_fused1d(const __grid_constant__ Job1 job) {
  const View1 v{job.st,          job.buf0, job.buf1, job.tab, job.N, job.do_meas, job.do_time, &job.mp,
                job.mp.z,        &job.tc,  job.mode};
  fused1d(v);
}

// Many filters, one CTA each; tcs (if not null) holds the item's constants.
__global__ void __launch_bounds__(kT1) k_fused1d_batch(const Slot1* __restrict__ slots,
                                                       const StepItem* __restrict__ items,
                                                       const TimeConsts* __restrict__ tcs) {
  const StepItem& it = items[blockIdx.x];
  const Slot1& sl = slots[it.slot];
  const View1 v{sl.st, sl.buf0, sl.buf1, sl.tab, sl.N, it.flags & 1, (it.flags >> 1) & 1, sl.mp, it.z,
                tcs ? tcs + blockIdx.x : sl.tc, sl.mode};
  fused1d(v);
}

}  // namespace

int tc1_supported(const pmf_config* cfg, std::string* why) {
  if (cfg->nx != 1 || cfg->N[0] % 8 || cfg->N[0] < 16 || cfg->N[0] > kMaxN1) {
    *why = "the 1-D kernel needs n_x = 1 and N a multiple of 8 in [16, 512]";
    return PMF_ERR_UNSUPPORTED;
  }
  if (cfg->transform == PMF_TRANSFORM_FFT && (cfg->N[0] & (cfg->N[0] - 1))) {
    *why = "the FFT form needs N a power of two";
    return PMF_ERR_UNSUPPORTED;
  }
  return PMF_OK;
}

size_t tc1_table_bytes(int N) { return sizeof(float) * (size_t)(N + 2 * (2 * N + 1)); }

int tc1_build_table(int N, void** dev) {
  std::vector<float> t(N + 2 * (2 * N + 1));
  const double w = 6.283185307179586476925286766559 / N;
  for (int r = 0; r < N; ++r) t[r] = (float)(std::cos(w * r) + std::sin(w * r));
  for (int m = -N; m <= N; ++m) {
    const double ang = 3.14159265358979323846 * m / N;
    t[N + 2 * (m + N)] = (float)std::cos(ang);
    t[N + 2 * (m + N) + 1] = (float)std::sin(ang);
  }
  *dev = nullptr;
  if (cudaMalloc(dev, t.size() * sizeof(float)) != cudaSuccess) return PMF_ERR_OOM;
  if (cudaMemcpy(*dev, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return PMF_ERR_CUDA;
  return PMF_OK;
}

int tc1_step(int N, const void* table, const MeasParams* mp, const TimeConsts* tc, DevState* st, float* b0,
             float* b1, cudaStream_t s, int mode) {
  if (!mp && !tc) return 0;
  Job1 job{};
  job.mode = mode;
  job.st = st;
  job.buf0 = b0;
  job.buf1 = b1;
  job.tab = (const float*)table;
  job.N = N;
  job.do_meas = mp != nullptr;
  job.do_time = tc != nullptr;
  if (mp) job.mp = *mp;
  if (tc) job.tc = *tc;
  k_fused1d<<<1, kT1, 0, s>>>(job);
  return 1;
}

int tc1_batch_step(const Slot1* slots, const StepItem* items, const TimeConsts* tcs, int k, cudaStream_t s) {
  if (k <= 0) return 0;
  k_fused1d_batch<<<k, kT1, 0, s>>>(slots, items, tcs);
  return 1;
}

}  // namespace pmf

namespace pmf {

namespace {

std::mutex g_tune_mu;
std::map<int, int> g_tune;      // N -> mode
std::map<int, std::pair<double, double>> g_tune_us;   // N -> (matrix-vector, FFT) microseconds
bool g_tune_loaded = false;

std::string tune_path() {
  Dl_info info;
  if (!dladdr((void*)&tc1_mode, &info) || !info.dli_fname) return "";
  std::string p = info.dli_fname;
  const size_t slash = p.rfind('/');
  return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/autotune.json";
}

// {"1d:N": {"mode": m, ...}, ...}: read the mode of every 1-D entry.
void tune_load() {
  g_tune_loaded = true;
  const std::string p = tune_path();
  FILE* f = p.empty() ? nullptr : std::fopen(p.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int N = 0, mode = -1;
    double tm = 0.0, tf = 0.0;
    const char* q = std::strstr(line, "\"1d:");
    const int got = q ? std::sscanf(q, "\"1d:%d\": {\"mode\": %d, \"matvec_us\": %lf, \"fft_us\": %lf", &N, &mode, &tm,
                                    &tf)
                      : 0;
    if (got >= 2 && (mode == 0 || mode == 1)) {
      g_tune[N] = mode;
      if (got == 4) g_tune_us[N] = {tm, tf};
    }
  }
  std::fclose(f);
}

void tune_save() {
  const auto& times = g_tune_us;
  const std::string p = tune_path();
  FILE* f = p.empty() ? nullptr : std::fopen(p.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : g_tune) {
    auto t = times.find(kv.first);
    std::fprintf(f, "  \"1d:%d\": {\"mode\": %d", kv.first, kv.second);
    if (t != times.end()) std::fprintf(f, ", \"matvec_us\": %.3f, \"fft_us\": %.3f", t->second.first, t->second.second);
    std::fprintf(f, "}%s\n", ++i < g_tune.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  std::fclose(f);
}

// Mean time of one epoch of a scratch filter of size N in the given mode.
double time_mode(int N, const void* table, int mode, cudaStream_t s) {
  pmf_config c{};
  c.nx = 1;
  c.N[0] = N;
  c.A[0] = -0.5;
  c.Q[0] = 0.5;
  c.P0[0] = 0.25;
  c.span_sigma = 6.0;
  c.dt_sub = 0.01;
  c.realign_rho = 0.5;
  c.precision = PMF_PREC_FP16X3;
  std::string why;
  Job1 job{};
  pmf_meas m{};
  m.kind = PMF_MEAS_LINEAR;
  m.nz = 1;
  m.z[0] = 0.1;
  m.R[0] = 0.01;
  m.H[0] = 1.0;
  if (meas_params(1, &m, &job.mp, &why) || time_consts(c, 0.1, &job.tc, &why)) return -1.0;
  DevState h = initial_state(c);
  std::vector<float> w(2 * (size_t)N);
  for (int j = 0; j < N; ++j) {
    const double u = (j - 0.5 * (N - 1)) / (N / 12.0);
    w[j] = (float)std::exp(-0.5 * u * u);
  }
  DevState* st = nullptr;
  float* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double us = -1.0;
  if (cudaMalloc(&st, sizeof(DevState)) == cudaSuccess && cudaMalloc(&buf, sizeof(float) * 2 * N) == cudaSuccess &&
      cudaMemcpy(st, &h, sizeof(DevState), cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(buf, w.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    job.st = st;
    job.buf0 = buf;
    job.buf1 = buf + N;
    job.tab = (const float*)table;
    job.N = N;
    job.do_meas = 1;
    job.do_time = 1;
    job.mode = mode;
    for (int i = 0; i < 3; ++i) k_fused1d<<<1, kT1, 0, s>>>(job);
    constexpr int kReps = 20;
    cudaEventRecord(e0, s);
    for (int i = 0; i < kReps; ++i) k_fused1d<<<1, kT1, 0, s>>>(job);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      us = 1e3 * ms / kReps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(st);
  cudaFree(buf);
  return us;
}

}  // namespace

int tc1_form(const pmf_config* cfg, const void* table, cudaStream_t s) {
  if (cfg->transform == PMF_TRANSFORM_GEMM) return 0;
  if (cfg->transform == PMF_TRANSFORM_FFT) return 1;
  return tc1_mode(cfg->N[0], table, s);
}

int tc1_mode(int N, const void* table, cudaStream_t s) {
  if (N < 16 || (N & (N - 1))) return 0;   // the FFT form needs a power of two
  if (const char* form = std::getenv("PMF_1D_FORM")) {   // explicit choice, no tuning
    if (!std::strcmp(form, "fft")) return 1;
    if (!std::strcmp(form, "matvec")) return 0;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  if (!g_tune_loaded) tune_load();
  auto it = g_tune.find(N);
  if (it != g_tune.end()) return it->second;
  const double tm = time_mode(N, table, 0, s), tf = time_mode(N, table, 1, s);
  const int mode = (tf > 0.0 && tm > 0.0 && tf < tm) ? 1 : 0;
  g_tune[N] = mode;
  g_tune_us[N] = {tm, tf};
  tune_save();
  return mode;
}

}  // namespace pmf
