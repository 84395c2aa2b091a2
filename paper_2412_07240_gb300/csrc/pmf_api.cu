// C ABI of libpmf (declared in include/pmf.h): filter contexts, validation,
// the float64 model constants of a time update, and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pmf_internal.cuh"
#include "pmf_kernels.cuh"
#include "pmf_model.cuh"
#include "pmf_f4.cuh"
#include "pmf_tc.cuh"

using namespace pmf;

struct pmf_ctx {
  pmf_config cfg;
  cudaStream_t stream = nullptr;
  Dims dims{};
  int path = 0;               // 0 float64 kernels, 1 fused 2-D tensor-core kernel,
                              // 2 3-D tensor-core pipelines, 3 1-D CUDA-core kernel,
                              // 4 float32 4-D kernels
  DevState* st = nullptr;     // device
  void* buf[2] = {nullptr, nullptr};
  double* partials = nullptr;
  double* pend = nullptr;
  double* interp[MAXN] = {};
  double* hfwd[MAXN] = {};
  double* hinv[MAXN] = {};
  double* prior_aux = nullptr;  // P0^{-1} (n*n) and m0 at kAuxM0
  double* scratch = nullptr;    // float64 path, shear re-alignment: intermediate grid
  TcTables tct{};               // tensor-core path tables (pmf_tc.cu)
  F4Tables f4{};                // float32 4-D path tables and scratch (pmf_f4.cu)
  void* tab1 = nullptr;         // 1-D kernel table (pmf_tc1.cu)
  int mode1 = 0;                // 1-D Hartley form (autotuned)
  void* tc3 = nullptr;          // 3-D pipeline state (pmf_tc3.cu)
  TimeConsts tc{};
  double tc_tau = -1.0;
  long long launches = 0;
  std::string err;
};

namespace {

int fail(pmf_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define PMF_CUDA(ctx, call)                                                          \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? PMF_ERR_OOM : PMF_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

int make_time_consts(pmf_ctx* ctx, double tau, TimeConsts* tc) {
  std::string why;
  const int rc = time_consts(ctx->cfg, tau, tc, &why);
  return rc ? fail(ctx, rc, why) : PMF_OK;
}

int build_meas(pmf_ctx* ctx, const pmf_meas* m, MeasParams* mp) {
  std::string why;
  const int rc = meas_params(ctx->cfg.nx, m, mp, &why);
  if (rc) return fail(ctx, rc, why);
  // the 2-D tensor-core kernels form the likelihood of at most two components;
  // the 3-D pipelines form linear and bearing + linear measurements only
  if (ctx->path == 1 && mp->nz > 2)
    return fail(ctx, PMF_ERR_UNSUPPORTED, "the 2-D tensor-core path takes at most two measurement components");
  if (ctx->path == 2 && mp->kind == PMF_MEAS_RANGE)
    return fail(ctx, PMF_ERR_UNSUPPORTED, "the 3-D tensor-core pipelines take linear and bearing + linear measurements");
  return PMF_OK;
}


void free_ctx(pmf_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->st);
  cudaFree(ctx->buf[0]);
  cudaFree(ctx->buf[1]);
  cudaFree(ctx->partials);
  cudaFree(ctx->pend);
  cudaFree(ctx->prior_aux);
  for (int a = 0; a < MAXN; ++a) {
    cudaFree(ctx->interp[a]);
    cudaFree(ctx->hfwd[a]);
    cudaFree(ctx->hinv[a]);
  }
  tc_free_tables(&ctx->tct);
  tc3_free(ctx->tc3);
  f4_free(&ctx->f4);
  cudaFree(ctx->tab1);
  cudaFree(ctx->scratch);
  delete ctx;
}

// The fast paths (fused 2-D kernel, 3-D pipelines, 1-D kernel, 4-D kernels);
// returns the kernel launches.
int fast_step(pmf_ctx* ctx, const MeasParams* mp, const TimeConsts* tc) {
  if (ctx->path == 4) {
    int n = 0;
    if (mp) n += f4_meas(ctx->dims, *mp, ctx->st, ctx->f4, (float*)ctx->buf[0], (float*)ctx->buf[1],
                         ctx->partials, ctx->stream);
    if (tc) n += f4_time(ctx->dims, *tc, ctx->st, ctx->f4, (float*)ctx->buf[0], (float*)ctx->buf[1],
                         ctx->partials, ctx->pend, ctx->stream);
    return n;
  }
  if (ctx->path == 3)
    return tc1_step(ctx->cfg.N[0], ctx->tab1, mp, tc, ctx->st, (float*)ctx->buf[0], (float*)ctx->buf[1],
                    ctx->stream, ctx->mode1);
  if (ctx->path == 2)
    return tc3_step(ctx->tc3, ctx->dims, ctx->cfg, &ctx->tct, mp, tc, ctx->st, (float*)ctx->buf[0],
                    (float*)ctx->buf[1], ctx->stream);
  return tc_step(ctx->dims, ctx->cfg, &ctx->tct, mp, tc, ctx->st, (float*)ctx->buf[0], (float*)ctx->buf[1],
                 ctx->stream);
}

int check_status(pmf_ctx* ctx) {
  int status = 0;
  PMF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  PMF_CUDA(ctx, cudaMemcpy(&status, &ctx->st->f.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != 0) {
    const int zero = 0;
    PMF_CUDA(ctx, cudaMemcpy(&ctx->st->f.status, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return fail(ctx, status, status == PMF_ERR_DEGENERATE
                                 ? "degenerate normaliser: density left unchanged"
                                 : "device reported an error");
  }
  return PMF_OK;
}

}  // namespace

extern "C" {

void pmf_config_defaults(pmf_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->span_sigma = 6.0;
  cfg->dt_sub = 0.01;
  cfg->realign_rho = 0.5;
  cfg->precision = PMF_PREC_FP64;
  cfg->psi_mode = PMF_PSI_EULER;
}

int pmf_create(pmf_ctx** out, const pmf_config* cfg, void* cuda_stream) {
  if (!out) return PMF_ERR_ARG;
  *out = nullptr;
  std::string why;
  int rc = validate_config(cfg, &why);
  if (rc) return rc;
  pmf_ctx* ctx = new (std::nothrow) pmf_ctx();
  if (!ctx) return PMF_ERR_OOM;
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cuda_stream;
  const int n = cfg->nx;
  ctx->dims.nx = n;
  ctx->dims.P = 1;
  for (int a = 0; a < MAXN; ++a) ctx->dims.N[a] = a < n ? cfg->N[a] : 1;
  for (int a = 0; a < n; ++a) ctx->dims.P *= cfg->N[a];
  const long long P = ctx->dims.P;

  if (cfg->transform == PMF_TRANSFORM_FFT &&
      (cfg->precision == PMF_PREC_FP64 ||
       (cfg->nx != 1 && !(cfg->nx == 2 && tc2_fft_ok(cfg->N[0], cfg->N[1], cfg->precision))))) {
    free_ctx(ctx);
    return PMF_ERR_UNSUPPORTED;   // the FFT form: 1-D kernel, fused 2-D kernel with axes 2^a 3^b
  }
  if (cfg->precision != PMF_PREC_FP64) {
    rc = cfg->nx == 1   ? tc1_supported(cfg, &why)
         : cfg->nx == 4 ? f4_supported(cfg, &why)
                        : tc_supported(cfg, &why);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
    ctx->path = cfg->nx == 1 ? 3 : cfg->nx == 4 ? 4 : cfg->nx == 3 ? 2 : 1;
  } else {
    // the float64 per-axis transforms tile lines 16 x 16 with the leading axes
    // on grid.z and the last axis' lines on grid.y (each at most 65535)
    long long lead = 1;
    for (int a = 0; a + 1 < n; ++a) lead *= cfg->N[a];
    const long long lead_but_one = lead / cfg->N[n - 2 < 0 ? 0 : n - 2];
    if ((lead + 15) / 16 > 65535 || (n > 1 && lead_but_one > 65535)) {
      free_ctx(ctx);
      return PMF_ERR_UNSUPPORTED;
    }
  }

#define ALLOC(ptr, bytes)                                     \
  do {                                                        \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));     \
    if (e_ != cudaSuccess) {                                  \
      free_ctx(ctx);                                          \
      return e_ == cudaErrorMemoryAllocation ? PMF_ERR_OOM : PMF_ERR_CUDA; \
    }                                                         \
  } while (0)

  ALLOC(ctx->st, sizeof(DevState));
  const size_t elem = ctx->path == 0 ? sizeof(double) : sizeof(float);
  ALLOC(ctx->buf[0], P * elem);
  ALLOC(ctx->buf[1], P * elem);
  ALLOC(ctx->partials, sizeof(double) * kMomentSlots * 4096);
  ALLOC(ctx->pend, sizeof(double) * kPendSize);
  ALLOC(ctx->prior_aux, sizeof(double) * kAuxSize);
  if (ctx->path == 0) {
    if (cfg->realign_mode == PMF_REALIGN_SHEAR) ALLOC(ctx->scratch, sizeof(double) * (P + 64));
    for (int a = 0; a < n; ++a) {
      const int N = cfg->N[a];
      ALLOC(ctx->interp[a], sizeof(double) * N * N);
      ALLOC(ctx->hfwd[a], sizeof(double) * N * N);
      ALLOC(ctx->hinv[a], sizeof(double) * N * N);
      double* H = new double[(size_t)N * N];
      hartley_host(N, 1.0 / N, H);
      cudaMemcpy(ctx->hfwd[a], H, sizeof(double) * N * N, cudaMemcpyHostToDevice);
      hartley_host(N, 1.0, H);
      cudaMemcpy(ctx->hinv[a], H, sizeof(double) * N * N, cudaMemcpyHostToDevice);
      delete[] H;
    }
  } else if (ctx->path == 4) {
    rc = f4_alloc(cfg, &ctx->f4);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
  } else if (ctx->path == 3) {
    rc = tc1_build_table(cfg->N[0], &ctx->tab1);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
    ctx->mode1 = tc1_form(cfg, ctx->tab1, ctx->stream);
  } else {
    rc = tc_build_tables(cfg, &ctx->tct, &why);
    if (rc == PMF_OK && ctx->path == 1) ctx->tct.fft = tc2_form(cfg, ctx->stream);
    if (rc == PMF_OK && ctx->path == 2) rc = tc3_alloc(&ctx->tc3);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
  }
#undef ALLOC

  // initial frame c = m0, M = chol(P0) diag(2 span / N)
  DevState h = initial_state(*cfg);
  double aux[kAuxSize] = {0};
  inv(n, cfg->P0, aux);
  for (int a = 0; a < n; ++a) aux[kAuxM0 + a] = cfg->m0[a];
  cudaError_t e = cudaMemcpyAsync(ctx->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->prior_aux, aux, sizeof(aux), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    free_ctx(ctx);
    return PMF_ERR_CUDA;
  }
  if (ctx->path == 0) {
    launch_prior_f64(ctx->dims, ctx->st, ctx->prior_aux, ctx->prior_aux + kAuxM0, (double*)ctx->buf[0],
                     ctx->stream);
    launch_moments_f64(ctx->dims, ctx->st, 0, (double*)ctx->buf[0], (double*)ctx->buf[1],
                       ctx->partials, 0, 0, nullptr, ctx->stream);
    ctx->launches += 3;
  } else {
    ctx->launches += tc_prior(ctx->dims, ctx->st, ctx->prior_aux, (float*)ctx->buf[0],
                              ctx->partials, ctx->stream);
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_ctx(ctx);
    return PMF_ERR_CUDA;
  }
  *out = ctx;
  return PMF_OK;
}

int pmf_time_update(pmf_ctx* ctx, double tau) {
  if (!ctx) return PMF_ERR_ARG;
  if (!std::isfinite(tau) || tau < 0) return fail(ctx, PMF_ERR_ARG, "tau must be finite and >= 0");
  if (tau == 0.0) return PMF_OK;
  if (tau != ctx->tc_tau) {
    int rc = make_time_consts(ctx, tau, &ctx->tc);
    if (rc) return rc;
    ctx->tc_tau = tau;
  }
  if (ctx->path == 0) {
    launch_time_f64(ctx->dims, ctx->tc, ctx->st, (double*)ctx->buf[0], (double*)ctx->buf[1],
                    ctx->partials, ctx->pend, ctx->interp, ctx->hfwd, ctx->hinv, ctx->scratch, ctx->stream);
    ctx->launches += launches_time_f64(ctx->cfg.nx) + (ctx->scratch ? ctx->cfg.nx + (ctx->cfg.nx > 2 ? 1 : 0) : 0);
  } else {
    ctx->launches += fast_step(ctx, nullptr, &ctx->tc);
  }
  PMF_CUDA(ctx, cudaGetLastError());
  return PMF_OK;
}

int pmf_meas_update(pmf_ctx* ctx, const pmf_meas* meas) {
  if (!ctx) return PMF_ERR_ARG;
  MeasParams mp;
  int rc = build_meas(ctx, meas, &mp);
  if (rc) return rc;
  if (ctx->path == 0) {
    launch_meas_f64(ctx->dims, mp, ctx->st, (double*)ctx->buf[0], (double*)ctx->buf[1],
                    ctx->partials, ctx->stream);
    ctx->launches += kLaunchesMeasF64;
  } else {
    ctx->launches += fast_step(ctx, &mp, nullptr);
  }
  PMF_CUDA(ctx, cudaGetLastError());
  return PMF_OK;
}

int pmf_step(pmf_ctx* ctx, const pmf_meas* meas, double tau) {
  if (!ctx) return PMF_ERR_ARG;
  if (ctx->path == 0) {
    int rc = pmf_meas_update(ctx, meas);
    if (rc) return rc;
    return pmf_time_update(ctx, tau);
  }
  MeasParams mp;
  int rc = build_meas(ctx, meas, &mp);
  if (rc) return rc;
  if (!std::isfinite(tau) || tau < 0) return fail(ctx, PMF_ERR_ARG, "tau must be finite and >= 0");
  const TimeConsts* tcp = nullptr;
  if (tau > 0.0) {
    if (tau != ctx->tc_tau) {
      rc = make_time_consts(ctx, tau, &ctx->tc);
      if (rc) return rc;
      ctx->tc_tau = tau;
    }
    tcp = &ctx->tc;
  }
  ctx->launches += fast_step(ctx, &mp, tcp);
  PMF_CUDA(ctx, cudaGetLastError());
  return PMF_OK;
}

int pmf_sync(pmf_ctx* ctx) {
  if (!ctx) return PMF_ERR_ARG;
  return check_status(ctx);
}

int pmf_moments(pmf_ctx* ctx, double* mean_out, double* cov_out) {
  if (!ctx) return PMF_ERR_ARG;
  // one copy brings the moments and the status word (the copy waits for the stream)
  FrameState h;
  PMF_CUDA(ctx, cudaMemcpyAsync(&h, &ctx->st->f, sizeof(FrameState), cudaMemcpyDeviceToHost, ctx->stream));
  PMF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h.status != 0) {
    const int zero = 0;
    PMF_CUDA(ctx, cudaMemcpy(&ctx->st->f.status, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return fail(ctx, h.status, h.status == PMF_ERR_DEGENERATE ? "degenerate normaliser: density left unchanged"
                                                              : "device reported an error");
  }
  const int n = ctx->cfg.nx;
  if (mean_out) std::memcpy(mean_out, h.mean, sizeof(double) * n);
  if (cov_out) std::memcpy(cov_out, h.cov, sizeof(double) * n * n);
  return PMF_OK;
}

int pmf_get_pdf(pmf_ctx* ctx, double* host_out, double* c_out, double* M_out) {
  if (!ctx) return PMF_ERR_ARG;
  int rc = check_status(ctx);
  if (rc) return rc;
  const int n = ctx->cfg.nx;
  DevState h;
  PMF_CUDA(ctx, cudaMemcpy(&h, ctx->st, offsetof(DevState, pa), cudaMemcpyDeviceToHost));
  if (c_out) std::memcpy(c_out, h.f.c, sizeof(double) * n);
  if (M_out) std::memcpy(M_out, h.f.M, sizeof(double) * n * n);
  if (host_out) {
    const long long P = ctx->dims.P;
    if (ctx->path == 0) {
      PMF_CUDA(ctx, cudaMemcpy(host_out, ctx->buf[h.f.cur], sizeof(double) * P, cudaMemcpyDeviceToHost));
      for (long long i = 0; i < P; ++i) host_out[i] *= h.f.pscale;
    } else {
      float* tmp = new (std::nothrow) float[P];
      if (!tmp) return fail(ctx, PMF_ERR_OOM, "host buffer");
      cudaError_t e = cudaMemcpy(tmp, ctx->buf[h.f.cur], sizeof(float) * P, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        delete[] tmp;
        return fail(ctx, PMF_ERR_CUDA, cudaGetErrorString(e));
      }
      for (long long i = 0; i < P; ++i) host_out[i] = h.f.pscale * (double)tmp[i];
      delete[] tmp;
    }
  }
  return PMF_OK;
}

int pmf_selftest_bounded_wait(long long polls, int arrive, void* cuda_stream) {
  if (polls < 1) return PMF_ERR_ARG;
  return tc_wait_probe(polls, arrive ? 1 : 0, (cudaStream_t)cuda_stream);
}

long long pmf_num_points(const pmf_ctx* ctx) { return ctx ? ctx->dims.P : 0; }
int pmf_path(const pmf_ctx* ctx) { return ctx ? ctx->path : -1; }
long long pmf_launch_count(const pmf_ctx* ctx) { return ctx ? ctx->launches : 0; }
const char* pmf_last_error(const pmf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
void pmf_destroy(pmf_ctx* ctx) { free_ctx(ctx); }

}  // extern "C"

// ---------------------------------------------------------------------------
// batches of independent 2-D filters (one fused launch per epoch)
// ---------------------------------------------------------------------------
struct pmf_batch {
  int count = 0, precision = 0;
  cudaStream_t stream = nullptr;
  std::vector<pmf_config> cfgs;
  std::vector<long long> npts;
  DevState* d_st = nullptr;
  float* d_w = nullptr;
  MeasParams* d_mp = nullptr;
  TimeConsts* d_tc = nullptr;
  FilterSlot* d_slots = nullptr;
  StepItem* d_items = nullptr;
  double* d_partials = nullptr;
  double* d_aux = nullptr;
  uint8_t* d_plan = nullptr;          // per filter: the front kernel's results of an epoch
  std::vector<void*> tables;          // per distinct N (and size class)
  std::vector<double> tau;            // tau of the constants resident for each filter
  std::vector<int> cls;               // size class of each filter's transform kernel
  std::vector<int> rank;              // position of each filter in the launch order (class, then size)
  std::vector<int> cnt;               // counting-sort positions (count + 1)
  int* d_ids = nullptr;               // filter ids of a moments/status query
  double* d_gather = nullptr;         // 8 doubles per queried filter
  int* h_ids = nullptr;               // pinned staging of the query
  double* h_gather = nullptr;
  StepItem* h_items[2] = {nullptr, nullptr};
  TimeConsts* h_tc[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int parity = 0;
  cudaStream_t cap = nullptr;                 // capture stream of the epoch graphs
  cudaStream_t cap2 = nullptr;                // second branch: the size-64 transform kernel
  cudaEvent_t evf = nullptr, evj = nullptr;   // fork and join of the two branches
  cudaGraphExec_t gx[2] = {nullptr, nullptr}; // item copy + batch kernel, per parity buffer
  int gk[2] = {0, 0};                         // batch size each graph was captured for
  int gk128[2] = {0, 0};                      // ... and its numbers of size-128
  int gk96[2] = {0, 0};                       // and size-96 filters
  int per_epoch = 0;                          // kernel launches in one epoch graph
  long long bytes = 0, launches = 0;
  std::string err;
};

namespace {

void free_batch(pmf_batch* b) {
  if (!b) return;
  cudaFree(b->d_st);
  cudaFree(b->d_w);
  cudaFree(b->d_mp);
  cudaFree(b->d_tc);
  cudaFree(b->d_slots);
  cudaFree(b->d_items);
  cudaFree(b->d_partials);
  cudaFree(b->d_aux);
  cudaFree(b->d_plan);
  cudaFree(b->d_ids);
  cudaFree(b->d_gather);
  cudaFreeHost(b->h_ids);
  cudaFreeHost(b->h_gather);
  for (void* p : b->tables) cudaFree(p);
  for (int i = 0; i < 2; ++i)
    if (b->gx[i]) cudaGraphExecDestroy(b->gx[i]);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  if (b->evf) cudaEventDestroy(b->evf);
  if (b->evj) cudaEventDestroy(b->evj);
  for (int i = 0; i < 2; ++i) {
    cudaFreeHost(b->h_items[i]);
    cudaFreeHost(b->h_tc[i]);
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  }
  delete b;
}

}  // namespace

extern "C" {

int pmf_batch_create(pmf_batch** out, const pmf_config* cfgs, const pmf_meas* models, int count,
                     size_t hbm_budget, void* cuda_stream) {
  if (!out || !cfgs || !models || count < 1) return PMF_ERR_ARG;
  *out = nullptr;
  std::string why;
  const int prec = cfgs[0].precision;
  std::vector<MeasParams> mps(count);
  std::vector<int> forms(count);      // Hartley form per filter (tc2_form)
  std::vector<int> sizes;             // key N * 1000 + size class of the table
  long long wfloats = 0;
  for (int i = 0; i < count; ++i) {
    int rc = validate_config(&cfgs[i], &why);
    if (rc) return rc;
    if (cfgs[i].nx != 2 || cfgs[i].precision != prec ||
        (cfgs[i].transform == PMF_TRANSFORM_FFT && !tc2_fft_ok(cfgs[i].N[0], cfgs[i].N[1], cfgs[i].precision)))
      return PMF_ERR_UNSUPPORTED;
    rc = tc_supported(&cfgs[i], &why);
    if (rc) return rc;
    rc = meas_params(2, &models[i], &mps[i], &why);
    if (rc) return rc;
    if (mps[i].nz > 2) return PMF_ERR_UNSUPPORTED;   // two likelihood components at most
    forms[i] = tc2_form(&cfgs[i], (cudaStream_t)cuda_stream);
    const int cls = tc_class_form(cfgs[i].N[0], cfgs[i].N[1], forms[i], prec);
    for (int a = 0; a < 2; ++a) {
      const int key = cfgs[i].N[a] * 1000 + cls;
      if (std::find(sizes.begin(), sizes.end(), key) == sizes.end()) sizes.push_back(key);
    }
    wfloats += 2LL * cfgs[i].N[0] * cfgs[i].N[1];
  }
  long long bytes = wfloats * 4 + (long long)count * (sizeof(DevState) + sizeof(MeasParams) +
                                                       sizeof(TimeConsts) + sizeof(FilterSlot) +
                                                       sizeof(StepItem) + sizeof(int) + 8 * sizeof(double) +
                                                       (long long)tc_plan_bytes()) +
                    sizeof(double) * (kMomentSlots * 4096 + 16 * (long long)count);
  for (int key : sizes) bytes += (long long)tc_axis_table_bytes(key / 1000, prec, key % 1000);
  if (hbm_budget && (size_t)bytes > hbm_budget) return PMF_ERR_ADMISSION;

  pmf_batch* b = new (std::nothrow) pmf_batch();
  if (!b) return PMF_ERR_OOM;
  b->count = count;
  b->precision = prec;
  b->stream = (cudaStream_t)cuda_stream;
  b->cfgs.assign(cfgs, cfgs + count);
  b->tau.assign(count, -1.0);
  b->cls.assign(count, 128);
  b->bytes = bytes;
#define BALLOC(ptr, n)                                                       \
  do {                                                                       \
    if (cudaMalloc((void**)&(ptr), (n)) != cudaSuccess) {                    \
      free_batch(b);                                                         \
      return PMF_ERR_OOM;                                                    \
    }                                                                        \
  } while (0)
  BALLOC(b->d_st, sizeof(DevState) * count);
  BALLOC(b->d_w, sizeof(float) * wfloats);
  BALLOC(b->d_mp, sizeof(MeasParams) * count);
  BALLOC(b->d_tc, sizeof(TimeConsts) * count);
  BALLOC(b->d_slots, sizeof(FilterSlot) * count);
  BALLOC(b->d_items, sizeof(StepItem) * count);
  BALLOC(b->d_partials, sizeof(double) * kMomentSlots * 4096);
  BALLOC(b->d_aux, sizeof(double) * kAuxSize * count);
  BALLOC(b->d_plan, tc_plan_bytes() * count);
  BALLOC(b->d_ids, sizeof(int) * count);
  BALLOC(b->d_gather, sizeof(double) * 8 * count);
#undef BALLOC
  if (cudaMallocHost((void**)&b->h_ids, sizeof(int) * count) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_gather, sizeof(double) * 8 * count) != cudaSuccess) {
    free_batch(b);
    return PMF_ERR_OOM;
  }
  for (int i = 0; i < 2; ++i) {
    if (cudaMallocHost((void**)&b->h_items[i], sizeof(StepItem) * count) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_tc[i], sizeof(TimeConsts) * count) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) != cudaSuccess) {
      free_batch(b);
      return PMF_ERR_OOM;
    }
  }
  std::vector<void*> tabs(sizes.size());
  std::vector<size_t> hbytes(sizes.size());
  for (size_t s = 0; s < sizes.size(); ++s) {
    if (tc_build_axis_table(sizes[s] / 1000, prec, &tabs[s], &hbytes[s], sizes[s] % 1000) != PMF_OK) {
      b->tables = tabs;
      free_batch(b);
      return PMF_ERR_OOM;
    }
  }
  b->tables = tabs;
  std::vector<DevState> hst(count);
  std::vector<FilterSlot> slots(count);
  std::vector<double> aux(kAuxSize * (size_t)count, 0.0);
  long long off = 0;
  b->npts.resize(count);
  for (int i = 0; i < count; ++i) {
    const pmf_config& c = cfgs[i];
    hst[i] = initial_state(c);
    inv(2, c.P0, &aux[kAuxSize * i]);
    aux[kAuxSize * i + kAuxM0] = c.m0[0];
    aux[kAuxSize * i + kAuxM0 + 1] = c.m0[1];
    const long long P = (long long)c.N[0] * c.N[1];
    b->npts[i] = P;
    FilterSlot& sl = slots[i];
    sl.st = b->d_st + i;
    sl.buf0 = b->d_w + off;
    sl.buf1 = b->d_w + off + P;
    off += 2 * P;
    const int cls = tc_class_form(c.N[0], c.N[1], forms[i], c.precision);
    b->cls[i] = cls;
    for (int a = 0; a < 2; ++a) {
      const size_t s = std::find(sizes.begin(), sizes.end(), c.N[a] * 1000 + cls) - sizes.begin();
      sl.hart[a] = (const uint8_t*)tabs[s];
      sl.sctab[a] = (const float*)((const uint8_t*)tabs[s] + hbytes[s]);
    }
    sl.N0 = c.N[0];
    sl.N1 = c.N[1];
    sl.mp = b->d_mp + i;
    sl.tc = b->d_tc + i;
    sl.plan = b->d_plan + tc_plan_bytes() * i;
    sl.fft = forms[i];
  }
  cudaMemcpy(b->d_st, hst.data(), sizeof(DevState) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_mp, mps.data(), sizeof(MeasParams) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_slots, slots.data(), sizeof(FilterSlot) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_aux, aux.data(), sizeof(double) * aux.size(), cudaMemcpyHostToDevice);
  for (int i = 0; i < count; ++i) {
    Dims d{};
    d.nx = 2;
    d.N[0] = cfgs[i].N[0];
    d.N[1] = cfgs[i].N[1];
    d.N[2] = 1;
    d.P = b->npts[i];
    b->launches += tc_prior(d, b->d_st + i, b->d_aux + kAuxSize * i, slots[i].buf0, b->d_partials, b->stream);
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    free_batch(b);
    return PMF_ERR_CUDA;
  }
  // launch order: size class 128 first, then 96, then 64 (one transform
  // kernel per range); within a class larger grids first (the hardware hands
  // CTAs out in order, so the longest run first and the tail is made of
  // small filters); ties by id.  Each step sorts its items by this rank.
  {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return b->cls[x] != b->cls[y] ? b->cls[x] > b->cls[y] : b->npts[x] > b->npts[y];
    });
    b->rank.assign(count, 0);
    for (int r = 0; r < count; ++r) b->rank[order[r]] = r;
    b->cnt.assign(count + 1, 0);
  }
  *out = b;
  return PMF_OK;
}

int pmf_batch_step(pmf_batch* b, const int* ids, const double* z, const int* do_meas,
                   const double* taus, int k) {
  if (!b || k < 0 || k > b->count || (k && (!ids || !taus))) return PMF_ERR_ARG;
  if (k == 0) return PMF_OK;
  for (int i = 0; i < k; ++i) {
    if (ids[i] < 0 || ids[i] >= b->count || !std::isfinite(taus[i]) || taus[i] < 0) return PMF_ERR_ARG;
    if ((!do_meas || do_meas[i]) && (!z || !finite_all(&z[(size_t)i * PMF_MAX_NZ], PMF_MAX_NZ)))
      return PMF_ERR_ARG;
  }
  const int p = b->parity;
  b->parity ^= 1;
  // the pinned buffers of this parity were last read by the copies two steps ago
  if (cudaEventSynchronize(b->ev[p]) != cudaSuccess) return PMF_ERR_CUDA;
  StepItem* items = b->h_items[p];
  TimeConsts* stage = b->h_tc[p];
  int nchanged = 0;
  std::vector<int> changed;
  std::vector<double> changed_tau;
  // items in launch order (the rank of each filter, fixed at creation): a
  // counting sort over the ranks of the listed ids, each item written once,
  // straight into its position.  Ranks are one per filter, so a count above
  // one is an id listed twice, which would step one filter in two CTAs.
  std::vector<int>& pos = b->cnt;
  std::fill(pos.begin(), pos.end(), 0);
  for (int i = 0; i < k; ++i)
    if (++pos[b->rank[ids[i]] + 1] > 1) {
      b->err = "an id is listed twice in one step";
      return PMF_ERR_ARG;
    }
  for (int r = 0; r < b->count; ++r) pos[r + 1] += pos[r];
  for (int i = 0; i < k; ++i) {
    const int id = ids[i];
    const double tau = taus[i];
    const bool meas = !do_meas || do_meas[i];
    StepItem& it = items[pos[b->rank[id]]++];
    it.slot = id;
    it.flags = (meas ? 1 : 0) | (tau > 0 ? 2 : 0);
    for (int j = 0; j < PMF_MAX_NZ; ++j) it.z[j] = meas ? z[(size_t)i * PMF_MAX_NZ + j] : 0.0;
    if (tau > 0 && tau != b->tau[id]) {
      std::string why;
      const int rc = time_consts(b->cfgs[id], tau, &stage[nchanged], &why);
      if (rc) {
        b->err = why;
        return rc;
      }
      changed.push_back(id);
      changed_tau.push_back(tau);
      ++nchanged;
    }
  }
  auto cls = [&](const StepItem& x) { return b->cls[x.slot]; };
  int k128 = 0, k96 = 0;
  while (k128 < k && cls(items[k128]) == 128) ++k128;
  while (k128 + k96 < k && cls(items[k128 + k96]) == 96) ++k96;
  for (int j = 0; j < nchanged; ++j)
    if (cudaMemcpyAsync(b->d_tc + changed[j], &stage[j], sizeof(TimeConsts), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
      return PMF_ERR_CUDA;
  // the resident constants are those of the new taus only once all of them
  // are computed and on their way (a rejected tau leaves every filter as it was)
  for (int j = 0; j < nchanged; ++j) b->tau[changed[j]] = changed_tau[j];
  // the item copy and the batch kernel replay as one CUDA graph, captured
  // once per parity buffer and batch size (the copy reads this parity's
  // pinned items when the graph runs)
  if (!b->gx[p] || b->gk[p] != k || b->gk128[p] != k128 || b->gk96[p] != k96) {
    if (b->gx[p]) {
      cudaGraphExecDestroy(b->gx[p]);
      b->gx[p] = nullptr;
    }
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return PMF_ERR_CUDA;
    if (!b->cap2 && (cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&b->evf, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&b->evj, cudaEventDisableTiming) != cudaSuccess))
      return PMF_ERR_CUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PMF_ERR_CUDA;
    cudaMemcpyAsync(b->d_items, items, sizeof(StepItem) * k, cudaMemcpyHostToDevice, b->cap);
    b->per_epoch = tc_batch_epoch(b->precision, b->d_slots, b->d_items, k, k128, k96, b->cap, nullptr, b->cap2,
                                  b->evf, b->evj);
    if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess) return PMF_ERR_CUDA;
    const cudaError_t e = cudaGraphInstantiate(&b->gx[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gx[p] = nullptr;
      return PMF_ERR_CUDA;
    }
    b->gk[p] = k;
    b->gk128[p] = k128;
    b->gk96[p] = k96;
  }
  if (cudaGraphLaunch(b->gx[p], b->stream) != cudaSuccess) return PMF_ERR_CUDA;
  cudaEventRecord(b->ev[p], b->stream);
  b->launches += b->per_epoch;
  return cudaGetLastError() == cudaSuccess ? PMF_OK : PMF_ERR_CUDA;
}

namespace {

// Gather {mean, cov, status} of the listed filters on the device (clearing
// their status words) and copy them to the pinned host buffer; synchronous.
int batch_query(pmf_batch* b, const int* ids, int k) {
  for (int i = 0; i < k; ++i)
    if (ids[i] < 0 || ids[i] >= b->count) return PMF_ERR_ARG;
  if (k == 0) return cudaStreamSynchronize(b->stream) == cudaSuccess ? PMF_OK : PMF_ERR_CUDA;
  // the copies and the gather follow the batch's epochs on its stream; the
  // previous query ended with a synchronisation, so the pinned ids are free
  std::memcpy(b->h_ids, ids, sizeof(int) * k);
  if (cudaMemcpyAsync(b->d_ids, b->h_ids, sizeof(int) * k, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return PMF_ERR_CUDA;
  b->launches += tc_batch_gather(b->d_st, b->d_ids, k, b->d_gather, b->stream);
  if (cudaMemcpyAsync(b->h_gather, b->d_gather, sizeof(double) * 8 * k, cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return PMF_ERR_CUDA;
  return PMF_OK;
}

}  // namespace

int pmf_batch_moments(pmf_batch* b, const int* ids, int k, double* means, double* covs) {
  if (!b || k < 0 || k > b->count || (k && !ids)) return PMF_ERR_ARG;
  const int q = batch_query(b, ids, k);
  if (q) return q;
  int rc = PMF_OK;
  for (int i = 0; i < k; ++i) {
    const double* g = b->h_gather + (size_t)i * 8;
    if (g[6] != 0.0) rc = (int)g[6];
    if (means) std::memcpy(means + 2 * i, g, sizeof(double) * 2);
    if (covs) std::memcpy(covs + 4 * i, g + 2, sizeof(double) * 4);
  }
  return rc;
}

int pmf_batch_status(pmf_batch* b, const int* ids, int k, int* status_out) {
  if (!b || k < 0 || k > b->count || (k && (!ids || !status_out))) return PMF_ERR_ARG;
  const int q = batch_query(b, ids, k);
  if (q) return q;
  for (int i = 0; i < k; ++i) status_out[i] = (int)b->h_gather[(size_t)i * 8 + 6];
  return PMF_OK;
}

int pmf_batch_get_pdf(pmf_batch* b, int id, double* host_out, double* c_out, double* M_out) {
  if (!b || id < 0 || id >= b->count) return PMF_ERR_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return PMF_ERR_CUDA;
  FrameState f;
  if (cudaMemcpy(&f, &b->d_st[id].f, sizeof(FrameState), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PMF_ERR_CUDA;
  if (c_out) std::memcpy(c_out, f.c, sizeof(double) * 2);
  if (M_out) std::memcpy(M_out, f.M, sizeof(double) * 4);
  if (host_out) {
    FilterSlot sl;
    if (cudaMemcpy(&sl, b->d_slots + id, sizeof(FilterSlot), cudaMemcpyDeviceToHost) != cudaSuccess)
      return PMF_ERR_CUDA;
    const long long P = b->npts[id];
    std::vector<float> tmp(P);
    if (cudaMemcpy(tmp.data(), f.cur ? sl.buf1 : sl.buf0, sizeof(float) * P, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return PMF_ERR_CUDA;
    for (long long i = 0; i < P; ++i) host_out[i] = f.pscale * (double)tmp[i];
  }
  return PMF_OK;
}

long long pmf_batch_bytes(const pmf_batch* b) { return b ? b->bytes : 0; }
long long pmf_batch_launch_count(const pmf_batch* b) { return b ? b->launches : 0; }
void pmf_batch_destroy(pmf_batch* b) { free_batch(b); }

}  // extern "C"
