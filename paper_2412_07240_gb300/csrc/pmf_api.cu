// C ABI of libpmf (declared in include/pmf.h): filter contexts, validation,
// the float64 model constants of a time update, and dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "pmf_internal.cuh"
#include "pmf_kernels.cuh"
#include "pmf_tc.cuh"

using namespace pmf;

struct pmf_ctx {
  pmf_config cfg;
  cudaStream_t stream = nullptr;
  Dims dims{};
  int path = 0;               // 0 float64 kernels, 1 fused tensor-core kernel
  DevState* st = nullptr;     // device
  void* buf[2] = {nullptr, nullptr};
  double* partials = nullptr;
  double* pend = nullptr;
  double* interp[MAXN] = {nullptr, nullptr, nullptr};
  double* hfwd[MAXN] = {nullptr, nullptr, nullptr};
  double* hinv[MAXN] = {nullptr, nullptr, nullptr};
  double* prior_aux = nullptr;  // P0^{-1} (9) and m0 (3)
  TcTables tct{};               // tensor-core path tables (pmf_tc.cu)
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

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Matrix exponential by scaling and squaring of the Taylor series (float64):
// ||X / 2^s||_1 <= 1/4, terms summed until below 1e-20 of the partial sum.
void expm_host(int n, const double* A, double* E) {
  double nrm = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::fabs(A[i * n + j]);
    nrm = std::fmax(nrm, s);
  }
  int sq = 0;
  if (nrm > 0.25) sq = (int)std::ceil(std::log2(nrm / 0.25));
  const double sc = std::ldexp(1.0, -sq);
  double X[64], T[64], U[64];
  for (int i = 0; i < n * n; ++i) {
    X[i] = A[i] * sc;
    E[i] = 0.0;
    T[i] = 0.0;
  }
  for (int i = 0; i < n; ++i) E[i * n + i] = T[i * n + i] = 1.0;
  for (int k = 1; k < 40; ++k) {
    mm(n, T, X, U);
    double tn = 0.0, en = 0.0;
    for (int i = 0; i < n * n; ++i) {
      T[i] = U[i] / k;
      E[i] += T[i];
      tn = std::fmax(tn, std::fabs(T[i]));
      en = std::fmax(en, std::fabs(E[i]));
    }
    if (tn < 1e-20 * en) break;
  }
  for (int s = 0; s < sq; ++s) {
    mm(n, E, E, U);
    for (int i = 0; i < n * n; ++i) E[i] = U[i];
  }
}

// Constants of a time update over tau (model only): Phi = e^{A tau},
// Q_d = int_0^tau e^{As} Q e^{A^T s} ds (Van Loan block exponential),
// Q_b = Phi^{-1} Q_d Phi^{-T}, E = e^{-A dt}, trace factor.
int make_time_consts(pmf_ctx* ctx, double tau, TimeConsts* tc) {
  const pmf_config& c = ctx->cfg;
  const int n = c.nx;
  *tc = TimeConsts{};
  tc->nx = n;
  for (int a = 0; a < n; ++a) tc->N[a] = c.N[a];
  int l = (int)std::ceil(tau / c.dt_sub - 1e-9);
  if (l < 1) l = 1;
  if (l > MAXL) return fail(ctx, PMF_ERR_ARG, "tau / dt_sub exceeds PMF_MAX_SUBSTEPS");
  tc->l = l;
  tc->tau = tau;
  tc->dt = tau / l;
  tc->exact = c.psi_mode == PMF_PSI_EXACT;
  tc->span = c.span_sigma;
  tc->rho_max = c.realign_rho;
  double At[9], mAt[9], mAdt[9];
  double trA = 0.0;
  for (int i = 0; i < n * n; ++i) {
    At[i] = c.A[i] * tau;
    mAt[i] = -c.A[i] * tau;
    mAdt[i] = -c.A[i] * tc->dt;
    tc->Q[i] = c.Q[i];
  }
  for (int i = 0; i < n; ++i) trA += c.A[i * n + i];
  expm_host(n, At, tc->Phi);
  expm_host(n, mAt, tc->PhiInv);
  expm_host(n, mAdt, tc->Estep);
  const int m = 2 * n;
  double C[36] = {0}, E[36];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      C[i * m + j] = -c.A[i * n + j] * tau;
      C[i * m + n + j] = c.Q[i * n + j] * tau;
      C[(n + i) * m + n + j] = c.A[j * n + i] * tau;
    }
  expm_host(m, C, E);
  double F12[9], Phi2[9], Qd[9];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      F12[i * n + j] = E[i * m + n + j];
      Phi2[i * n + j] = E[(n + j) * m + n + i];  // (F22)^T
    }
  mm(n, Phi2, F12, Qd);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) Qd[i * n + j] = Qd[j * n + i] = 0.5 * (Qd[i * n + j] + Qd[j * n + i]);
  congruence(n, tc->PhiInv, Qd, tc->Qb);
  // rotated diffusion at the sub-step ends: e^{-A q dt} Q e^{-A^T q dt}, q = 1..l
  double Eq[9], mAq[9], Qq[9];
  for (int q = 1; q <= l; ++q) {
    for (int i = 0; i < n * n; ++i) mAq[i] = -c.A[i] * (tc->dt * q);
    expm_host(n, mAq, Eq);
    congruence(n, Eq, c.Q, Qq);
    double* o = tc->Qt[q - 1];
    o[0] = Qq[0];
    o[1] = n > 1 ? Qq[1] : 0.0;
    o[2] = n > 2 ? Qq[2] : 0.0;
    o[3] = n > 1 ? Qq[n + 1] : 0.0;
    o[4] = n > 2 ? Qq[5] : 0.0;
    o[5] = n > 2 ? Qq[8] : 0.0;
  }
  tc->g = tc->exact ? std::exp(-trA * tau) : std::pow(1.0 - tc->dt * trA, (double)l);
  return PMF_OK;
}

int validate_config(const pmf_config* c, std::string* why) {
  if (!c) { *why = "null config"; return PMF_ERR_ARG; }
  if (c->nx < 1 || c->nx > PMF_MAX_NX) { *why = "nx out of range"; return PMF_ERR_ARG; }
  const int n = c->nx;
  for (int a = 0; a < n; ++a)
    if (c->N[a] < 4 || (c->N[a] & 1) || c->N[a] > 4096) { *why = "N must be even, 4..4096"; return PMF_ERR_ARG; }
  if (!finite_all(c->A, n * n) || !finite_all(c->Q, n * n) || !finite_all(c->m0, n) ||
      !finite_all(c->P0, n * n)) { *why = "non-finite model value"; return PMF_ERR_ARG; }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (std::fabs(c->Q[i * n + j] - c->Q[j * n + i]) > 1e-12 * (1 + std::fabs(c->Q[i * n + j])) ||
          std::fabs(c->P0[i * n + j] - c->P0[j * n + i]) > 1e-12 * (1 + std::fabs(c->P0[i * n + j]))) {
        *why = "Q and P0 must be symmetric";
        return PMF_ERR_ARG;
      }
  double L[9], Qs[9], tr = 0.0;
  for (int i = 0; i < n; ++i) tr += std::fabs(c->Q[i * n + i]);
  for (int i = 0; i < n * n; ++i) Qs[i] = c->Q[i];
  for (int i = 0; i < n; ++i) Qs[i * n + i] += 1e-12 * (tr + 1e-300);
  if (tr > 0.0 && !chol(n, Qs, L)) { *why = "Q is not positive semidefinite"; return PMF_ERR_ARG; }
  for (int i = 0; i < n; ++i)
    if (c->Q[i * n + i] < 0) { *why = "Q is not positive semidefinite"; return PMF_ERR_ARG; }
  if (!chol(n, c->P0, L)) { *why = "P0 is not positive definite"; return PMF_ERR_ARG; }
  if (!(c->span_sigma > 0) || !(c->dt_sub > 0) || !(c->realign_rho > 0)) { *why = "span, dt_sub, rho must be > 0"; return PMF_ERR_ARG; }
  if (c->precision < PMF_PREC_FP64 || c->precision > PMF_PREC_FP16X3) { *why = "unknown precision"; return PMF_ERR_ARG; }
  if (c->psi_mode != PMF_PSI_EULER && c->psi_mode != PMF_PSI_EXACT) { *why = "unknown psi mode"; return PMF_ERR_ARG; }
  return PMF_OK;
}

// Hartley matrix cas(2 pi k j / N) with exact integer reduction of k j mod N.
void hartley_host(int N, double scale, double* H) {
  const double w = 6.283185307179586476925286766559 / N;
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j) {
      const long long r = ((long long)k * j) % N;
      H[k * N + j] = scale * (std::cos(w * r) + std::sin(w * r));
    }
}

int build_meas(pmf_ctx* ctx, const pmf_meas* m, MeasParams* mp) {
  const int n = ctx->cfg.nx;
  if (!m) return fail(ctx, PMF_ERR_ARG, "null measurement");
  int nz = m->nz;
  if (m->kind == PMF_MEAS_RANGE) {
    if (nz != 1 || n < 2) return fail(ctx, PMF_ERR_ARG, "range measurement needs nz = 1, nx >= 2");
  } else if (m->kind == PMF_MEAS_BEARING_LINEAR3) {
    if (nz != 2 || n < 3) return fail(ctx, PMF_ERR_ARG, "bearing measurement needs nz = 2, nx = 3");
  } else if (m->kind == PMF_MEAS_LINEAR) {
    if (nz < 1 || nz > PMF_MAX_NZ) return fail(ctx, PMF_ERR_ARG, "linear measurement nz out of range");
    if (!finite_all(m->H, nz * n)) return fail(ctx, PMF_ERR_ARG, "non-finite H");
  } else {
    return fail(ctx, PMF_ERR_ARG, "unknown measurement kind");
  }
  if (!finite_all(m->z, nz) || !finite_all(m->R, nz * nz))
    return fail(ctx, PMF_ERR_ARG, "non-finite z or R");
  double L[9];
  if (!chol(nz, m->R, L)) return fail(ctx, PMF_ERR_ARG, "R is not positive definite");
  *mp = MeasParams{};
  mp->kind = m->kind;
  mp->nz = nz;
  mp->nx = n;
  for (int i = 0; i < nz; ++i) mp->z[i] = m->z[i];
  for (int i = 0; i < nz * n; ++i) mp->H[i] = m->H[i];
  inv(nz, m->R, mp->Rinv);
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
  delete ctx;
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

  if (cfg->precision != PMF_PREC_FP64) {
    rc = tc_supported(cfg, &why);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
    ctx->path = 1;
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
  ALLOC(ctx->partials, sizeof(double) * 10 * 4096);
  ALLOC(ctx->pend, sizeof(double) * 32);
  ALLOC(ctx->prior_aux, sizeof(double) * 16);
  if (ctx->path == 0) {
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
  } else {
    rc = tc_build_tables(cfg, &ctx->tct, &why);
    if (rc) {
      free_ctx(ctx);
      return rc;
    }
  }
#undef ALLOC

  // initial frame c = m0, M = chol(P0) diag(2 span / N)
  DevState h{};
  double L[9];
  chol(n, cfg->P0, L);
  for (int a = 0; a < n; ++a) h.f.c[a] = cfg->m0[a];
  for (int r = 0; r < n; ++r)
    for (int a = 0; a < n; ++a) h.f.M[r * n + a] = L[r * n + a] * (2.0 * cfg->span_sigma / cfg->N[a]);
  inv(n, h.f.M, h.f.Minv);
  h.f.V = std::fabs(det(n, h.f.M));
  h.f.pscale = 1.0;
  double aux[16] = {0};
  inv(n, cfg->P0, aux);
  for (int a = 0; a < n; ++a) aux[9 + a] = cfg->m0[a];
  cudaError_t e = cudaMemcpyAsync(ctx->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->prior_aux, aux, sizeof(aux), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    free_ctx(ctx);
    return PMF_ERR_CUDA;
  }
  if (ctx->path == 0) {
    launch_prior_f64(ctx->dims, ctx->st, ctx->prior_aux, ctx->prior_aux + 9, (double*)ctx->buf[0],
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
                    ctx->partials, ctx->pend, ctx->interp, ctx->hfwd, ctx->hinv, ctx->stream);
    ctx->launches += launches_time_f64(ctx->cfg.nx);
  } else {
    ctx->launches += tc_step(ctx->dims, ctx->cfg, &ctx->tct, nullptr, &ctx->tc, ctx->st,
                             (float*)ctx->buf[0], (float*)ctx->buf[1], ctx->stream);
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
    ctx->launches += tc_step(ctx->dims, ctx->cfg, &ctx->tct, &mp, nullptr, ctx->st,
                             (float*)ctx->buf[0], (float*)ctx->buf[1], ctx->stream);
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
  ctx->launches += tc_step(ctx->dims, ctx->cfg, &ctx->tct, &mp, tcp, ctx->st, (float*)ctx->buf[0],
                           (float*)ctx->buf[1], ctx->stream);
  PMF_CUDA(ctx, cudaGetLastError());
  return PMF_OK;
}

int pmf_sync(pmf_ctx* ctx) {
  if (!ctx) return PMF_ERR_ARG;
  return check_status(ctx);
}

int pmf_moments(pmf_ctx* ctx, double* mean_out, double* cov_out) {
  if (!ctx) return PMF_ERR_ARG;
  int rc = check_status(ctx);
  if (rc) return rc;
  const int n = ctx->cfg.nx;
  DevState h;
  PMF_CUDA(ctx, cudaMemcpy(&h, ctx->st, offsetof(DevState, pa), cudaMemcpyDeviceToHost));
  if (mean_out) std::memcpy(mean_out, h.f.mean, sizeof(double) * n);
  if (cov_out) std::memcpy(cov_out, h.f.cov, sizeof(double) * n * n);
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

long long pmf_num_points(const pmf_ctx* ctx) { return ctx ? ctx->dims.P : 0; }
int pmf_path(const pmf_ctx* ctx) { return ctx ? ctx->path : -1; }
long long pmf_launch_count(const pmf_ctx* ctx) { return ctx ? ctx->launches : 0; }
const char* pmf_last_error(const pmf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
void pmf_destroy(pmf_ctx* ctx) { free_ctx(ctx); }

}  // extern "C"
