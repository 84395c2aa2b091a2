// Host-side model constants and validation shared by the C entry points
// (pmf_api.cu) and the request server (pmf_serve.cu): float64, no device code.
#include <cmath>
#include <cstring>
#include <string>

#include "pmf_model.cuh"

namespace pmf {

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
int time_consts(const pmf_config& c, double tau, TimeConsts* tc, std::string* why) {
  const int n = c.nx;
  *tc = TimeConsts{};
  tc->nx = n;
  for (int a = 0; a < n; ++a) tc->N[a] = c.N[a];
  int l = (int)std::ceil(tau / c.dt_sub - 1e-9);
  if (l < 1) l = 1;
  if (l > MAXL) {
    *why = "tau / dt_sub exceeds PMF_MAX_SUBSTEPS";
    return PMF_ERR_ARG;
  }
  tc->l = l;
  tc->tau = tau;
  tc->dt = tau / l;
  tc->exact = c.psi_mode == PMF_PSI_EXACT;
  tc->realign_mode = c.realign_mode;
  tc->span = c.span_sigma;
  tc->rho_max = c.realign_rho;
  double At[16], mAt[16], mAdt[16];
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
  double C[64] = {0}, E[64];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      C[i * m + j] = -c.A[i * n + j] * tau;
      C[i * m + n + j] = c.Q[i * n + j] * tau;
      C[(n + i) * m + n + j] = c.A[j * n + i] * tau;
    }
  expm_host(m, C, E);
  double F12[16], Phi2[16], Qd[16];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      F12[i * n + j] = E[i * m + n + j];
      Phi2[i * n + j] = E[(n + j) * m + n + i];  // (F22)^T
    }
  mm(n, Phi2, F12, Qd);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) Qd[i * n + j] = Qd[j * n + i] = 0.5 * (Qd[i * n + j] + Qd[j * n + i]);
  congruence(n, tc->PhiInv, Qd, tc->Qb);
  // rotated diffusion at the sub-step ends: e^{-A q dt} Q e^{-A^T q dt}, q = 1..l,
  // with e^{-A q dt} = (e^{-A dt})^q
  double Eq[16], En[16], Qq[16];
  for (int i = 0; i < n * n; ++i) Eq[i] = tc->Estep[i];
  for (int q = 1; q <= l; ++q) {
    if (q > 1) {
      mm(n, Eq, tc->Estep, En);
      for (int i = 0; i < n * n; ++i) Eq[i] = En[i];
    }
    congruence(n, Eq, c.Q, Qq);
    double* o = tc->Qt[q - 1];
    for (int k = 0; k < 10; ++k) o[k] = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = a; b < n; ++b) o[packed_sym(a, b)] = Qq[a * n + b];
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
  double L[16], Qs[16], tr = 0.0;
  for (int i = 0; i < n; ++i) tr += std::fabs(c->Q[i * n + i]);
  for (int i = 0; i < n * n; ++i) Qs[i] = c->Q[i];
  for (int i = 0; i < n; ++i) Qs[i * n + i] += 1e-12 * (tr + 1e-300);
  if (tr > 0.0 && !chol(n, Qs, L)) { *why = "Q is not positive semidefinite"; return PMF_ERR_ARG; }
  for (int i = 0; i < n; ++i)
    if (c->Q[i * n + i] < 0) { *why = "Q is not positive semidefinite"; return PMF_ERR_ARG; }
  if (!chol(n, c->P0, L)) { *why = "P0 is not positive definite"; return PMF_ERR_ARG; }
  if (!(c->span_sigma > 0) || !(c->dt_sub > 0) || !(c->realign_rho > 0)) { *why = "span, dt_sub, rho must be > 0"; return PMF_ERR_ARG; }
  if (c->precision < PMF_PREC_FP64 || c->precision > PMF_PREC_BF16X6 || c->precision == 2) {
    *why = "unknown precision";
    return PMF_ERR_ARG;
  }
  if (c->psi_mode != PMF_PSI_EULER && c->psi_mode != PMF_PSI_EXACT) { *why = "unknown psi mode"; return PMF_ERR_ARG; }
  if (c->realign_mode != PMF_REALIGN_MULTILINEAR && c->realign_mode != PMF_REALIGN_SHEAR) {
    *why = "unknown re-alignment mode";
    return PMF_ERR_ARG;
  }
  if (c->transform < PMF_TRANSFORM_AUTO || c->transform > PMF_TRANSFORM_FFT) {
    *why = "unknown transform form";
    return PMF_ERR_ARG;
  }
  if (c->realign_mode == PMF_REALIGN_SHEAR && c->nx < 2) {
    *why = "shear re-alignment is defined for n_x = 2, 3 and 4";
    return PMF_ERR_ARG;
  }
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

int meas_params(int n, const pmf_meas* m, MeasParams* mp, std::string* why) {
  if (!m) { *why = "null measurement"; return PMF_ERR_ARG; }
  const int nz = m->nz;
  if (m->kind == PMF_MEAS_RANGE) {
    if (nz != 1 || n < 2) { *why = "range measurement needs nz = 1, nx >= 2"; return PMF_ERR_ARG; }
  } else if (m->kind == PMF_MEAS_BEARING_LINEAR3) {
    if (nz != 2 || n < 3) { *why = "bearing measurement needs nz = 2, nx = 3"; return PMF_ERR_ARG; }
  } else if (m->kind == PMF_MEAS_LINEAR) {
    if (nz < 1 || nz > PMF_MAX_NZ) { *why = "linear measurement nz out of range"; return PMF_ERR_ARG; }
    if (!finite_all(m->H, nz * n)) { *why = "non-finite H"; return PMF_ERR_ARG; }
  } else if (m->kind == PMF_MEAS_TERRAIN_GM) {
    if (nz != 1 || n != 4) { *why = "terrain measurement needs nz = 1, nx = 4"; return PMF_ERR_ARG; }
    if (!finite_all(m->p, 22) || !(m->p[17] >= 0.0 && m->p[17] <= 1.0) || !(m->p[20] > 0.0) || !(m->p[21] > 0.0)) {
      *why = "terrain measurement: invalid terrain or mixture parameters";
      return PMF_ERR_ARG;
    }
  } else {
    *why = "unknown measurement kind";
    return PMF_ERR_ARG;
  }
  if (!finite_all(m->z, nz)) { *why = "non-finite z"; return PMF_ERR_ARG; }
  *mp = MeasParams{};
  mp->kind = m->kind;
  mp->nz = nz;
  mp->nx = n;
  for (int i = 0; i < nz; ++i) mp->z[i] = m->z[i];
  if (m->kind == PMF_MEAS_TERRAIN_GM) {
    for (int i = 0; i < PMF_MEAS_NPARAM; ++i) mp->p[i] = m->p[i];
    const double w1 = m->p[17], v1 = m->p[20], v2 = m->p[21];
    mp->gm[0] = 0.5 / v1;
    mp->gm[1] = 0.5 / v2;
    // component constants 1/2 log v_g - log w_g, shifted by a common amount
    // (a constant factor of the likelihood, removed by the normalisation) so
    // that the smaller is log 2: every exponent is then >= 0, which the
    // bitwise minimum over the grid relies on
    double c1 = 0.5 * std::log(v1) - std::log(w1);
    double c2 = 0.5 * std::log(v2) - std::log(1.0 - w1);
    const double lo = std::fmin(c1, c2) - 0.69314718055994530942;
    c1 -= lo;
    c2 -= lo;
    mp->gm[2] = c1;
    mp->gm[3] = c2;
    mp->gm[4] = m->p[18];
    mp->gm[5] = m->p[19];
    return PMF_OK;
  }
  if (!finite_all(m->R, nz * nz)) { *why = "non-finite R"; return PMF_ERR_ARG; }
  double L[9];
  if (!chol(nz, m->R, L)) { *why = "R is not positive definite"; return PMF_ERR_ARG; }
  for (int i = 0; i < nz * n; ++i) mp->H[i] = m->H[i];
  inv(nz, m->R, mp->Rinv);
  return PMF_OK;
}

// Initial frame c = m0, M = chol(P0) diag(2 span / N) and unit normaliser.
DevState initial_state(const pmf_config& c) {
  DevState h{};
  const int n = c.nx;
  double L[16];
  chol(n, c.P0, L);
  for (int a = 0; a < n; ++a) h.f.c[a] = c.m0[a];
  for (int r = 0; r < n; ++r)
    for (int a = 0; a < n; ++a) h.f.M[r * n + a] = L[r * n + a] * (2.0 * c.span_sigma / c.N[a]);
  inv(n, h.f.M, h.f.Minv);
  h.f.V = std::fabs(det(n, h.f.M));
  if (n == 3) {
    h.f.hc[0] = std::atan2(h.f.c[1], h.f.c[0]);
    h.f.hc[1] = h.f.c[0] * h.f.c[0] + h.f.c[1] * h.f.c[1];
  }
  h.f.pscale = 1.0;
  return h;
}

}  // namespace pmf
