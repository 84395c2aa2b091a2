// Host-side model constants and validation (pmf_model.cu).
#pragma once

#include <string>

#include "pmf_internal.cuh"

namespace pmf {

bool finite_all(const double* v, int n);
// Matrix exponential (float64, scaling and squaring of the Taylor series).
void expm_host(int n, const double* A, double* E);
// Constants of a time update over tau: Phi = e^{A tau}, Q_b, the per-sub-step
// rotated diffusion, the trace factor.  PMF_ERR_ARG if tau / dt_sub needs more
// than PMF_MAX_SUBSTEPS sub-steps.
int time_consts(const pmf_config& c, double tau, TimeConsts* tc, std::string* why);
int validate_config(const pmf_config* c, std::string* why);
// Hartley matrix cas(2 pi k j / N) * scale (row-major N x N).
void hartley_host(int N, double scale, double* H);
int meas_params(int n, const pmf_meas* m, MeasParams* mp, std::string* why);
// Initial frame c = m0, M = chol(P0) diag(2 span / N), unit normaliser.
DevState initial_state(const pmf_config& c);

}  // namespace pmf
