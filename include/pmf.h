/*
 * pmf.h -- C ABI of the GB300 spectral point-mass filter (libpmf.so).
 *
 * The library implements the grid-based filter of Matousek, Dunik and Brandner,
 * "Efficient Spectral Differentiation in Grid-Based Continuous State
 * Estimation" (FUSION 2024) for the model of Sec. I:
 *
 *     dx = A x dt + Q dw,   E[dw dw^T] = I dt        (eq. dynam)
 *     z_k = h(x_k) + v_k,   v_k ~ N(0, R)             (eq. meas)
 *
 * Q is the diffusion (covariance-rate) matrix of the Fokker-Planck equation
 * (eq. fokker).  The density is a point-mass density (eq. PDF_pm) on an
 * equidistant grid held in an affine frame x = c + M u, u_m = j_m - (N_m-1)/2,
 * that moves with the dynamics (eq. gridMov).  A time update solves the moved
 * Fokker-Planck equation (eq. easyFPE) with the spectral second derivative
 * (eq. secDer) inside the Euler scheme of the Sec. V-B algorithm; a measurement
 * update applies Bayes' rule (eq. filt).
 *
 * Conventions for every entry point
 *   - Matrices are row-major float64 arrays, n_x <= PMF_MAX_NX.
 *   - Grid arrays are C-order (axis n_x-1 fastest), N_m points along axis m.
 *   - Host pointers are caller-owned and read (or written) only during the
 *     call.  Device memory is owned by the context that allocated it.
 *   - A CUDA stream handle (cudaStream_t passed as void*, NULL = legacy
 *     default stream) is borrowed: all work of a context is enqueued on it
 *     and it must outlive the context.  Calls return once the work is
 *     enqueued, except the ones documented as synchronous.
 *   - Functions return PMF_OK or a PMF_ERR_* code and never throw.  The text
 *     of the last error of a context is available from pmf_last_error().
 */
#ifndef PMF_H
#define PMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMF_MAX_NX 4
#define PMF_MEAS_NPARAM 24
#define PMF_MAX_NZ 3
#define PMF_MAX_SUBSTEPS 64

/* Return codes. */
enum {
  PMF_OK = 0,
  PMF_ERR_ARG = 1,         /* invalid argument (sizes, non-finite values, Q not PSD ...) */
  PMF_ERR_OOM = 2,         /* device allocation failed */
  PMF_ERR_CUDA = 3,        /* CUDA runtime error (message in pmf_last_error) */
  PMF_ERR_DEGENERATE = 4,  /* normaliser zero or non-finite; density left unchanged */
  PMF_ERR_TIMEOUT = 5,     /* a bounded device wait expired */
  PMF_ERR_ADMISSION = 6,   /* request exceeds the device-memory budget */
  PMF_ERR_UNSUPPORTED = 7  /* configuration not supported by the selected path */
};

/* Arithmetic of the per-axis transforms (the differentiation GEMMs).
 *   FP64    : float64 grid and float64 transforms (the plain reference path).
 *   TF32    : float32 grid, one TF32 tensor-core product per transform.
 *   BF16X3  : float32 grid, split BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate.
 *   FP16X3  : float32 grid, split FP16 with power-of-two operand scaling,
 *             (hi*hi + hi*lo + lo*hi), FP32 accumulate.
 *   BF16X6  : float32 grid, each operand split into three BF16 pieces
 *             (hi + mid + lo carry its 24 significand bits) and six products
 *             (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid), FP32
 *             accumulate: float32-class transforms from BF16 tensor cores.
 *             n_x = 2 only (single filters, batches and the server's 2-D
 *             filters, whose 3-D filters then run FP16X3), GEMM form of the
 *             transforms only (its operand planes fill the shared memory
 *             the FFT form uses as scratch).
 * Everything else of a step runs in float32 on the non-FP64 paths, with the
 * frame, the normalisation constant and the moment combination in float64.
 * For n_x = 1 every precision other than FP64 selects the float32 CUDA-core
 * kernel (a 1-D transform is a matrix-vector product, not a tensor-core tile).
 * For n_x = 4 every precision other than FP64 selects the float32 4-D kernels
 * (float32 weights, split-FP16 tensor-core contractions along axes 0 and 1
 * and float32 shared-memory contractions along axes 2 and 3, N <= 64 per
 * axis; the measurement exponents and moment sums keep float64-class
 * accuracy). */
enum {
  PMF_PREC_FP64 = 0,
  PMF_PREC_TF32 = 1,
  /* 2 is not assigned */
  PMF_PREC_BF16X3 = 3,
  PMF_PREC_FP16X3 = 4,
  PMF_PREC_BF16X6 = 5
};

/* Diffusion multiplier of the time update.
 *   EULER : the Sec. V-B algorithm, Psi = prod_{n=1..l} psi(t_k + n dt) and
 *           trace factor (1 - dt tr A)^l, l = ceil(tau / dt_sub).
 *   EXACT : exact in time, Psi = exp(int d(k, t) dt), trace factor e^{-tr A tau}
 *           (the alternative time stepping named as future work in Sec. VII). */
enum { PMF_PSI_EULER = 0, PMF_PSI_EXACT = 1 };

/* Fill of a re-aligned frame (the regrid when the frame's whitened
 * correlation exceeds realign_rho; Sec. V grid reshaping).
 *   MULTILINEAR : multilinear interpolation of the old weights (any n_x).
 *   SHEAR       : n_x = 2, 3 or 4: the trigonometric interpolant (eq.
 *                 interFreq) of the old weights at the new nodes, as n
 *                 line-wise passes (per line: DFT, evaluation at that line's
 *                 affine positions); spectrally accurate for densities well
 *                 inside the box. */
enum { PMF_REALIGN_MULTILINEAR = 0, PMF_REALIGN_SHEAR = 1 };

/* Form of the per-axis Hartley transforms (step 1 and step 5 of the Sec. V-B
 * algorithm).
 *   AUTO : per grid size the faster form, measured on first use: n_x = 1
 *          (matrix-vector or FFT; PMF_1D_FORM=matvec|fft overrides it) and
 *          n_x = 2 on the tensor-core paths (GEMM or FFT, per (N0, N1,
 *          precision); PMF_2D_FORM=gemm|fft overrides it); the choices are
 *          cached in autotune.json / autotune_2d.json beside the library.
 *          The contraction everywhere else.
 *   GEMM : the dense contraction with the N x N transform matrix (every path).
 *   FFT  : shared-memory FFTs of the real lines (H_k = Re Z_k - Im Z_k):
 *          n_x = 1 with N a power of two (radix 2), n_x = 2 with both axes
 *          2^a 3^b (radix 3 and 2; the regrid stays a tensor-core GEMM);
 *          non-FP64 precision other than BF16X6; PMF_ERR_UNSUPPORTED
 *          elsewhere. */
enum { PMF_TRANSFORM_AUTO = 0, PMF_TRANSFORM_GEMM = 1, PMF_TRANSFORM_FFT = 2 };

/* Measurement functions h of eq. meas. */
enum {
  PMF_MEAS_LINEAR = 0,          /* h(x) = H x, nz rows of H */
  PMF_MEAS_RANGE = 1,           /* h(x) = sqrt(x1^2 + x2^2), nz = 1 */
  PMF_MEAS_BEARING_LINEAR3 = 2  /* h(x) = [atan2(x2, x1), x3], nz = 2; the bearing
                                   residual is wrapped to (-pi, pi] */,
  PMF_MEAS_TERRAIN_GM = 3       /* n_x = 4, state [p_x, v_x, p_y, v_y], nz = 1:
                                   h(x) = p[16] + sum_{i<4} p[4i] sin(p[4i+1] p_x
                                          + p[4i+2] p_y + p[4i+3]) (a smooth
                                   terrain altitude), noise a two-component
                                   Gaussian mixture: weight p[17] (the other
                                   1 - p[17]), means p[18], p[19], variances
                                   p[20], p[21] (Sec. VI); R is not used */
};

typedef struct pmf_config {
  int nx;                       /* state dimension, 1..PMF_MAX_NX */
  int N[PMF_MAX_NX];            /* grid points per axis (even; the tensor-core
                                   paths need multiples of 16 and N <= 128, the
                                   1-D kernel a multiple of 8 in [16, 512]) */
  double A[PMF_MAX_NX * PMF_MAX_NX];   /* drift, nx x nx row-major packed (a_ij at i*nx+j) */
  double Q[PMF_MAX_NX * PMF_MAX_NX];   /* diffusion, symmetric PSD, packed like A */
  double m0[PMF_MAX_NX];        /* prior mean */
  double P0[PMF_MAX_NX * PMF_MAX_NX];  /* prior covariance, symmetric PD, packed like A */
  double span_sigma;            /* grid half-width in standard deviations (default 6) */
  double dt_sub;                /* Euler sub-step bound (default 0.01) */
  double realign_rho;           /* whitened-correlation threshold for re-alignment (0.5) */
  int precision;                /* PMF_PREC_* */
  int psi_mode;                 /* PMF_PSI_* */
  int realign_mode;             /* PMF_REALIGN_* (default MULTILINEAR) */
  int transform;                /* PMF_TRANSFORM_* (default AUTO) */
} pmf_config;

typedef struct pmf_meas {
  int kind;                     /* PMF_MEAS_* */
  int nz;                       /* measurement dimension (1..PMF_MAX_NZ; at most 2
                                   for 2-D filters on the tensor-core path, in
                                   batches and in the server: PMF_ERR_UNSUPPORTED;
                                   3-D tensor-core filters take LINEAR and
                                   BEARING_LINEAR3, not RANGE) */
  double z[PMF_MAX_NZ];         /* measurement */
  double R[PMF_MAX_NZ * PMF_MAX_NZ];   /* noise covariance, symmetric PD, nz x nz packed */
  double H[PMF_MAX_NZ * PMF_MAX_NX];   /* LINEAR only: nz x nx row-major packed */
  double p[PMF_MEAS_NPARAM];    /* parameters of the model kinds that need them */
} pmf_meas;

typedef struct pmf_ctx pmf_ctx;

/* Fill a config with the defaults (span 6, dt_sub 0.01, rho 0.5, FP64, EULER). */
void pmf_config_defaults(pmf_config* cfg);

/* Create a filter: allocate its device grid, build the transform tables and
 * sample the prior N(m0, P0) on the initial frame c = m0,
 * M = chol(P0) diag(2 span / N_m) (the box covers +-span whitened sigma).
 * Eq. PDF_pm: weights normalised so that |det M| sum P = 1.
 * Errors: PMF_ERR_ARG, PMF_ERR_OOM, PMF_ERR_CUDA, PMF_ERR_UNSUPPORTED
 * (e.g. a tensor-core precision for a grid the fused kernel cannot hold).
 * On error *out is NULL. */
int pmf_create(pmf_ctx** out, const pmf_config* cfg, void* cuda_stream);

/* Time update over tau >= 0 (Sec. V-B algorithm on the moving grid of
 * eq. gridMov), preceded by the regrid that re-centres the grid on the current
 * mean and sizes it for +-span sigma of the predicted covariance pulled back by
 * e^{-A tau}.  tau = 0 is a no-op.  Asynchronous.  Errors: PMF_ERR_ARG. */
int pmf_time_update(pmf_ctx* ctx, double tau);

/* Measurement update (eq. filt): weights times exp(-1/2 r^T R^-1 r),
 * r = z - h(x), normalised; the mean and covariance are recomputed on the
 * device.  Asynchronous; a degenerate normaliser is reported by the next
 * synchronous call (pmf_moments / pmf_get_pdf / pmf_sync) as
 * PMF_ERR_DEGENERATE, with the weights of before the update kept. */
int pmf_meas_update(pmf_ctx* ctx, const pmf_meas* meas);

/* One filter epoch: measurement update with *meas, then time update over tau.
 * Same semantics as the two calls in sequence; on the fused tensor-core path
 * it is a single kernel launch. */
int pmf_step(pmf_ctx* ctx, const pmf_meas* meas, double tau);

/* Mean (nx) and covariance (nx*nx, row-major) of the current density as point
 * sums m = V sum P x, C = V sum P (x-m)(x-m)^T.  Synchronous on the stream. */
int pmf_moments(pmf_ctx* ctx, double* mean_out, double* cov_out);

/* Copy the normalised weights (prod N_m doubles, C-order) and the frame
 * (c: nx, M: nx*nx) to host memory; any pointer may be NULL.  Synchronous. */
int pmf_get_pdf(pmf_ctx* ctx, double* host_out, double* c_out, double* M_out);

/* Wait for the context's stream and report a pending device-side status. */
int pmf_sync(pmf_ctx* ctx);

/* Number of grid points (prod N_m) and the selected path:
 * 0 = plain FP64 kernels, 1 = fused 2-D tensor-core kernel, 2 = 3-D
 * tensor-core pipelines, 3 = 1-D CUDA-core kernel, 4 = float32 4-D kernels. */
long long pmf_num_points(const pmf_ctx* ctx);
int pmf_path(const pmf_ctx* ctx);

/* Kernel launches issued by this context so far (for launch accounting). */
long long pmf_launch_count(const pmf_ctx* ctx);

const char* pmf_last_error(const pmf_ctx* ctx);
void pmf_destroy(pmf_ctx* ctx);

/* ---- batches of independent filters ------------------------------------------
 * A batch holds many filters resident on the device (weights, frames, moments,
 * model constants) and advances any subset of them per epoch with one CUDA
 * graph: a front kernel (measurement update, moments, float64 regrid
 * decision; one CTA per filter) and one transform kernel per size class
 * (largest axis up to 64, 96 or 128; one CTA per filter, larger grids
 * scheduled first).  All filters of a batch share n_x = 2 and the precision
 * of cfgs[0] (a tensor-core format); grid sizes may differ (multiples of 16
 * up to 128).  The per-filter semantics are those of pmf_step. */
typedef struct pmf_batch pmf_batch;

/* Create `count` filters from cfgs[i] with measurement models models[i] (z is
 * ignored; the measurement of each epoch comes with pmf_batch_step).  Device
 * memory needed: pmf_batch_bytes().  If it exceeds hbm_budget (bytes; 0 = no
 * limit) nothing is allocated and PMF_ERR_ADMISSION is returned.  Errors:
 * PMF_ERR_ARG, PMF_ERR_UNSUPPORTED, PMF_ERR_OOM, PMF_ERR_CUDA. */
int pmf_batch_create(pmf_batch** out, const pmf_config* cfgs, const pmf_meas* models, int count,
                     size_t hbm_budget, void* cuda_stream);

/* One epoch for k filters ids[0..k): measurement update with
 * z[i*PMF_MAX_NZ ...] (skipped when do_meas[i] == 0; do_meas may be NULL = all)
 * then time update over taus[i] (skipped when taus[i] == 0).  Asynchronous;
 * ids must be distinct within a call.  Model constants are recomputed on the
 * host only for filters whose tau changed.  The item upload and the batch
 * kernels run as a CUDA graph, captured on the first epoch of each batch
 * size (and split into size classes) and replayed afterwards.  PMF_ERR_ARG
 * for an id out of range or listed twice, a negative or non-finite tau, a
 * non-finite z of a measured filter, or a tau needing more than
 * PMF_MAX_SUBSTEPS sub-steps (then no filter of the call is stepped);
 * PMF_ERR_CUDA on a copy or launch error. */
int pmf_batch_step(pmf_batch* b, const int* ids, const double* z, const int* do_meas,
                   const double* taus, int k);

/* Means (k*nx) and covariances (k*nx*nx) of filters ids[0..k), k <= count
 * (gathered on the device, one copy back).  Synchronous.  Returns
 * PMF_ERR_DEGENERATE if any listed filter reported a degenerate normaliser
 * (its density is left unchanged); the listed status words are then clear. */
int pmf_batch_moments(pmf_batch* b, const int* ids, int k, double* means, double* covs);

/* Status words of filters ids[0..k), k <= count (PMF_OK or the PMF_ERR_*
 * their last epoch reported, e.g. PMF_ERR_DEGENERATE), cleared after reading.
 * Synchronous. */
int pmf_batch_status(pmf_batch* b, const int* ids, int k, int* status_out);

/* Normalised weights of filter id (prod N_m doubles) and its frame.  Synchronous. */
int pmf_batch_get_pdf(pmf_batch* b, int id, double* host_out, double* c_out, double* M_out);

/* Device bytes held by the batch, and kernel launches issued so far. */
long long pmf_batch_bytes(const pmf_batch* b);
long long pmf_batch_launch_count(const pmf_batch* b);
void pmf_batch_destroy(pmf_batch* b);

/* Finite-difference comparator of Sec. III-B/III-C (eq. fdiff, eq. FST), as
 * a baseline for the accuracy per grid point of the spectral method.
 * count independent 1-D grids of N interior nodes with zero boundary values
 * (model dx = a x dt + q dw) are advanced by l explicit sub-steps of length
 * dt, the node spacing moving as delta_n = e^{a dt} delta_{n-1} from delta0,
 * through the sine-transform form P' = 2/(N+1) R diag(prod lambda) R P
 * (float64, two DST-I matrix products).  P_in, P_out: device arrays of
 * count * N doubles (grid g at g * N), not aliased; work: device array of at
 * least count * N + 4 * N + 2 doubles (caller-owned scratch).  Asynchronous
 * on cuda_stream.  PMF_ERR_ARG on bad sizes or parameters. */
int pmf_fdm_transition(const double* P_in, double* P_out, double* work, int N, int count, double q, double a,
                       double dt, int l, double delta0, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving: resident filters of mixed dimension updated by continuous batching.
 * (The paper runs one filter; this layer has no counterpart there.)
 *
 * A server owns the device memory of every admitted filter (grids, frame
 * state, measurement model) and three CUDA streams of its own.  A request is a
 * measurement z followed by a time update over tau, the time to the filter's
 * next measurement (pmf_step semantics).  Requests queue per filter; whenever
 * fewer than PMF_SERVE_INFLIGHT batches are on the device the server forms a
 * batch from the head request of every idle filter that has one: the 1-D
 * filters in one launch of the 1-D kernel, the 2-D filters through the
 * batched 2-D kernels (front kernel and size-class transform kernels), the
 * 3-D filters through their pipelines on the third stream, all three
 * overlapping.  A filter has at most one request on the
 * device, and each runs in its own CTAs, so its results do not depend on what
 * else shares the batch.  A tau needing more than PMF_MAX_SUBSTEPS sub-steps
 * runs as consecutive time updates of at most that many.
 * ------------------------------------------------------------------------- */
#define PMF_SERVE_INFLIGHT 4
#define PMF_SERVE_NSTATS 6
typedef struct pmf_server pmf_server;

/* hbm_budget: device bytes the server may hold for filters and their tables
 * (0 = no limit); max_filters: size of the id space (ids 0..max_filters-1);
 * precision: PMF_PREC_FP16X3, _BF16X3, _BF16X6 or _TF32 for the 2-D and
 * 3-D filters (1-D filters use the float32 kernel; with BF16X6 the 3-D
 * filters run FP16X3, the other split format within 1e-5).  PMF_ERR_ARG on bad arguments,
 * PMF_ERR_OOM / PMF_ERR_CUDA if the server's own buffers cannot be made. */
int pmf_server_create(pmf_server** out, size_t hbm_budget, int max_filters, int precision);

/* Admit a filter with measurement model `model` (z is ignored); its prior is
 * formed on the device before the call returns.  *id_out receives its id.
 * PMF_ERR_ADMISSION if its memory would exceed the budget or no id is free,
 * PMF_ERR_UNSUPPORTED if no fast path holds the grid (1-D: N multiple of 8 in
 * [16, 512]; 2-D and 3-D: multiples of 16 up to 128), PMF_ERR_ARG on an
 * invalid configuration or model. */
int pmf_server_admit(pmf_server* s, const pmf_config* cfg, const pmf_meas* model, int* id_out);

/* Release filter id and its memory (after its work on the device). */
int pmf_server_evict(pmf_server* s, int id);

/* Device bytes held for the admitted filters and shared tables (the amount
 * the budget is checked against). */
long long pmf_server_bytes(const pmf_server* s);

/* Replay a request log in real time on the calling thread.  Request i arrives
 * t_arrival[i] seconds after the call starts (ascending), for filter ids[i],
 * with measurement z[i*PMF_MAX_NZ ...] and then a time update over taus[i]
 * (finite, >= 0).  Returns when every request has completed.  latency_out[i]
 * (may be NULL) = completion observed on the host - arrival, in seconds.
 * stats_out (may be NULL) receives PMF_SERVE_NSTATS doubles: wall seconds,
 * batches, kernel launches, largest batch, mean batch, requests.  All arrays
 * are caller-owned host memory, read during the call only. */
int pmf_server_replay(pmf_server* s, long long n, const double* t_arrival, const int* ids, const double* z,
                      const double* taus, double* latency_out, double* stats_out);

/* Mean (nx) and covariance (nx*nx) of filter id.  Synchronous; returns the
 * filter's pending device status (e.g. PMF_ERR_DEGENERATE), then clears it. */
int pmf_server_moments(pmf_server* s, int id, double* mean_out, double* cov_out);

/* Weights (prod N), frame centre and matrix of filter id, as pmf_get_pdf. */
int pmf_server_get_pdf(pmf_server* s, int id, double* host_out, double* c_out, double* M_out);

const char* pmf_server_last_error(const pmf_server* s);
void pmf_server_destroy(pmf_server* s);

/* ---- moments without device allocation --------------------------------------
 * The paper has no counterpart to this entry point: it is a service for
 * callers that cannot allocate device memory when they need the moments --
 * hosts whose own allocator owns all device memory and forbids libraries to
 * allocate, and real-time loops that must not pay the latency or risk the
 * failure of a cudaMalloc.  It computes S0 = sum w and the mean and covariance
 * of the point sums of a float64 weight array on a frame x = c + M u,
 * u_m = j_m - (N_m-1)/2, exactly like pmf_moments does for a context
 * (mean = c + M E[u], cov = M Cov[u] M^T, weights need not be normalised).
 * If S0 is zero or not finite, out[0] = S0 and the mean and covariance are
 * written as NaN.
 *
 *   weights : device pointer, prod N_m float64 values, C-order (caller-owned)
 *   nx, N   : state dimension (1..PMF_MAX_NX) and points per axis (host)
 *   c, M    : frame centre (nx) and axes (nx*nx row-major), host float64
 *   out     : device pointer to 1 + nx + nx*nx float64: {S0, mean, cov}
 *   stream  : cudaStream_t as void* (NULL = legacy default stream)
 *
 * It calls no allocating routine.  Its block partial sums live in one fixed
 * device array of PMF_NOALLOC_MAX_POINTS / 256 * 15 float64 (480 KiB) that
 * every GPU which loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (a runtime query,
 * once per device, with the device current); later calls reuse it.  All
 * calls share the array, so calls whose kernels overlap on the GPU (different
 * streams, or other host threads) race: serialise them on one stream.  Each
 * call rewrites every partial it reads, so nothing needs clearing between
 * calls.  Asynchronous; returns PMF_ERR_ARG for null pointers, nx out of range
 * or more than PMF_NOALLOC_MAX_POINTS points, PMF_ERR_CUDA on a launch error. */
#define PMF_NOALLOC_MAX_POINTS (1 << 20)
int pmf_moments_noalloc(const double* weights, int nx, const int* N, const double* c,
                        const double* M, double* out, void* cuda_stream);

/* Self-test of the bounded device waits (no counterpart in the paper).  Every
 * wait of the tensor-core kernels on an mbarrier (bulk copies, MMA completion)
 * polls at most a fixed number of times and then records PMF_ERR_TIMEOUT in
 * the filter's status and returns, so a lost completion ends the kernel with
 * an error the host reads instead of a hung GPU.  This call runs that wait in
 * a one-warp kernel on a barrier that expects one arrival:
 *   arrive = 1 : the arrival happens before the wait; expected PMF_OK.
 *   arrive = 0 : nothing arrives; the wait gives up after `polls` polls
 *                (>= 1) and the call returns PMF_ERR_TIMEOUT.
 * Synchronous on `cuda_stream` (NULL = legacy default stream); PMF_ERR_ARG
 * for polls < 1, PMF_ERR_CUDA if the launch or the synchronisation fails (the
 * context stays usable after a timeout). */
int pmf_selftest_bounded_wait(long long polls, int arrive, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PMF_H */
