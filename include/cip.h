/*
 * cip.h -- C ABI of a GB300 (sm_103a) library for the ADMM reconstruction of
 * convolutional inverse problems (Dogan & Oktem, "Efficient Algorithms for
 * Convolutional Inverse Problems in Multidimensional Imaging",
 * arXiv 2006.08303).
 *
 * Model (Section II, Eq. forward model): K measurements y_k, each the sum of
 * M unknown N x N channels x_m circularly convolved with known PSFs h_{k,m}:
 *     y_k = sum_m h_{k,m} (*) x_m + w_k.
 * Problem (Eq. rls): min_x beta/2 ||y - H x||^2 + R(x), R = lambda ||T x||_1
 * (analysis prior, Eq. analysis).  Solved by Alg. 1 (ADMM, splitting t = T x,
 * scaled dual u):
 *     x^{l+1} = F^H Psi^{-1} (beta Lambda^H F y + rho F T^H (t^l - u^l))   (Eq. solx_Trans_DFT)
 *     t^{l+1} = soft(T x^{l+1} + u^l, lambda / rho)                        (Eq. solt_trans)
 *     u^{l+1} = u^l + T x^{l+1} - t^{l+1}                                  (Eq. subu_trans)
 * with Psi(w) = rho g(w) I + beta Lambda(w)^H Lambda(w), g the DFT
 * eigenvalues of T^H T (g = 1 for an orthonormal T).
 *
 * Conventions for every call:
 *   - Arrays are row-major C order.  PSFs have their origin at index (0,0)
 *     and wrap circularly.  Real arrays use the plan's dtype (float32 for
 *     CIP_F32, float64 for CIP_F64).
 *   - Data pointers may be device pointers or host pointers; the library
 *     detects which (cudaPointerGetAttributes).  Host inputs are copied to a
 *     device staging buffer in stream order.  A call that writes to a host
 *     pointer synchronises the stream before returning.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous with respect to the host unless stated otherwise.
 *   - The caller owns every pointer it passes and may reuse an input buffer
 *     once the stream has passed the call.  The plan owns all spectra,
 *     factors and ADMM state until cip_plan_destroy.
 *   - Every call returns a cip_status; nothing throws across the ABI.
 *     On failure, cip_last_error(plan) returns a message (thread-safe per
 *     plan; plans must not be used from two threads at once).
 */
#ifndef CIP_H_
#define CIP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cip_status {
  CIP_OK = 0,
  CIP_ERR_INVALID_ARG = 1,  /* null pointer, size out of range, bad enum */
  CIP_ERR_UNSUPPORTED = 2,  /* N not a power of two in [64, 2048], M > 16, shape too large for a kernel */
  CIP_ERR_OOM = 3,          /* device allocation failed */
  CIP_ERR_CUDA = 4,         /* a CUDA runtime call failed (message in cip_last_error) */
  CIP_ERR_STATE = 5,        /* call out of order (e.g. iterate before set_psfs) */
  CIP_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
  CIP_ERR_DIVERGED = 7      /* residuals became NaN/Inf */
} cip_status;

typedef enum cip_dtype { CIP_F32 = 0, CIP_F64 = 1 } cip_dtype;

typedef enum cip_prior {
  CIP_PRIOR_TV = 0,   /* anisotropic TV: T = [D_h; D_v], circular forward differences (2 components) */
  CIP_PRIOR_DCT8 = 1, /* orthonormal DCT-II on 8x8 blocks aligned at (0,0) (1 component) */
  CIP_PRIOR_L1 = 2,   /* T = I (1 component) */
  CIP_PRIOR_CONVDICT = 3, /* synthesis prior with a 2D convolutional dictionary shared by all channels
                            (Alg. 2): x ~ sum_l d_l (*) z_{l,m}, l1 on the coefficient maps z */
  CIP_PRIOR_TV_ISO = 4, /* isotropic TV, lambda sum_pixels ||(D_h x, D_v x)||_2 (Section III-A): the
                          same T and x-update as CIP_PRIOR_TV, the t-update the per-pixel group
                          shrinkage (v max(0, 1 - (lambda/rho)/||v||)), 2 components */
  CIP_PRIOR_WDCT = 5   /* Kronecker basis T = W (x) C of Section V (1 component): W the periodic 2D
                          Symmlet-8 wavelet transform of each channel (orthonormal filter with 8
                          vanishing moments and the least-asymmetric root choice of Daubechies'
                          factorisation; Mallat levels, rows then columns, down to a 16 x 16 coarse
                          band), C the orthonormal DCT-II along the M channels; t and u hold the
                          coefficients [M][1][N][N] (index 0 = DCT frequency along channels, Mallat
                          layout in the plane) */
} cip_prior;

typedef struct cip_options {
  int col_tile;     /* accepted for compatibility (0, 1, 2 or 4); the fused column pass works on one
                       half-spectrum column per CTA */
  int check_every;  /* residual check period for cip_iterate with tol > 0; 0 = 10 */
  int column_pass;  /* 0 = autotuned at cip_set_measurements (fused vs split, tile width; cached per
                       N, M, dtype and prior for the process, and in the file named by the environment
                       variable CIP_TUNE_CACHE when set, one "N M dtype prior mode cc variant" line per
                       decision, read on first use), 1 = fused kernel (one CTA per half-spectrum column, factor
                       streamed by TMA bulk copies; CIP_ERR_UNSUPPORTED where its tile does not fit
                       in shared memory), 2 = split (column FFT / solve / FFT).  TV plans with
                       N >= 2048 always use the split form: it carries their low-column correction
                       (near DC the x-update takes Q from the transforms of the two components of
                       t - u, not of T^H (t - u), whose FP32 rounding Psi^{-1} amplifies) */
  int precision;    /* CIP_F32 plans: 0 = mixed (factor and data term Psi^{-1} beta Lambda^H F y formed
                       in double-float, about 44 bits, rounded once; the default), 1 = plain FP32
                       method (factor formed and
                       inverted in FP32, x = Psi^{-1} (beta Lambda^H F y + rho F T^H (t - u)) applied in
                       FP32 every iteration; analysis priors only) */
  int prior_fft;    /* FFT elements per thread of the prior pass for CIP_F32 plans with 256 <= N <= 1024
                       and the TV, isotropic TV, DCT, l1 and dictionary (l1 on the codes) priors: 0 =
                       chosen by the autotuner together
                       with the column-pass form (timing whole iterations; the default width when
                       column_pass != 0), 8 or 16 = that width; ignored for other plans */
  int reserved[11];
} cip_options;

typedef struct cip_plan cip_plan;

/* Library / status strings. */
const char* cip_version(void);
const char* cip_status_string(cip_status s);
const char* cip_last_error(const cip_plan* plan); /* plan may be NULL: last error of plan creation */

/* The wavelet lowpass filter of CIP_PRIOR_WDCT for p vanishing moments (Section V names p = 8,
 * "Symmlet-8"): writes the 2p taps h[0..2p) of the orthonormal filter from Daubechies' spectral
 * factorisation with the least-asymmetric root choice (the highpass is g_k = (-1)^k h_{2p-1-k}).
 * Host computation only (no device use).  CIP_ERR_INVALID_ARG for a null h or p outside [1, 8]. */
cip_status cip_wavelet_lowpass(int p, double* h);

/* Create a plan for N x N images, K measurements, M channels (1 <= K, M <= 16;
 * N a power of two in [64, 2048]).  Allocates all device buffers on the
 * current device.  opt may be NULL. */
cip_status cip_plan_create(cip_plan** out, int N, int K, int M, cip_dtype dtype, const cip_options* opt);
/* Same, with the plan's buffers allocated in stream order on `stream` (the stream-ordered
 * allocator); every later call allocates and frees on its own stream and cip_plan_destroy frees
 * on the stream of the plan's last call, so no call synchronises the whole device. */
cip_status cip_plan_create_on_stream(cip_plan** out, int N, int K, int M, cip_dtype dtype, const cip_options* opt,
                                     void* stream);
/* Frees the plan's buffers in stream order on the stream of its last call (which must still
 * exist); work already queued on that stream completes first. */
cip_status cip_plan_destroy(cip_plan* plan);

/* Device bytes a plan with these sizes holds (for admission by HBM budget). */
size_t cip_plan_bytes(int N, int K, int M, cip_dtype dtype, cip_prior prior);

/* Prior and ADMM weights (Alg. 1 line 1): lambda > 0, rho > 0, beta > 0.
 * Must precede cip_set_psfs; calling it again afterwards re-forms the factor
 * from the kept PSF spectra and requires cip_set_measurements again
 * (the precomputed data term depends on the factor). */
cip_status cip_set_prior(cip_plan* plan, cip_prior prior, double lambda, double rho, double beta, void* stream);

/* PSFs h[K][M][N][N] (plan dtype).  Forms Lambda = DFT2(h) and the
 * per-frequency factor Psi^{-1} (Alg. 1 line 2; Section IV-A) in the setup
 * precision -- double-float (about 44 bits, on the FP32 pipes) for CIP_F32
 * plans, FP64 for CIP_F64 plans -- kept in the plan's precision.  Resets the
 * ADMM state. */
cip_status cip_set_psfs(cip_plan* plan, const void* h, void* stream);

/* Measurements y[K][N][N] (plan dtype): the data term of the x-update,
 * Psi^{-1} beta Lambda^H F y (Alg. 1 line 2), formed in the setup precision and rounded
 * once to the plan's precision.  Resets the ADMM state (t = u = 0). */
cip_status cip_set_measurements(cip_plan* plan, const void* y, void* stream);

/* Convolutional dictionary (prior CIP_PRIOR_CONVDICT; Section III-B "Convolutional
 * Dictionary", Alg. 2): filters d[L][P][P] (plan dtype, centre at index P/2, 1 <= L <= 32),
 * embedded on the N x N torus with their centre at (0,0).  Call after
 * cip_set_prior(CIP_PRIOR_CONVDICT, lambda, rho, beta) and before cip_set_psfs.  Alg. 2 then
 * runs with x-update factor (I + beta Lambda^H Lambda)^{-1} (Eq. solx_synt_DFT, t = 1), the
 * per-frequency Sherman-Morrison z-update (Eq. solz_DFT_SM), t = soft(z + u, lambda/rho)
 * (Eq. softADMM) and u += z - t (Eq. subu_dic), from z = t = u = 0.  The ADMM variables
 * t, u and the coefficient maps z have shape [M][L][N][N] (channel-major). */
cip_status cip_set_dictionary(cip_plan* plan, const void* filters, int L, int P, void* stream);

/* Convolutional dictionary with 3D filters (Section IV-B, 3D case): filters d[L][Q][P][P] (plan
 * dtype, centre at (Q/2, P/2, P/2), 1 <= L <= 32, 1 <= Q <= M), embedded on the M x N x N torus
 * with the centre at (0,0,0) -- the convolution is circular along the channels too -- and one
 * code map of M x N x N per filter, so t, u and z keep the [M][L][N][N] shape of the 2D
 * dictionary.  Theta_l(kappa, w) is the 3D DFT of filter l (FP64-formed, rounded once); the
 * x-update keeps the 2D factor (I + beta Lambda^H Lambda)^{-1} with its last term
 * (F_1D^H (x) I) sum_l Theta_l F_3D z_l (Eq. solx_synt_DFT), and the z-update solves
 * Eq. solz_DFT_SM by Sherman-Morrison in every 3D bin (kappa, w), with M-point DFTs along the
 * channels around it.  Call after cip_set_prior(CIP_PRIOR_CONVDICT, ...) and before
 * cip_set_psfs.  Q = 1 is the 2D dictionary.  CIP_ERR_UNSUPPORTED with the code gradient
 * penalty or the online dictionary update on (both 2D only), or when M * L is too large for the
 * per-bin tile. */
cip_status cip_set_dictionary_3d(cip_plan* plan, const void* filters, int L, int Q, int P, void* stream);

/* Gradient (Tikhonov) penalty on the codes of a CIP_PRIOR_CONVDICT plan (Section III-B,
 * "Convolutional Dictionary with Tikhonov Regularization", Eq. DL_PriorHP_conv in 2D):
 * adds mu/2 sum_m (||r_1 * z_m||^2 + ||r_2 * z_m||^2), r_1, r_2 the circular differences
 * along the two image axes.  The z-update of each frequency w then solves
 * ((rho + mu g(w)) I + conj(theta) theta^T) v = c by Sherman-Morrison, g(w) = 4 sin^2(pi k1/N)
 * + 4 sin^2(pi k2/N) (the mu sum_i R_i^H R_i term noted after Eq. solz).  mu >= 0, finite;
 * 0 (the default) is plain Alg. 2.  Takes effect from the next iteration; the factor and the
 * state are unchanged.  CIP_ERR_STATE for other priors. */
cip_status cip_set_code_gradient_weight(cip_plan* plan, double mu);

/* Online convolutional dictionary update (Section IV-B, Eqs. d_admm, g_admm, h_admm with the
 * sum over channels of Eq. sold_3D) for a CIP_PRIOR_CONVDICT plan; call after
 * cip_set_dictionary.  sigma > 0 turns it on: the filters start as those given to
 * cip_set_dictionary (g = d, scaled dual e = 0, both N x N planes) and after the z-update of
 * every iteration one step of the filter ADMM runs on that iteration's x and z:
 *   d-hat(w) = (sigma I + Z(w)^H Z(w))^{-1} (Z(w)^H x-hat(w) + sigma F(g - e)(w)),
 *   g = (d + e) restricted to the P x P support, scaled to unit Frobenius norm,
 *   e <- e + d - g,
 * Z(w) the M x L matrix of code spectra; the next iteration uses theta = F g.  The filters
 * persist across cip_set_measurements and cip_reset; cip_set_dictionary starts them again.
 * sigma = 0 turns the update off (the filters learnt so far stay); a new sigma > 0 while on
 * keeps g and e.  The learnt g and e (and sigma) are part of cip_state_export's buffer while on.
 * One step is three kernel launches: e is kept as its spectrum and g on its support, so the
 * spatial values the projection needs are partial inverse DFTs at the P x P support points.
 * CIP_ERR_STATE without a dictionary, CIP_ERR_UNSUPPORTED for M > 8 or P > 32,
 * CIP_ERR_INVALID_ARG for sigma < 0 or not finite.  Enqueued on `stream`. */
cip_status cip_set_dictionary_learning(cip_plan* plan, double sigma, void* stream);

/* Adaptation of the filter ADMM's penalty sigma (Section V applies the rule of Eq. paramS to it):
 * after every check_every-th filter step of the plan (counted over all its iterations), with
 * r = ||d - g|| and s = sigma ||g - g_prev|| over all filters, sigma becomes tau sigma if
 * r > mu s, sigma / tau if s > mu r, and stays otherwise; on a change the scaled dual e is
 * multiplied by sigma_old / sigma_new (the multiplier sigma e is unchanged).  Each check reads
 * the two residual sums back and synchronises the stream.  tau = 0 turns it off;
 * CIP_ERR_INVALID_ARG unless tau > 1 and mu > 1 (finite).  Applies to cip_iterate. */
cip_status cip_set_sigma_adaptation(cip_plan* plan, double tau, double mu);

/* Current penalty sigma of the dictionary update (0 while the update is off). */
cip_status cip_get_sigma(cip_plan* plan, double* sigma);

/* Learnt filters g, filters[L][P][P] (plan dtype, centre at index P/2, host or device pointer;
 * a host copy synchronises `stream`).  CIP_ERR_STATE unless the dictionary update is on. */
cip_status cip_get_dictionary(cip_plan* plan, void* filters, void* stream);

/* Coefficient maps z[M][L][N][N] of the last z-update (CIP_PRIOR_CONVDICT only). */
cip_status cip_get_coefficients(cip_plan* plan, void* z, void* stream);

/* Set the dictionary ADMM state from z, t, u [M][L][N][N] (as after Alg. 2 line 7). */
cip_status cip_state_import_coefficients(cip_plan* plan, const void* z, const void* t, const void* u,
                                         void* stream);

/* t = u = 0 (Alg. 1 line 1 with zero initial values). */
cip_status cip_reset_state(cip_plan* plan, void* stream);

/* Adaptive penalty (Section IV-C, Eq. paramS): at each residual check of cip_iterate (every
 * check_every iterations; the checks synchronise the stream), rho becomes tau rho if the
 * primal residual ||Tx - t|| exceeds mu times the dual residual rho ||t - t_prev||, rho / tau
 * if the dual exceeds mu times the primal, and stays otherwise (the paper uses tau = 2,
 * mu = 10).  On a change the scaled dual u is multiplied by rho_old / rho_new (the multiplier
 * rho u is unchanged), the factor and the data term are formed again for the new rho (analysis
 * priors; the dictionary's x-update factor does not depend on rho), and the next update's
 * right-hand side is formed again.  tau = 0 turns adaptation off (the default); otherwise
 * tau > 1 and mu > 1.  For analysis priors call it before cip_set_measurements, which then
 * keeps the measurement spectra (K half-spectrum maps, 16 bytes per bin) for re-forming the data
 * term; CIP_ERR_STATE otherwise.  rho keeps its adapted value until cip_set_prior.  Applies to cip_iterate (not to
 * batches or the request server). */
cip_status cip_set_rho_adaptation(cip_plan* plan, double tau, double mu);

/* Current penalty rho of the plan (the adapted value when adaptation is on). */
cip_status cip_get_rho(cip_plan* plan, double* rho);

/* Run ADMM iterations (Alg. 1 lines 3-8).  tol <= 0: exactly max_iter
 * iterations.  tol > 0: stop after the first check at which both relative
 * residuals r/max(||Tx||,||t||) and s/||rho u|| (r = ||Tx - t||,
 * s = rho ||t - t_prev||, Eq. paramS quantities) are below tol; checks run
 * every check_every iterations and synchronise the stream.  iters_done may
 * be NULL.  Residuals of the last iteration are always computed. */
cip_status cip_iterate(cip_plan* plan, int max_iter, double tol, int* iters_done, void* stream);

/* x[M][N][N] of the last x-update (the inverse row DFT of the kept row
 * spectra).  Before any iteration: zeros. */
cip_status cip_get_x(cip_plan* plan, void* x, void* stream);

/* Scaled dual u[M][ncomp][N][N] (ncomp = 2 for TV, else 1). */
cip_status cip_get_u(cip_plan* plan, void* u, void* stream);

/* Relative residuals of the last iteration that computed them (synchronises).
 * Returns CIP_ERR_TIMEOUT if a kernel of the plan gave up a bounded wait for one of
 * its asynchronous copies since the last state reset (the iterate is then invalid);
 * cip_iterate with tol > 0 checks the same flag at each residual check. */
cip_status cip_get_residuals(cip_plan* plan, double* r_rel, double* s_rel);

/* Iterations run since the last reset/import. */
cip_status cip_get_iteration(cip_plan* plan, int* iteration);

/* Set the ADMM state from t, u [M][ncomp][N][N] (as after Alg. 1 line 6). */
cip_status cip_state_import(cip_plan* plan, const void* t, const void* u, void* stream);

/* Opaque checkpoint of the ADMM state (bitwise resumable): size, export, restore. */
cip_status cip_state_size(cip_plan* plan, size_t* bytes);
cip_status cip_state_export(cip_plan* plan, void* buf, void* stream);
cip_status cip_state_restore(cip_plan* plan, const void* buf, void* stream);

/* Per-kernel timing with CUDA events around every prior-pass and
 * column-pass launch of cip_iterate (0 = off, the default). */
cip_status cip_set_timing(cip_plan* plan, int on);
/* Sum of elapsed ms and launch counts since the last call (synchronises). */
cip_status cip_get_timing(cip_plan* plan, double* prior_pass_ms, int* prior_pass_n, double* column_pass_ms,
                          int* column_pass_n);

/* Test-only fault switch for the bounded device waits (no counterpart in the paper).
 * kind 1: the prior pass of CIP_PRIOR_DCT8 / CIP_PRIOR_L1 plans (at sizes whose u rows it stages
 * in shared memory by a bulk copy) arms its copy barrier for two arrivals, gives one and issues no
 * copy, then waits at most 64 polls: the wait gives up with nothing in flight, the kernel reads u
 * from global memory instead (the iterate is unchanged) and flags the plan, so that
 * cip_get_residuals (and the residual checks of cip_iterate) return CIP_ERR_TIMEOUT until the
 * next state reset.  kind 0: off (the default).  CIP_ERR_INVALID_ARG for other kinds. */
cip_status cip_set_test_fault(cip_plan* plan, int kind);

/* Number of CUDA kernels this plan has launched since creation. */
cip_status cip_get_launches(cip_plan* plan, unsigned long long* launches);

/* FFT elements per thread of the plan's prior-pass kernel (8 or 16; after cip_set_measurements
 * this is the autotuner's choice where it has one). */
cip_status cip_get_prior_fft(cip_plan* plan, int* elems_per_thread);

/* Launch configuration the plan uses (for reporting). */
cip_status cip_get_config(cip_plan* plan, int* rows_per_tile, int* col_tile, int* prior_pass_blocks,
                          int* column_pass_blocks, int* column_pass);

/* Batched launch of many independent plans (uneven N, M and prior allowed; every plan
 * set up and ready to iterate).  cip_batch_iterate runs `iters` iterations of every plan:
 * the iterations are recorded once into a CUDA graph with one branch per plan (spread
 * over `nstreams` capture streams, 0 = 8) and the graph is replayed, so the kernels of
 * small instances run side by side; the last two iterations run outside the graph and
 * compute each plan's residuals.  The batch does not own the plans; destroy it before
 * them.  Plans of a batch must not be iterated concurrently on other streams.  The graph
 * is re-recorded when a plan's buffers changed side since the last recording. */
typedef struct cip_batch cip_batch;
cip_status cip_batch_create(cip_batch** out, cip_plan* const* plans, int n, int nstreams);
cip_status cip_batch_iterate(cip_batch* batch, int iters, void* stream);
const char* cip_batch_last_error(const cip_batch* batch);
cip_status cip_batch_destroy(cip_batch* batch);

/* Request server: continuous batching of reconstructions on the current device.
 * Requests (analysis priors, float32) are queued at submit; a worker thread
 * admits them in arrival order whenever fewer than max_active are running and
 * their device memory fits hbm_budget (cached factors are evicted least recently
 * used to make room), runs each on its own stream in chunks of check_every
 * iterations ending with the relative-residual test of cip_iterate (tol), and
 * retires it when it converges or reaches max_iter: x is written to x_out and its
 * memory is released for the next request.  Running requests' kernels overlap on
 * the device.  Requests with the same nonzero psf_key and the same (N, K, M, prior,
 * rho, beta) share one factor (formed once, then copied).  h and y are copied at
 * submit; x_out must stay valid until the request is done. */
typedef struct cip_server cip_server;
typedef struct cip_request {
  int N, K, M;
  int prior;                      /* CIP_PRIOR_TV, CIP_PRIOR_TV_ISO, CIP_PRIOR_DCT8, CIP_PRIOR_L1 or CIP_PRIOR_WDCT */
  double lambda, rho, beta;
  const float* h;                 /* host [K][M][N][N] */
  const float* y;                 /* host [K][N][N] */
  float* x_out;                   /* host [M][N][N], written when the request is done */
  double tol;                     /* relative primal/dual residual stop; <= 0: run max_iter */
  int max_iter;
  unsigned long long psf_key;     /* 0 = no factor sharing */
  double rho_tau, rho_mu;         /* adaptive penalty (Eq. paramS) at every check: rho_tau > 1 and
                                     rho_mu > 1 turn it on (as cip_set_rho_adaptation), 0 = off; an
                                     adaptive request keeps its own factor (psf_key is ignored) and
                                     its setup buffers, so it holds cip_plan_bytes while it runs */
} cip_request;
typedef struct cip_result {
  int state;                      /* 0 queued, 1 running, 2 done, 3 failed, 4 cancelled */
  int status;                     /* cip_status of a failed request */
  int iterations;
  double r_rel, s_rel;            /* relative residuals at the last check */
  double t_submit, t_admit, t_done; /* seconds since the server was created */
} cip_result;
cip_status cip_server_create(cip_server** out, size_t hbm_budget, int max_active, int check_every);
cip_status cip_server_submit(cip_server* srv, const cip_request* req, unsigned long long* id);
cip_status cip_server_poll(cip_server* srv, unsigned long long id, cip_result* res);
/* Blocks until the request is done, failed or cancelled (CIP_ERR_TIMEOUT after timeout_s). */
cip_status cip_server_wait(cip_server* srv, unsigned long long id, cip_result* res, double timeout_s);
cip_status cip_server_cancel(cip_server* srv, unsigned long long id);
cip_status cip_server_stats(cip_server* srv, double* voxel_iters, int* running, int* queued, size_t* bytes_in_use,
                            int* cache_hits, int* cache_misses);
cip_status cip_server_destroy(cip_server* srv);

/* Shrinkage, dual update and residual norms of one ADMM iteration without any
 * device allocation.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory -- code recording a CUDA stream capture
 * that must not gain allocation nodes, host frameworks that hand the library
 * a fixed arena and forbid it to grow its footprint, and real-time loops in
 * which a driver allocation could stall.
 *
 * Given x[M][N][N] (an x-update's result), u_in and t_prev [M][ncomp][N][N]
 * (ncomp = 2 for TV, else 1), all DEVICE pointers of the given dtype, it
 * computes w = T x, t = soft(w + u_in, lambda/rho), u_out = u_in + w - t,
 * writes u_out (and t_out unless it is NULL; both device pointers, not
 * aliasing the inputs), and stores the relative residuals
 * {r/max(||Tx||,||t||), s/||rho u_out||}, r = ||Tx - t||,
 * s = rho ||t - t_prev||, into resid_out[2] (host or device pointer; a host
 * pointer makes the call synchronise the stream, so while `stream` is being
 * captured resid_out must be device memory: CIP_ERR_INVALID_ARG otherwise).
 * Same results as the prior pass inside cip_iterate.  Each launch's own status
 * is checked; an error the caller left pending is neither reported as this
 * call's nor cleared.
 *
 * No cudaMalloc, cudaFree or other allocating call is made.  Its scratch
 * (per-block partial sums) is a fixed static device array of 1.25 MiB that
 * every GPU loading the library holds until exit; sizes needing more than
 * 32768 blocks (impossible within N <= 2048, M <= 16) return
 * CIP_ERR_UNSUPPORTED.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current: make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents (every value a call reads is written by the
 * same call first); calls whose kernels overlap on the GPU race on it, so
 * order them on one stream. */
cip_status cip_shrink_dual_noalloc(cip_dtype dtype, cip_prior prior, int N, int M, double lambda, double rho,
                                   const void* x, const void* u_in, const void* t_prev, void* u_out, void* t_out,
                                   double* resid_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CIP_H_ */
