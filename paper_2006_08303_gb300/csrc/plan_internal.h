// Internal plan operations used by the request server (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/cip.h"

namespace cip {

// Doubles plan_iterate_async writes to host_resid: the five residual sums of squares
// (||Tx - t||^2, ||Tx||^2, ||t||^2, ||u||^2, ||t - t_prev||^2), then {r_rel, s_rel}.
constexpr int kResidHost = 7;

// Enqueue k >= 1 iterations on s with no host synchronisation: t is kept before
// the last iteration and on it, the last one computes the residuals, which are copied to
// host_resid[kResidHost] (pinned), then ev is recorded.
cip_status plan_iterate_async(cip_plan* p, int k, cudaStream_t s, double* host_resid, cudaEvent_t ev);

// The adaptive-penalty rule of Eq. paramS (as in cip_iterate) on the sums host_resid of the
// check just completed: on a change of rho, the scaled dual is rescaled and the factor, the data
// term and q are formed again on s.  The plan needs cip_set_rho_adaptation before
// cip_set_measurements and its setup buffers (no plan_trim).
cip_status plan_adapt_rho(cip_plan* p, const double* host_resid, cudaStream_t s);

// Give dst the factor of src (same N, K, M, dtype, prior, rho, beta, precision):
// a device copy of the packed factor; dst's next cip_set_measurements forms its
// data term from src's kept FP64 spectra (src must stay alive until then).
cip_status plan_adopt_factor(cip_plan* dst, const cip_plan* src, cudaStream_t s);

// Release the buffers only setup needs (FP64 PSF spectra and FP64 factor copy)
// once the data term is formed; the plan keeps iterating.
cip_status plan_trim(cip_plan* p);

// Device bytes of a trimmed plan (what stays resident while it iterates).
size_t plan_resident_bytes(int N, int K, int M, cip_dtype dtype, cip_prior prior);

}  // namespace cip
