// Internal plan operations used by the request server (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/cip.h"

namespace cip {

// Enqueue k >= 1 iterations on s with no host synchronisation: t is kept before
// the last iteration, the last one computes the residuals, whose relative
// values {r_rel, s_rel} are copied to host_resid[2] (pinned), then ev is recorded.
cip_status plan_iterate_async(cip_plan* p, int k, cudaStream_t s, double* host_resid, cudaEvent_t ev);

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
