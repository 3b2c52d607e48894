// cip_shrink_dual_noalloc: the shrinkage, dual update and residual norms of
// one ADMM iteration, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA stream
// capture that must not add allocation nodes, host frameworks that hand out
// fixed device arenas and forbid the library from growing its footprint, and
// real-time loops where an allocation could stall on the driver.  This entry
// point works on buffers the caller already owns.  The only memory it needs
// besides them, the per-block partial sums of the residual norms and the
// reduced result, lives in a file-scope __device__ array of fixed size
// (kScratchBlocks * kNPart + 8 doubles, 1.25 MiB) that every GPU which loads
// the library holds until the process exits.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents.  Each call overwrites every partial it later reads, so
// nothing needs clearing, but two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <mutex>

#include "../../include/cip.h"
#include "kernels.h"

namespace cip {
namespace {

constexpr int kScratchBlocks = 32768;  // enough for M * N^2 <= 16 * 2048^2 at 2048 pixels per block
constexpr int kPixPerBlock = 2048;     // TV / l1: 256 threads x 8 pixels
constexpr int kThreads = 256;

__device__ __align__(256) double g_scratch[kScratchBlocks * kNPart + 8];

std::mutex g_mu;
double* g_scratch_dev[64] = {nullptr};  // per device ordinal, device address of g_scratch

template <typename T>
__device__ __forceinline__ void accumulate(T (&p)[kNPart], T w, T t, T un, T tp) {
  // per-thread sums (at most 64 terms) in the working precision; block and grid sums in double
  const T r = w - t, d = t - tp;
  p[0] = fma(r, r, p[0]);
  p[1] = fma(w, w, p[1]);
  p[2] = fma(t, t, p[2]);
  p[3] = fma(un, un, p[3]);
  p[4] = fma(d, d, p[4]);
}

template <typename T>
__device__ void block_store(const T (&v)[kNPart], double* out) {
  __shared__ double red[kThreads / 32][kNPart];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kNPart; ++i) {
    double x = (double)v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kNPart; ++i) {
      double acc = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) acc += red[w][i];
      out[(size_t)blockIdx.x * kNPart + i] = acc;
    }
  }
}

// TV and l1: element-wise over the flattened [M][N][N] image, 8 pixels per thread.
template <typename T, int PRIOR>
__global__ void __launch_bounds__(kThreads) shrink_dual_px(const T* __restrict__ x, const T* __restrict__ u_in,
                                                          const T* __restrict__ t_prev, T* __restrict__ u_out,
                                                          T* __restrict__ t_out, int N, int M, T tau,
                                                          double* partials) {
  constexpr int NC = PRIOR == PRIOR_TV ? 2 : 1;
  const size_t plane = (size_t)N * N;
  const size_t total = (size_t)M * plane;
  T part[kNPart] = {T(0), T(0), T(0), T(0), T(0)};
  for (int e = 0; e < kPixPerBlock / kThreads; ++e) {
    const size_t idx = (size_t)blockIdx.x * kPixPerBlock + (size_t)e * kThreads + threadIdx.x;
    if (idx >= total) break;
    const size_t m = idx / plane, pix = idx - m * plane;
    const int r = (int)(pix / N), c = (int)(pix - (size_t)r * N);
    const T* xm = x + m * plane;
    const T x0 = xm[pix];
    T w[NC];
    if (PRIOR == PRIOR_TV) {
      w[0] = xm[(size_t)r * N + ((c + 1) & (N - 1))] - x0;
      w[NC - 1] = xm[(size_t)((r + 1) & (N - 1)) * N + c] - x0;
    } else {
      w[0] = x0;
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const size_t g = (m * NC + k) * plane + pix;
      const T u = u_in[g];
      const T t = soft(w[k] + u, tau);
      const T un = u + w[k] - t;
      u_out[g] = un;
      if (t_out) t_out[g] = t;
      accumulate(part, w[k], t, un, t_prev[g]);
    }
  }
  block_store<T>(part, partials);
}

// 8x8 block DCT: one thread per 8x8 block, 256 blocks per CTA.
template <typename T>
__global__ void __launch_bounds__(kThreads) shrink_dual_dct(const T* __restrict__ x, const T* __restrict__ u_in,
                                                           const T* __restrict__ t_prev, T* __restrict__ u_out,
                                                           T* __restrict__ t_out, int N, int M, T tau,
                                                           const PassAArgs<T> dctsrc, double* partials) {
  const size_t plane = (size_t)N * N;
  const int nb = N / 8;
  const size_t nblocks = (size_t)M * nb * nb;
  const size_t b = (size_t)blockIdx.x * kThreads + threadIdx.x;
  T part[kNPart] = {T(0), T(0), T(0), T(0), T(0)};
  if (b < nblocks) {
    const size_t m = b / ((size_t)nb * nb);
    const int rem = (int)(b - m * nb * nb);
    const int br = rem / nb, bc = rem - br * nb;
    const T* d = dctsrc.dct;
    T v[8][8], tmp[8][8];
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) v[i][j] = x[m * plane + (size_t)(br * 8 + i) * N + bc * 8 + j];
    // W = C V C^T
    for (int i = 0; i < 8; ++i)
      for (int k = 0; k < 8; ++k) {
        T acc = T(0);
        for (int j = 0; j < 8; ++j) acc = fma(d[k * 8 + j], v[i][j], acc);
        tmp[i][k] = acc;
      }
    for (int k = 0; k < 8; ++k)
      for (int j = 0; j < 8; ++j) {
        T acc = T(0);
        for (int i = 0; i < 8; ++i) acc = fma(d[k * 8 + i], tmp[i][j], acc);
        const size_t g = m * plane + (size_t)(br * 8 + k) * N + bc * 8 + j;
        const T u = u_in[g];
        const T t = soft(acc + u, tau);
        const T un = u + acc - t;
        u_out[g] = un;
        if (t_out) t_out[g] = t;
        accumulate(part, acc, t, un, t_prev[g]);
      }
  }
  block_store<T>(part, partials);
}

// Device address of g_scratch on the current device, looked up once per device.
cip_status scratch_ptr(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CIP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return CIP_ERR_CUDA;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return CIP_OK;
}

template <typename T>
cip_status run(int prior, int N, int M, double lambda, double rho, const void* x, const void* u_in,
               const void* t_prev, void* u_out, void* t_out, double* resid_out, cudaStream_t s) {
  double* scratch = nullptr;
  cip_status st = scratch_ptr(&scratch);
  if (st != CIP_OK) return st;
  const T tau = (T)(lambda / rho);
  // Under stream capture only device memory can receive the residuals: a copy to pageable host
  // memory and the stream synchronisation it needs would invalidate the caller's capture.
  cudaPointerAttributes at;
  const bool dev_out = cudaPointerGetAttributes(&at, resid_out) == cudaSuccess &&
                       (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return CIP_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone && !dev_out) return CIP_ERR_INVALID_ARG;
  // every launch below reports its own status (no cudaGetLastError: an error the caller left
  // pending is neither taken for this call's nor cleared)
  int nblk = 0;
  cudaError_t e = cudaSuccess;
  if (prior == PRIOR_DCT8) {
    const size_t nb8 = (size_t)M * (N / 8) * (N / 8);
    nblk = (int)((nb8 + kThreads - 1) / kThreads);
    PassAArgs<T> d{};
    for (int k = 0; k < 8; ++k)
      for (int n = 0; n < 8; ++n) {
        const double a = k == 0 ? sqrt(1.0 / 8.0) : sqrt(2.0 / 8.0);
        d.dct[k * 8 + n] = (T)(a * cos(M_PI * (2 * n + 1) * k / 16.0));
      }
    e = launch_plain(shrink_dual_dct<T>, dim3(nblk), dim3(kThreads), 0, s, (const T*)x, (const T*)u_in,
                     (const T*)t_prev, (T*)u_out, (T*)t_out, N, M, tau, d, scratch);
  } else {
    const size_t total = (size_t)M * N * N;
    nblk = (int)((total + kPixPerBlock - 1) / kPixPerBlock);
    if (prior == PRIOR_TV)
      e = launch_plain(shrink_dual_px<T, PRIOR_TV>, dim3(nblk), dim3(kThreads), 0, s, (const T*)x, (const T*)u_in,
                       (const T*)t_prev, (T*)u_out, (T*)t_out, N, M, tau, scratch);
    else
      e = launch_plain(shrink_dual_px<T, PRIOR_L1>, dim3(nblk), dim3(kThreads), 0, s, (const T*)x, (const T*)u_in,
                       (const T*)t_prev, (T*)u_out, (T*)t_out, N, M, tau, scratch);
  }
  if (e != cudaSuccess) return CIP_ERR_CUDA;
  double* result = scratch + (size_t)kScratchBlocks * kNPart;
  if (launch_reduce_partials(scratch, nblk, rho, 0.0, result, nullptr, s) != cudaSuccess) return CIP_ERR_CUDA;
  if (cudaMemcpyAsync(resid_out, result + kNPart, 2 * sizeof(double),
                      dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIP_ERR_CUDA;
  if (!dev_out && cudaStreamSynchronize(s) != cudaSuccess) return CIP_ERR_CUDA;
  return CIP_OK;
}

}  // namespace
}  // namespace cip

extern "C" cip_status cip_shrink_dual_noalloc(cip_dtype dtype, cip_prior prior, int N, int M, double lambda,
                                              double rho, const void* x, const void* u_in, const void* t_prev,
                                              void* u_out, void* t_out, double* resid_out, void* stream) {
  using namespace cip;
  if (!x || !u_in || !t_prev || !u_out || !resid_out) return CIP_ERR_INVALID_ARG;
  if (N < 64 || N > 2048 || (N & (N - 1)) != 0 || M < 1 || M > 16) return CIP_ERR_UNSUPPORTED;
  if (prior != CIP_PRIOR_TV && prior != CIP_PRIOR_DCT8 && prior != CIP_PRIOR_L1) return CIP_ERR_INVALID_ARG;
  if (!(lambda > 0) || !(rho > 0)) return CIP_ERR_INVALID_ARG;
  // block counts for the largest sizes stay within the static scratch
  const size_t need = prior == CIP_PRIOR_DCT8 ? ((size_t)M * (N / 8) * (N / 8) + kThreads - 1) / kThreads
                                              : ((size_t)M * N * N + kPixPerBlock - 1) / kPixPerBlock;
  if (need > (size_t)kScratchBlocks) return CIP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CIP_F32) return run<float>(prior, N, M, lambda, rho, x, u_in, t_prev, u_out, t_out, resid_out, s);
  if (dtype == CIP_F64) return run<double>(prior, N, M, lambda, rho, x, u_in, t_prev, u_out, t_out, resid_out, s);
  return CIP_ERR_INVALID_ARG;
}
