// Stand-alone 2D-DFT building blocks used outside the iteration: the PSF and
// measurement spectra at setup (Alg. 1 line 2), in the setup precision.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

constexpr int kRowThreads = 256;
#ifndef SETUP_FFT_E
#define SETUP_FFT_E 8
#endif
constexpr int kE = SETUP_FFT_E;  // FFT elements per thread in these kernels (8 measured faster than 16 for the double-float setup)

// Two real rows per complex FFT.  Each team of N/kE threads owns one row pair.
template <typename Tc, typename Tin, int LOGN>
__global__ void __launch_bounds__(kRowThreads) row_r2c_kernel(const Tin* __restrict__ in,
                                                                typename CT<Tc>::type* __restrict__ out, int nrows,
                                                                Tc scale, const typename CT<Tc>::type* tw) {
  using C = typename CT<Tc>::type;
  constexpr int N = 1 << LOGN, H = N / 2 + 1, P = half_pitch(N), ZS = spad(N), TEAM = N / kE;
  constexpr int PAIRS = kRowThreads / TEAM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* zb = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * PAIRS * 2;
  for (int idx = tid; idx < PAIRS * N; idx += kRowThreads) {
    const int p = idx / N, n = idx - p * N;
    const int ra = row0 + 2 * p, rb = ra + 1;
    const Tc xa = ra < nrows ? (Tc)in[(size_t)ra * N + n] : Tc(0);
    const Tc xb = rb < nrows ? (Tc)in[(size_t)rb * N + n] : Tc(0);
    zb[p * ZS + spad(n)] = cpack<C>(xa * scale * Tc(0.5f), xb * scale * Tc(0.5f));
  }
  __syncthreads();
  const int team = tid / TEAM;
  fft_team<C, LOGN, 1, kE, -1>(zb + team * ZS, tid % TEAM, tw, make_block_team_sync(team, TEAM));
  __syncthreads();
  for (int idx = tid; idx < PAIRS * H; idx += kRowThreads) {
    const int p = idx / H, k = idx - p * H;
    const int ra = row0 + 2 * p, rb = ra + 1;
    C qa, qb;
    pair_spectrum_get(zb + p * ZS, N, k, qa, qb);
    if (ra < nrows) out[(size_t)ra * P + k] = qa;
    if (rb < nrows) out[(size_t)rb * P + k] = qb;
  }
}

// In-place column DFT of a [N][P] half-spectrum map; CTA = 4 columns of one map.
template <typename Tc, int LOGN, int SIGN>
__global__ void col_c2c_kernel(typename CT<Tc>::type* data, const typename CT<Tc>::type* tw) {
  using C = typename CT<Tc>::type;
  constexpr int N = 1 << LOGN, H = N / 2 + 1, P = half_pitch(N), CC = 4, TEAM = N * CC / kE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* zb = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CC;
  C* map = data + (size_t)blockIdx.y * N * P;
  for (int idx = tid; idx < N * CC; idx += TEAM) {
    const int n = idx / CC, c = idx - n * CC;
    zb[spad(idx)] = (c0 + c < H) ? map[(size_t)n * P + c0 + c] : mk<C>(0.0, 0.0);
  }
  __syncthreads();
  TeamSync ts;
  ts.bar_id = 0;
  ts.nthreads = TEAM;
  ts.mask = TEAM >= 32 ? 0xffffffffu : ((1u << TEAM) - 1u);
  ts.cta = false;
  fft_team<C, LOGN, CC, kE, SIGN>(zb, tid, tw, ts);
  __syncthreads();
  for (int idx = tid; idx < N * CC; idx += TEAM) {
    const int n = idx / CC, c = idx - n * CC;
    if (c0 + c < H) map[(size_t)n * P + c0 + c] = zb[spad(idx)];
  }
}

template <typename Tc, typename Tin, int LOGN>
cudaError_t rr2c(const Tin* in, typename CT<Tc>::type* out, int nrows, Tc scale, const typename CT<Tc>::type* tw,
                 cudaStream_t s) {
  using C = typename CT<Tc>::type;
  constexpr int N = 1 << LOGN, PAIRS = kRowThreads / (N / kE);
  const size_t sm = (size_t)PAIRS * spad(N) * sizeof(C);
  auto k = row_r2c_kernel<Tc, Tin, LOGN>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int nblk = (nrows + 2 * PAIRS - 1) / (2 * PAIRS);
  k<<<nblk, kRowThreads, sm, s>>>(in, out, nrows, scale, tw);
  return cudaGetLastError();
}

template <typename Tc, int LOGN>
cudaError_t cc2c(typename CT<Tc>::type* data, int nmaps, int sign, const typename CT<Tc>::type* tw, cudaStream_t s) {
  using C = typename CT<Tc>::type;
  constexpr int N = 1 << LOGN, CC = 4, TEAM = N * CC / kE;
  const size_t sm = (size_t)spad(N * CC) * sizeof(C);
  dim3 grid((N / 2 + 1 + CC - 1) / CC, nmaps);
  if (sign < 0) {
    auto k = col_c2c_kernel<Tc, LOGN, -1>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<grid, TEAM, sm, s>>>(data, tw);
  } else {
    auto k = col_c2c_kernel<Tc, LOGN, +1>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<grid, TEAM, sm, s>>>(data, tw);
  }
  return cudaGetLastError();
}

}  // namespace

#define CIP_SWITCH_N(N, CALL)          \
  switch (N) {                         \
    case 64: { constexpr int L = 6; return CALL; }   \
    case 128: { constexpr int L = 7; return CALL; }  \
    case 256: { constexpr int L = 8; return CALL; }  \
    case 512: { constexpr int L = 9; return CALL; }  \
    case 1024: { constexpr int L = 10; return CALL; } \
    case 2048: { constexpr int L = 11; return CALL; } \
    default: return cudaErrorInvalidValue;           \
  }

template <typename Tc, typename Tin>
cudaError_t launch_row_r2c(const Tin* in, typename CT<Tc>::type* out, int N, int nrows, Tc scale,
                           const typename CT<Tc>::type* tw, cudaStream_t s) {
  CIP_SWITCH_N(N, (rr2c<Tc, Tin, L>(in, out, nrows, scale, tw, s)))
}

template <typename Tc>
cudaError_t launch_col_c2c(typename CT<Tc>::type* data, int N, int nmaps, int sign,
                           const typename CT<Tc>::type* tw, cudaStream_t s) {
  CIP_SWITCH_N(N, (cc2c<Tc, L>(data, nmaps, sign, tw, s)))
}

template cudaError_t launch_row_r2c<df64, float>(const float*, cdf*, int, int, df64, const cdf*, cudaStream_t);
template cudaError_t launch_row_r2c<df64, double>(const double*, cdf*, int, int, df64, const cdf*, cudaStream_t);
template cudaError_t launch_row_r2c<double, double>(const double*, double2*, int, int, double, const double2*,
                                                    cudaStream_t);
template cudaError_t launch_row_r2c<float, float>(const float*, float2*, int, int, float, const float2*,
                                                  cudaStream_t);
template cudaError_t launch_col_c2c<float>(float2*, int, int, int, const float2*, cudaStream_t);
template cudaError_t launch_col_c2c<double>(double2*, int, int, int, const double2*, cudaStream_t);
template cudaError_t launch_col_c2c<df64>(cdf*, int, int, int, const cdf*, cudaStream_t);

}  // namespace cip
