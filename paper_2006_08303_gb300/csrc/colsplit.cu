// Split form of the column pass (the x-update of Eq. solx_Trans_DFT, three
// kernels instead of one): a forward column DFT of q-hat into the column
// buffer, an element-wise per-frequency solve X = xb + Psi^{-1}/N^2 Q over
// that layout, and an inverse column DFT into x-hat.  It moves 16 more bytes
// per voxel than the fused kernel (colpass.cu) but needs no shared-memory tile
// of all channels; the plan's autotuner chooses between the two per shape.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

// X = xb + Pinv Q at every bin, in place on colbuf; thread = (k2, k1), k1 fastest.
// 128-thread CTAs at <= ~72 registers (complex64) keep every bin of a
// 512 x 512 x 10 problem resident in one wave; before waiting for the forward
// column DFTs, each CTA prefetches its slab of the factor and the data term
// (independent of them) into L2.
constexpr int kSolveThreads = 128;
template <typename T, int MMAX> constexpr int solve_minblocks() {
  return sizeof(T) == 4 ? (MMAX <= 12 ? 7 : 5) : 3;
}

template <typename T, int MMAX>
__global__ void __launch_bounds__(kSolveThreads, solve_minblocks<T, MMAX>())
    solve_split_kernel(typename CT<T>::type* __restrict__ colbuf, const typename CT<T>::type* __restrict__ pinv,
                       const typename CT<T>::type* __restrict__ xb, int N, int M, int plain,
                       const typename CT<T>::type* __restrict__ lowcol, const typename CT<T>::type* __restrict__ tw,
                       T rho) {
  using C = typename CT<T>::type;
  const int k1 = blockIdx.x * kSolveThreads + threadIdx.x;
  const int k2 = blockIdx.y;
  {
    // the CTA's bins [k1lo, k1lo + 128) are whole 32-bin blocks: one contiguous run of the
    // blocked factor and one of the data term
    const int npk = M * (M + 1) / 2;
    const int k1lo = blockIdx.x * kSolveThreads;
    const int cnt = min(kSolveThreads, N - k1lo);
    if (threadIdx.x == 0) prefetch_l2(pinv + binp(k2, 0, k1lo, npk, N), (size_t)cnt * npk * sizeof(C));
    if (threadIdx.x == 1) prefetch_l2(xb + binp(k2, 0, k1lo, M, N), (size_t)cnt * M * sizeof(C));
  }
  grid_dep_wait();  // the forward column DFTs are complete from here on
  grid_dep_launch();
  if (k1 >= N) return;
  const int npk = M * (M + 1) / 2;
  const int CP = col_pitch(N);
  C* col = colbuf + (size_t)k2 * M * CP + k1;
  const C* xcol = xb + binp(k2, 0, k1, M, N);      // plane stride kBinBlock
  const C* pcol = pinv + binp(k2, 0, k1, npk, N);  // plane stride kBinBlock
  C r[MMAX], x[MMAX];
  // columns k2 < kLowK of a TV plan with the low-column correction: Q from the column DFTs of the
  // components of t - u, the differences applied as spectral products
  const bool low = lowcol && k2 < kLowK;
  C dh = mk<C>(0.0, 0.0), dv = dh;
  if (low) {
    const C wh = ldg_tw(&tw[k2 * (kTwN / N)]), wv = ldg_tw(&tw[k1 * (kTwN / N)]);
    dh = mk<C>(wh.x - 1.0, -wh.y);  // exp(+2 pi i k2 / N) - 1
    dv = mk<C>(wv.x - 1.0, -wv.y);
  }
#pragma unroll
  for (int i = 0; i < MMAX; ++i) {
    if (i < M) {
      if (low) {
        C q = mk<C>(0.0, 0.0);
        cfmac(q, dh, lowcol[((size_t)k2 * M + i) * CP + k1]);
        cfmac(q, dv, lowcol[((size_t)(kLowK + k2) * M + i) * CP + k1]);
        r[i] = mk<C>(rho * q.x, rho * q.y);
      } else {
        r[i] = col[(size_t)i * CP];
      }
      x[i] = xcol[(size_t)i * kBinBlock];
      if (plain) {  // plain FP32 method: X = Pinv (b + Q)
        r[i] = cadd(r[i], x[i]);
        x[i] = mk<C>(0.0, 0.0);
      }
    }
  }
  int pk = 0;
#pragma unroll
  for (int i = 0; i < MMAX; ++i) {
    if (i < M) {
#pragma unroll
      for (int j = i; j < MMAX; ++j) {
        if (j < M) {
          const C pij = pcol[(size_t)pk * kBinBlock];
          ++pk;
          cfma(x[i], pij, r[j]);
          if (j != i) cfmac(x[j], pij, r[i]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MMAX; ++i)
    if (i < M) col[(size_t)i * CP] = x[i];
}

template <typename T>
cudaError_t solve_m(typename CT<T>::type* colbuf, const typename CT<T>::type* pinv, const typename CT<T>::type* xb,
                    int N, int M, int plain, const typename CT<T>::type* lowcol, const typename CT<T>::type* tw,
                    T rho, cudaStream_t s) {
  const dim3 grid((N + kSolveThreads - 1) / kSolveThreads, N / 2 + 1), block(kSolveThreads);
#define CIP_SOLVE(MM) \
  return launch_pdl(solve_split_kernel<T, MM>, grid, block, 0, s, 0, colbuf, pinv, xb, N, M, plain, lowcol, tw, rho)
  if (M <= 4) CIP_SOLVE(4);
  if (M <= 8) CIP_SOLVE(8);
  if (M <= 10) CIP_SOLVE(10);
  if (M <= 12) CIP_SOLVE(12);
  if (M <= 16) CIP_SOLVE(16);
#undef CIP_SOLVE
  return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
cudaError_t launch_passB_split(const PassBArgs<T>& a, typename CT<T>::type* colbuf, int N, cudaStream_t s,
                               int* launches, const typename CT<T>::type* lowbuf, typename CT<T>::type* lowcol,
                               T rho) {
  // q-hat and x-hat use the column layout already: the column DFTs need no transposition; the
  // low-column maps of the correction (2 kLowK M columns) ride along in the forward launch
  cudaError_t e = launch_cols_fft<T>(a.qh, colbuf, a.tw, N, a.M, -1, s, lowbuf, lowcol, lowbuf ? 2 * kLowK * a.M : 0);
  if (e != cudaSuccess) return e;
  e = solve_m<T>(colbuf, a.pinv, a.bhat, N, a.M, a.plain, lowbuf ? lowcol : nullptr, a.tw, rho, s);
  if (e != cudaSuccess) return e;
  e = launch_cols_fft<T>(colbuf, a.xh, a.tw, N, a.M, +1, s);
  if (launches) *launches += 3;
  return e;
}

template cudaError_t launch_passB_split<float>(const PassBArgs<float>&, float2*, int, cudaStream_t, int*,
                                               const float2*, float2*, float);
template cudaError_t launch_passB_split<double>(const PassBArgs<double>&, double2*, int, cudaStream_t, int*,
                                                const double2*, double2*, double);

}  // namespace cip
