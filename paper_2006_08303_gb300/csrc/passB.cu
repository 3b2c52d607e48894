// Pass B: column DFT, per-frequency solve and inverse column DFT, fused
// (the x-update of Eq. solx_Trans_DFT / Eq. solx_synt_DFT).
//
// One CTA owns CC adjacent half-spectrum columns k2 of every channel.  It
// stages the M x N x CC tile in shared memory, runs the forward column DFTs
// (CC interleaved FFTs per channel, one thread team per channel), then for
// every frequency (k1, k2) of the tile reads the M channel values once,
// applies the packed Hermitian M x M matrix Psi^{-1}(w) / N^2 to Q(w) and
// adds the FP64-formed data term xb(w) = Psi^{-1} beta Lambda^H F y / N^2
// (the same x-update by linearity, without rounding the ill-conditioned
// product every iteration), and finally runs the inverse column DFTs and
// writes the row-domain half spectra of the new x.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

constexpr int kE = 16;  // FFT elements per thread

template <typename T> int cols_for(int N, int M) {
  using C = typename CT<T>::type;
  // widest tile whose smem stays within 2 CTAs per SM, and at least 1
  for (int cc = 4; cc >= 1; cc /= 2) {
    size_t sm = (size_t)M * spad(N * cc) * sizeof(C);
    if (sm <= 110 * 1024) return cc;
  }
  return 1;
}

template <typename T, int LOGN, int CC, int MMAX>
__global__ void __launch_bounds__(512) passB_kernel(const PassBArgs<T> a) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int P = half_pitch(N);
  constexpr int ZS = spad(N * CC);
  constexpr int TEAM = N * CC / kE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* data = reinterpret_cast<C*>(smem_raw);
  const int M = a.M;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int c0 = blockIdx.x * CC;
  const size_t mplane = (size_t)N * P;

  // load q-hat tile: [m][n1][c]
  for (int idx = tid; idx < M * N * CC; idx += nth) {
    const int m = idx / (N * CC);
    const int rem = idx - m * (N * CC);
    const int n1 = rem / CC, c = rem - n1 * CC;
    const int k2 = c0 + c;
    C v = mk<C>(0.0, 0.0);
    if (k2 < H) v = a.qh[m * mplane + (size_t)n1 * P + k2];
    data[m * ZS + spad(rem)] = v;
  }
  __syncthreads();
  const int nteams = nth / TEAM;
  const int team = tid / TEAM;
  if (team < nteams) {
    const TeamSync ts = make_team_sync(team, TEAM);
    for (int m = team; m < M; m += nteams) fft_team<C, LOGN, CC, kE, -1>(data + m * ZS, tid % TEAM, a.tw, ts);
  }
  __syncthreads();

  // per-frequency solve: x = xb + Pinv Q
  for (int idx = tid; idx < N * CC; idx += nth) {
    const int k1 = idx / CC, c = idx - k1 * CC;
    const int k2 = c0 + c;
    if (k2 >= H) continue;
    const size_t off = (size_t)k1 * P + k2;
    C r[MMAX], x[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i) {
      if (i < M) {
        r[i] = data[i * ZS + spad(idx)];
        x[i] = a.bhat[i * mplane + off];
      }
    }
    int pk = 0;
#pragma unroll
    for (int i = 0; i < MMAX; ++i) {
      if (i < M) {
#pragma unroll
        for (int j = i; j < MMAX; ++j) {
          if (j < M) {
            const C pij = a.pinv[(size_t)pk * mplane + off];
            ++pk;
            cfma(x[i], pij, r[j]);
            if (j != i) cfmac(x[j], pij, r[i]);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < M) data[i * ZS + spad(idx)] = x[i];
  }
  __syncthreads();
  if (team < nteams) {
    const TeamSync ts = make_team_sync(team, TEAM);
    for (int m = team; m < M; m += nteams) fft_team<C, LOGN, CC, kE, +1>(data + m * ZS, tid % TEAM, a.tw, ts);
  }
  __syncthreads();
  for (int idx = tid; idx < M * N * CC; idx += nth) {
    const int m = idx / (N * CC);
    const int rem = idx - m * (N * CC);
    const int n1 = rem / CC, c = rem - n1 * CC;
    const int k2 = c0 + c;
    if (k2 < H) a.xh[m * mplane + (size_t)n1 * P + k2] = data[m * ZS + spad(rem)];
  }
}

template <typename T, int LOGN, int CC, int MMAX>
cudaError_t launchB(const PassBArgs<T>& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  constexpr int TEAM = N * CC / kE;
  using C = typename CT<T>::type;
  // teams: as many channels in parallel as fit in 512 threads / 15 named barriers,
  // balanced so every team runs the same number of channel FFTs
  int maxteams = 512 / TEAM;
  if (maxteams > 15) maxteams = 15;
  if (maxteams < 1) maxteams = 1;
  const int rounds = (a.M + maxteams - 1) / maxteams;
  const int nteams = (a.M + rounds - 1) / rounds;
  int nth = nteams * TEAM;
  if (nth < 128) nth = 128;
  nth = ((nth + 31) / 32) * 32;
  const size_t sm = (size_t)a.M * spad(N * CC) * sizeof(C);
  auto kern = passB_kernel<T, LOGN, CC, MMAX>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int ntiles = (N / 2 + 1 + CC - 1) / CC;
  kern<<<ntiles, nth, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LOGN, int CC>
cudaError_t dispatchB_m(const PassBArgs<T>& a, cudaStream_t s) {
  if (a.M <= 4) return launchB<T, LOGN, CC, 4>(a, s);
  if (a.M <= 16) return launchB<T, LOGN, CC, 16>(a, s);
  return cudaErrorInvalidValue;
}

template <typename T, int LOGN>
cudaError_t dispatchB_c(const PassBArgs<T>& a, int cc, cudaStream_t s) {
  switch (cc) {
    case 1: return dispatchB_m<T, LOGN, 1>(a, s);
    case 2: return dispatchB_m<T, LOGN, 2>(a, s);
    case 4: return dispatchB_m<T, LOGN, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T> int passB_cols(int N, int M) { return cols_for<T>(N, M); }
template <typename T> size_t passB_smem(int N, int M, int cc) {
  return (size_t)M * spad(N * cc) * sizeof(typename CT<T>::type);
}

template <typename T> cudaError_t launch_passB(const PassBArgs<T>& a, int N, int cc, cudaStream_t s) {
  switch (N) {
    case 64: return dispatchB_c<T, 6>(a, cc, s);
    case 128: return dispatchB_c<T, 7>(a, cc, s);
    case 256: return dispatchB_c<T, 8>(a, cc, s);
    case 512: return dispatchB_c<T, 9>(a, cc, s);
    case 1024: return dispatchB_c<T, 10>(a, cc, s);
    case 2048: return dispatchB_c<T, 11>(a, cc, s);
    default: return cudaErrorInvalidValue;
  }
}

template int passB_cols<PASSB_T>(int, int);
template size_t passB_smem<PASSB_T>(int, int, int);
template cudaError_t launch_passB<PASSB_T>(const PassBArgs<PASSB_T>&, int, int, cudaStream_t);

}  // namespace cip
