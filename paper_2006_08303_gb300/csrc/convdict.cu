// Convolutional-dictionary synthesis prior (Alg. 2, 2D filters shared by all
// channels), the per-frequency part of one iteration:
//   x(w)   = xb(w) + Psi^{-1}(w)/N^2 p(w),  p_m = sum_l theta_l v_{l,m}      (Eq. solx_synt_DFT)
//   c_l    = conj(theta_l) x_m + rho G_{l,m},  G = F (t - u)                 (Eq. solz_DFT)
//   v_{.,m} = (c - conj(theta) (theta^T c) / (rho_w + ||theta||^2)) / rho_w  (Eq. solz_DFT_SM)
// with rho_w = rho, or rho + mu g(w) when the codes carry the gradient (Tikhonov) penalty of
// Eq. DL_PriorHP_conv (g = |r1^|^2 + |r2^|^2, the circular differences along both axes: the
// mu sum_i R_i^H R_i term of the note after Eq. solz keeps each bin's matrix diagonal + rank one)
// where theta_l is the DFT of filter l, Psi = I + beta Lambda^H Lambda (t = 1
// in Eq. solx_synt_DFT) and p is carried from the previous iteration's v.  One
// thread owns one (frequency, channel) pair; the L coefficient spectra of the
// channel are contiguous planes in the column layout [k2][m*L + l][k1].  The
// column DFTs around it and the element-wise shrinkage on the coefficient
// maps (the l1 prior pass over L*M maps) are the analysis path's kernels.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

template <typename T, int MMAX, int LMAX>
__global__ void __launch_bounds__(128) cd_solve_kernel(CDArgs<T> a) {
  using C = typename CT<T>::type;
  const int N = a.N, M = a.M, L = a.L;
  const int CP = col_pitch(N);
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y;
  const int m = blockIdx.z;
  if (k1 >= N) return;
  const int npk = M * (M + 1) / 2;
  // All spectra here carry the inverse-DFT scale 1/N^2 (G, v, p, x, xb); the
  // stored factor is Psi^{-1}/N^2, so x = xb + N^2 (Psi^{-1}/N^2) p.
  // x_m = xb_m + sum_j P(m, j) p_j  (P Hermitian, packed upper triangle per bin)
  const C* pin = a.p_in + (size_t)k2 * M * CP + k1;
  const C* pcol = a.pinv + (size_t)k2 * npk * CP + k1;
  C acc = mk<C>(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < MMAX; ++j) {
    if (j < M) {
      const int i0 = min(m, j), j0 = max(m, j);
      const int pk = i0 * M - (i0 * (i0 - 1)) / 2 + (j0 - i0);
      const C pij = pcol[(size_t)pk * CP];
      const C pj = pin[(size_t)j * CP];
      if (m <= j) cfma(acc, pij, pj);
      else cfmac(acc, pij, pj);
    }
  }
  C x = a.xb[((size_t)k2 * M + m) * CP + k1];
  x.x += a.n2 * acc.x;
  x.y += a.n2 * acc.y;
  a.xcol[((size_t)k2 * M + m) * CP + k1] = x;
  // c_l = conj(theta_l) x + G_l ; s = theta^T c ; nrm = ||theta||^2
  C* g = a.colbuf + ((size_t)k2 * M * L + (size_t)m * L) * CP + k1;
  const C* th = a.theta + (size_t)k2 * L * CP + k1;
  C c[LMAX];
  C s = mk<C>(0.0, 0.0);
  T nrm = T(0);
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l < L) {
      const C t = th[(size_t)l * CP];
      C cl = g[(size_t)l * CP];
      cfmac(cl, t, x);
      c[l] = cl;
      cfma(s, t, cl);
      nrm += t.x * t.x + t.y * t.y;
    }
  }
  const T rho_w = a.mu == T(0) ? a.rho : a.rho + a.mu * (T)(a.gs[k1] + a.gs[k2]);
  const T inv_rho = T(1) / rho_w;
  const T den = T(1) / (rho_w + nrm);
  const C coef = mk<C>(s.x * den, s.y * den);
  C pn = mk<C>(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l < L) {
      const C t = th[(size_t)l * CP];
      C v = c[l];
      // v = (c - conj(theta) coef) / rho
      v.x -= t.x * coef.x + t.y * coef.y;
      v.y -= t.x * coef.y - t.y * coef.x;
      v.x *= inv_rho;
      v.y *= inv_rho;
      g[(size_t)l * CP] = v;
      cfma(pn, t, v);
    }
  }
  a.p_out[((size_t)k2 * M + m) * CP + k1] = pn;
}

// filters d[L][P][P] (centre P/2) placed on the N x N torus with the centre at (0,0)
template <typename Tin>
__global__ void embed_kernel(const Tin* __restrict__ d, double* __restrict__ out, int L, int P, int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * P * P) return;
  const int l = idx / (P * P), r = idx - l * P * P;
  const int i = r / P, j = r - i * P;
  const int c = P / 2;
  const int a = ((i - c) % N + N) % N, b = ((j - c) % N + N) % N;
  out[((size_t)l * N + a) * N + b] = (double)d[idx];
}

// theta from the half-pitch layout [L][N][P] (FP64) to the column layout [k2][L][CP]
template <typename T>
__global__ void theta_store_kernel(const SetupC<T>* __restrict__ th64, typename CT<T>::type* __restrict__ th, int L,
                                   int N) {
  using C = typename CT<T>::type;
  const int H = N / 2 + 1, P = half_pitch(N), CP = col_pitch(N);
  const size_t total = (size_t)L * N * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % N);
    const size_t r = i / N;
    const int l = (int)(r % L);
    const int k2 = (int)(r / L);
    th[((size_t)k2 * L + l) * CP + k1] = cconv<C>(th64[((size_t)l * N + k1) * P + k2]);
  }
}

// p_m = sum_l theta_l Z_{m,l} / N^2 from the column spectra Z of imported coefficient maps
template <typename T>
__global__ void p_from_z_kernel(const typename CT<T>::type* __restrict__ zcol, const typename CT<T>::type* __restrict__ th,
                                typename CT<T>::type* __restrict__ p, int N, int M, int L) {
  using C = typename CT<T>::type;
  const int CP = col_pitch(N);
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y, m = blockIdx.z;
  if (k1 >= N) return;
  const T s = T(1) / ((T)N * (T)N);
  C acc = mk<C>(0.0, 0.0);
  for (int l = 0; l < L; ++l)
    cfma(acc, th[((size_t)k2 * L + l) * CP + k1], zcol[((size_t)k2 * M * L + (size_t)m * L + l) * CP + k1]);
  p[((size_t)k2 * M + m) * CP + k1] = mk<C>(acc.x * s, acc.y * s);
}

}  // namespace

template <typename T>
cudaError_t launch_p_from_z(const typename CT<T>::type* zcol, const typename CT<T>::type* th,
                            typename CT<T>::type* p, int N, int M, int L, cudaStream_t s) {
  dim3 grid((N + 127) / 128, N / 2 + 1, M);
  p_from_z_kernel<T><<<grid, 128, 0, s>>>(zcol, th, p, N, M, L);
  return cudaGetLastError();
}
template cudaError_t launch_p_from_z<float>(const float2*, const float2*, float2*, int, int, int, cudaStream_t);
template cudaError_t launch_p_from_z<double>(const double2*, const double2*, double2*, int, int, int, cudaStream_t);

template <typename T> cudaError_t launch_cd_solve(const CDArgs<T>& a, cudaStream_t s) {
  dim3 grid((a.N + 127) / 128, a.N / 2 + 1, a.M);
  if (a.L > 32) return cudaErrorInvalidValue;
  if (a.M <= 4) {
    if (a.L <= 8) cd_solve_kernel<T, 4, 8><<<grid, 128, 0, s>>>(a);
    else cd_solve_kernel<T, 4, 32><<<grid, 128, 0, s>>>(a);
  } else if (a.M <= 16) {
    if (a.L <= 8) cd_solve_kernel<T, 16, 8><<<grid, 128, 0, s>>>(a);
    else cd_solve_kernel<T, 16, 32><<<grid, 128, 0, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Tin>
cudaError_t launch_embed_filters(const Tin* d, double* out, int L, int P, int N, cudaStream_t s) {
  const int n = L * P * P;
  embed_kernel<Tin><<<(n + 255) / 256, 256, 0, s>>>(d, out, L, P, N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_theta_store(const SetupC<T>* th64, typename CT<T>::type* th, int L, int N, cudaStream_t s) {
  theta_store_kernel<T><<<512, 256, 0, s>>>(th64, th, L, N);
  return cudaGetLastError();
}

template cudaError_t launch_cd_solve<float>(const CDArgs<float>&, cudaStream_t);
template cudaError_t launch_cd_solve<double>(const CDArgs<double>&, cudaStream_t);
template cudaError_t launch_embed_filters<float>(const float*, double*, int, int, int, cudaStream_t);
template cudaError_t launch_embed_filters<double>(const double*, double*, int, int, int, cudaStream_t);
template cudaError_t launch_theta_store<float>(const cdf*, float2*, int, int, cudaStream_t);
template cudaError_t launch_theta_store<double>(const double2*, double2*, int, int, cudaStream_t);

}  // namespace cip
