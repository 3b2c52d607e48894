// Convolutional dictionary with 3D filters (Section IV-B, 3D case): L filters of Q x P x P taps
// (Q <= M, circular along the channels as well, reading R27) and one M x N x N code map per
// filter (R28).  The 3D DFT F_3D = F_1D (x) F_2D diagonalises the dictionary, so per 2D frequency
// w (the 2D spectra carry the inverse-DFT scale 1/N^2 as in the 2D dictionary path):
//   x-update (Eq. solx_synt_DFT):  x_s(w) = xb_s(w) + Psi^{-1}(w)/N^2 p_s(w),
//       p_s = (1/M) sum_kappa e^{+2 pi i s kappa / M} sum_l Theta_l(kappa, w) v_l(kappa, w),
//     i.e. the last term (F_1D^H (x) I) sum_l Theta_l F_3D z_l of the paper, carried from the
//     previous iteration's v;
//   z-update (Eqs. solz_DFT, solz_DFT_SM in every 3D bin):
//       X(kappa) = sum_s e^{-2 pi i kappa s / M} x_s,   G_l(kappa) = sum_m e^{-2 pi i kappa m / M} G_{m,l},
//       c_l = conj(Theta_l(kappa)) X(kappa) + G_l(kappa),   G = F_2D rho (t - u) / N^2,
//       v = (c - conj(Theta) (Theta^T c) / (rho + ||Theta||^2)) / rho   (Sherman-Morrison, R10),
//       V_{m,l} = (1/M) sum_kappa e^{+2 pi i m kappa / M} v_l(kappa)     (back to channels).
// One CTA holds BB bins of one column k2 and all M channel frequencies: thread (b, kappa) owns
// one 3D bin; the M-point DFTs along the channels go through shared memory.  The channel-domain
// spectra stay in the 2D dictionary's layout ([k2][m*L + l][k1]), so the column DFTs around the
// solve and the l1 pass on the code maps are the 2D path's kernels.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

// bins per CTA: the shared tile [M][L][BB] complex stays within ~96 KB
template <typename T> int cd3_bins(int M, int L) {
  const size_t per = (size_t)M * L * sizeof(typename CT<T>::type);
  if (32 * per <= 96 * 1024) return 32;
  if (16 * per <= 96 * 1024) return 16;
  return 8;
}

template <typename T, int LMAX>
__global__ void __launch_bounds__(512) cd3_solve_kernel(CD3Args<T> a) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, M = a.M, L = a.L, BB = blockDim.x;
  const int CP = col_pitch(N);
  const int b = threadIdx.x, m = threadIdx.y;  // m: channel index, then channel frequency kappa
  const int k1 = blockIdx.x * BB + b, k2 = blockIdx.y;
  C* gs = reinterpret_cast<C*>(smem_raw);            // [M][L][BB]: G, then v
  C* xs = gs + (size_t)M * L * BB;                    // [M][BB]: x, then p3
  C* wt = xs + (size_t)M * BB;                        // [M][M]: e^{-2 pi i k m / M} (symmetric in k, m)
  const int npk = M * (M + 1) / 2;
  for (int i = m * BB + b; i < M * M; i += M * BB) wt[i] = a.w[((i / M) * (i % M)) % M];
  // 1. G of channel m, and the channel's x-update (as in the 2D dictionary: p from the previous v)
  C* gcol = a.colbuf + ((size_t)k2 * M * L + (size_t)m * L) * CP + k1;
  for (int l = 0; l < L; ++l) gs[((size_t)m * L + l) * BB + b] = gcol[(size_t)l * CP];
  {
    const C* pin = a.p_in + (size_t)k2 * M * CP + k1;
    const C* pcol = a.pinv + binp(k2, 0, k1, npk, N);  // plane stride kBinBlock
    C acc = mk<C>(0.0, 0.0);
    for (int j = 0; j < M; ++j) {
      const int i0 = min(m, j), j0 = max(m, j);
      const int pk = i0 * M - (i0 * (i0 - 1)) / 2 + (j0 - i0);
      const C pij = pcol[(size_t)pk * kBinBlock];
      const C pj = pin[(size_t)j * CP];
      if (m <= j) cfma(acc, pij, pj);
      else cfmac(acc, pij, pj);
    }
    C x = a.xb[binp(k2, m, k1, M, N)];
    x.x += a.n2 * acc.x;
    x.y += a.n2 * acc.y;
    a.xcol[((size_t)k2 * M + m) * CP + k1] = x;
    xs[(size_t)m * BB + b] = x;
  }
  __syncthreads();
  // 2. thread (b, kappa = m): DFTs along the channels, Sherman-Morrison in the 3D bin
  const int kap = m;
  C X = mk<C>(0.0, 0.0);
  const C* wk = wt + (size_t)kap * M;  // the same row for the whole warp (one kappa per warp row)
  for (int s = 0; s < M; ++s) cfma(X, wk[s], xs[(size_t)s * BB + b]);
  const C* th = a.theta + ((size_t)k2 * M * L + (size_t)kap * L) * CP + k1;
  C c[LMAX];
  C sdot = mk<C>(0.0, 0.0);
  T nrm = T(0);
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l < L) {
      C g = mk<C>(0.0, 0.0);
      for (int mm = 0; mm < M; ++mm) cfma(g, wk[mm], gs[((size_t)mm * L + l) * BB + b]);
      const C t = th[(size_t)l * CP];
      cfmac(g, t, X);
      c[l] = g;
      cfma(sdot, t, g);
      nrm += t.x * t.x + t.y * t.y;
    }
  }
  const T inv_rho = T(1) / a.rho;
  const T den = T(1) / (a.rho + nrm);
  const C coef = mk<C>(sdot.x * den, sdot.y * den);
  C p3 = mk<C>(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l < L) {
      const C t = th[(size_t)l * CP];
      C v = c[l];
      v.x -= t.x * coef.x + t.y * coef.y;
      v.y -= t.x * coef.y - t.y * coef.x;
      v.x *= inv_rho;
      v.y *= inv_rho;
      c[l] = v;
      cfma(p3, t, v);
    }
  }
  __syncthreads();  // every thread has read G and x
#pragma unroll
  for (int l = 0; l < LMAX; ++l)
    if (l < L) gs[((size_t)kap * L + l) * BB + b] = c[l];
  xs[(size_t)kap * BB + b] = p3;
  __syncthreads();
  // 3. thread (b, m): back to the channels (inverse DFT along kappa, 1/M)
  const T invM = T(1) / (T)M;
  C p = mk<C>(0.0, 0.0);
  const C* wm = wt + (size_t)m * M;
  for (int k = 0; k < M; ++k) cfmac(p, wm[k], xs[(size_t)k * BB + b]);
  a.p_out[((size_t)k2 * M + m) * CP + k1] = mk<C>(p.x * invM, p.y * invM);
  for (int l = 0; l < L; ++l) {
    C v = mk<C>(0.0, 0.0);
    for (int k = 0; k < M; ++k) cfmac(v, wm[k], gs[((size_t)k * L + l) * BB + b]);
    gcol[(size_t)l * CP] = mk<C>(v.x * invM, v.y * invM);
  }
}

// p_s = (1/M) sum_kappa e^{+2 pi i s kappa/M} sum_l Theta_l(kappa) sum_m e^{-2 pi i kappa m/M} Z_{m,l},
// scaled by `sc`, from the 2D column spectra Z of imported code maps
template <typename T, int LMAX>
__global__ void __launch_bounds__(512) p3_from_z_kernel(const typename CT<T>::type* __restrict__ zcol,
                                                        const typename CT<T>::type* __restrict__ th3,
                                                        typename CT<T>::type* __restrict__ p, CD3Args<T> a, T sc) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, M = a.M, L = a.L, BB = blockDim.x;
  const int CP = col_pitch(N);
  const int b = threadIdx.x, m = threadIdx.y;
  const int k1 = blockIdx.x * BB + b, k2 = blockIdx.y;
  C* zs = reinterpret_cast<C*>(smem_raw);  // [M][L][BB]
  C* qs = zs + (size_t)M * L * BB;         // [M][BB]
  for (int l = 0; l < L; ++l)
    zs[((size_t)m * L + l) * BB + b] = zcol[((size_t)k2 * M * L + (size_t)m * L + l) * CP + k1];
  __syncthreads();
  const int kap = m;
  C q = mk<C>(0.0, 0.0);
  for (int l = 0; l < L; ++l) {
    C z3 = mk<C>(0.0, 0.0);
    for (int mm = 0; mm < M; ++mm) cfma(z3, a.w[(kap * mm) % M], zs[((size_t)mm * L + l) * BB + b]);
    cfma(q, th3[((size_t)k2 * M * L + (size_t)kap * L + l) * CP + k1], z3);
  }
  qs[(size_t)kap * BB + b] = q;
  __syncthreads();
  C r = mk<C>(0.0, 0.0);
  for (int k = 0; k < M; ++k) cfmac(r, a.w[(k * m) % M], qs[(size_t)k * BB + b]);
  const T s = sc / (T)M;
  p[((size_t)k2 * M + m) * CP + k1] = mk<C>(r.x * s, r.y * s);
}

// Q x P x P filters (centre (Q/2, P/2, P/2)) placed on the M x N x N torus with the centre at
// (0, 0, 0): out[l][(q - Q/2) mod M][(i - P/2) mod N][(j - P/2) mod N] = d[l][q][i][j]
template <typename Tin>
__global__ void embed3_kernel(const Tin* __restrict__ d, double* __restrict__ out, int L, int Q, int P, int M,
                              int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * Q * P * P) return;
  const int l = idx / (Q * P * P), r = idx - l * Q * P * P;
  const int q = r / (P * P), r2 = r - q * P * P;
  const int i = r2 / P, j = r2 - i * P;
  const int s = ((q - Q / 2) % M + M) % M;
  const int a0 = ((i - P / 2) % N + N) % N, b0 = ((j - P / 2) % N + N) % N;
  out[(((size_t)l * M + s) * N + a0) * N + b0] = (double)d[idx];
}

// Theta_l(kappa, w) = sum_m e^{-2 pi i kappa m/M} F_2D(filter l, channel m)(w), in FP64 from the
// setup-precision 2D spectra [L*M][N][P] (map l*M + m), rounded once into [k2][kappa*L + l][CP]
template <typename T>
__global__ void theta3_store_kernel(const SetupC<T>* __restrict__ th64, typename CT<T>::type* __restrict__ th,
                                    const double2* __restrict__ w, int L, int M, int N) {
  using C = typename CT<T>::type;
  const int H = N / 2 + 1, P = half_pitch(N), CP = col_pitch(N);
  const size_t total = (size_t)L * N * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % N);
    const size_t r = i / N;
    const int l = (int)(r % L);
    const int k2 = (int)(r / L);
    double2 v[16];
    for (int m = 0; m < M; ++m) v[m] = cconv<double2>(th64[(((size_t)l * M + m) * N + k1) * P + k2]);
    for (int k = 0; k < M; ++k) {
      double2 acc = make_double2(0.0, 0.0);
      for (int m = 0; m < M; ++m) cfma(acc, w[(k * m) % M], v[m]);
      th[((size_t)k2 * M * L + (size_t)k * L + l) * CP + k1] = cconv<C>(acc);
    }
  }
}

template <typename T> size_t cd3_smem(int M, int L, int BB) {
  return ((size_t)M * L * BB + (size_t)M * BB + (size_t)M * M) * sizeof(typename CT<T>::type);
}

}  // namespace

template <typename T> cudaError_t launch_cd3_solve(const CD3Args<T>& a, cudaStream_t s) {
  if (a.L > 32 || a.M > 16) return cudaErrorInvalidValue;
  const int BB = cd3_bins<T>(a.M, a.L);
  const size_t sm = cd3_smem<T>(a.M, a.L, BB);
  const dim3 grid(a.N / BB, a.N / 2 + 1), block(BB, a.M);
  auto k8 = cd3_solve_kernel<T, 8>;
  auto k32 = cd3_solve_kernel<T, 32>;
  auto k = a.L <= 8 ? k8 : k32;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  return launch_plain(k, grid, block, sm, s, a);
}

template <typename T>
cudaError_t launch_p3_from_z(const typename CT<T>::type* zcol, const typename CT<T>::type* th3,
                             typename CT<T>::type* p, const CD3Args<T>& a, double scale, cudaStream_t s) {
  if (a.L > 32 || a.M > 16) return cudaErrorInvalidValue;
  const int BB = cd3_bins<T>(a.M, a.L);
  const size_t sm = cd3_smem<T>(a.M, a.L, BB);
  const dim3 grid(a.N / BB, a.N / 2 + 1), block(BB, a.M);
  auto k = p3_from_z_kernel<T, 32>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const T sc = scale > 0 ? (T)scale : T(1) / ((T)a.N * (T)a.N);
  return launch_plain(k, grid, block, sm, s, zcol, th3, p, a, sc);
}

template <typename Tin>
cudaError_t launch_embed_filters3d(const Tin* d, double* out, int L, int Q, int P, int M, int N, cudaStream_t s) {
  const int n = L * Q * P * P;
  return launch_plain(embed3_kernel<Tin>, dim3((n + 255) / 256), dim3(256), 0, s, d, out, L, Q, P, M, N);
}

template <typename T>
cudaError_t launch_theta3_store(const SetupC<T>* th64, typename CT<T>::type* th, const double2* w, int L, int M, int N,
                                cudaStream_t s) {
  return launch_plain(theta3_store_kernel<T>, dim3(512), dim3(256), 0, s, th64, th, w, L, M, N);
}

template <typename T> bool cd3_fits(int M, int L) {
  return L <= 32 && M <= 16 && cd3_smem<T>(M, L, cd3_bins<T>(M, L)) <= 200 * 1024 &&
         cd3_bins<T>(M, L) * M <= 512;
}

template cudaError_t launch_cd3_solve<float>(const CD3Args<float>&, cudaStream_t);
template cudaError_t launch_cd3_solve<double>(const CD3Args<double>&, cudaStream_t);
template cudaError_t launch_p3_from_z<float>(const float2*, const float2*, float2*, const CD3Args<float>&, double,
                                             cudaStream_t);
template cudaError_t launch_p3_from_z<double>(const double2*, const double2*, double2*, const CD3Args<double>&,
                                              double, cudaStream_t);
template cudaError_t launch_embed_filters3d<float>(const float*, double*, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_embed_filters3d<double>(const double*, double*, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_theta3_store<float>(const cdf*, float2*, const double2*, int, int, int, cudaStream_t);
template cudaError_t launch_theta3_store<double>(const double2*, double2*, const double2*, int, int, int,
                                                 cudaStream_t);
template bool cd3_fits<float>(int, int);
template bool cd3_fits<double>(int, int);

}  // namespace cip
