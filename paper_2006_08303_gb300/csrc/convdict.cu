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
#include <algorithm>

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
  const C* pcol = a.pinv + binp(k2, 0, k1, npk, N);  // plane stride kBinBlock
  C acc = mk<C>(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < MMAX; ++j) {
    if (j < M) {
      const int i0 = min(m, j), j0 = max(m, j);
      const int pk = i0 * M - (i0 * (i0 - 1)) / 2 + (j0 - i0);
      const C pij = pcol[(size_t)pk * kBinBlock];
      const C pj = pin[(size_t)j * CP];
      if (m <= j) cfma(acc, pij, pj);
      else cfmac(acc, pij, pj);
    }
  }
  C x = a.xb[binp(k2, m, k1, M, N)];
  x.x += a.n2 * acc.x;
  x.y += a.n2 * acc.y;
  a.xcol[((size_t)k2 * M + m) * CP + k1] = x;
  // c_l = conj(theta_l) x + G_l ; s = theta^T c ; nrm = ||theta||^2
  C* g = a.colbuf + ((size_t)k2 * M * L + (size_t)m * L) * CP + k1;
  const C* th = a.theta + (size_t)k2 * a.th_planes * CP + k1;
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
                                typename CT<T>::type* __restrict__ p, int N, int M, int L, int thp, T s) {
  using C = typename CT<T>::type;
  const int CP = col_pitch(N);
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y, m = blockIdx.z;
  if (k1 >= N) return;
  C acc = mk<C>(0.0, 0.0);
  for (int l = 0; l < L; ++l)
    cfma(acc, th[((size_t)k2 * thp + l) * CP + k1], zcol[((size_t)k2 * M * L + (size_t)m * L + l) * CP + k1]);
  p[((size_t)k2 * M + m) * CP + k1] = mk<C>(acc.x * s, acc.y * s);
}

// ---- online dictionary update (Section IV-B, Eqs. d_admm, g_admm, h_admm, sold_3D) ----------

// Per frequency, one thread (k1 = threadIdx + block offset, k2 = blockIdx.y, so that the warps
// read the column layout contiguously): the filter normal equation summed over the M channels,
// (sigma I + W W^H) d = b with W = [conj(zhat_{l,s})] (L x M) and b = W xhat + sigma F(g - e), by
// the Woodbury identity d = (b - W alpha) / sigma, (sigma I_M + W^H W) alpha = W^H b.  The L
// filters are streamed twice: once to accumulate W^H W and W^H b, once to form d; the M x M system
// is solved by Cholesky in registers.  zcol holds the code spectra and xcol the image spectra
// scaled by 1/N^2 (the column solve's convention); ge holds F(g - e) (gep planes per bin); dcol
// receives d-hat / N^2 (so that an unnormalised inverse gives d).
template <typename T, int M>
__global__ void __launch_bounds__(64) dl_solve_kernel(const typename CT<T>::type* __restrict__ zcol,
                                                      const typename CT<T>::type* __restrict__ xcol,
                                                      const typename CT<T>::type* __restrict__ gecol, int gep,
                                                      typename CT<T>::type* __restrict__ dcol, int N, int L,
                                                      T sigma) {
  using C = typename CT<T>::type;
  const int CP = col_pitch(N);
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x, k2 = blockIdx.y;
  if (k1 >= N) return;
  const T n2 = (T)N * (T)N;
  const C* zb = zcol + (size_t)k2 * M * L * CP + k1;  // z_{l,s} at zb[(s L + l) CP]
  const C* gb = gecol + (size_t)k2 * gep * CP + k1;
  C x[M], c[M], G[M][M];
#pragma unroll
  for (int s = 0; s < M; ++s) {
    const C v = xcol[((size_t)k2 * M + s) * CP + k1];
    x[s] = mk<C>(v.x * n2, v.y * n2);
    c[s] = mk<C>(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < M; ++t) G[s][t] = mk<C>(0.0, 0.0);
  }
  // b_l = sigma ge_l + sum_s conj(z_{l,s}) x_s
  auto load_b = [&](int l, C (&z)[M]) {
    const C ge = __ldg(gb + (size_t)l * CP);
    C b = mk<C>(sigma * ge.x, sigma * ge.y);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const C v = __ldg(zb + ((size_t)s * L + l) * CP);
      z[s] = mk<C>(v.x * n2, v.y * n2);
      cfmac(b, z[s], x[s]);
    }
    return b;
  };
#pragma unroll 2
  for (int l = 0; l < L; ++l) {
    C z[M];
    const C b = load_b(l, z);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      cfma(c[s], z[s], b);  // W^H b
#pragma unroll
      for (int t = 0; t <= s; ++t) cfmac(G[s][t], z[t], z[s]);  // z_s conj(z_t)
    }
  }
  // Cholesky of sigma I + G = R R^H (lower, in place), then R w = c and R^H alpha = w
#pragma unroll
  for (int j = 0; j < M; ++j) {
    T d = sigma + G[j][j].x;
#pragma unroll
    for (int k = 0; k < j; ++k) d -= G[j][k].x * G[j][k].x + G[j][k].y * G[j][k].y;
    const T r = sqrt(d > T(0) ? d : T(0)), inv = r > T(0) ? T(1) / r : T(0);
    G[j][j] = mk<C>(r, 0.0);
#pragma unroll
    for (int i = j + 1; i < M; ++i) {
      C acc = G[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) {  // acc -= G_ik conj(G_jk)
        const C a = G[i][k], bb = G[j][k];
        acc.x -= a.x * bb.x + a.y * bb.y;
        acc.y -= a.y * bb.x - a.x * bb.y;
      }
      G[i][j] = mk<C>(acc.x * inv, acc.y * inv);
    }
  }
  C w[M], al[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    C acc = c[i];
#pragma unroll
    for (int k = 0; k < i; ++k) {
      acc.x -= G[i][k].x * w[k].x - G[i][k].y * w[k].y;
      acc.y -= G[i][k].x * w[k].y + G[i][k].y * w[k].x;
    }
    const T inv = T(1) / G[i][i].x;
    w[i] = mk<C>(acc.x * inv, acc.y * inv);
  }
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    C acc = w[i];
#pragma unroll
    for (int k = i + 1; k < M; ++k) {  // acc -= conj(G_ki) alpha_k
      acc.x -= G[k][i].x * al[k].x + G[k][i].y * al[k].y;
      acc.y -= G[k][i].x * al[k].y - G[k][i].y * al[k].x;
    }
    const T inv = T(1) / G[i][i].x;
    al[i] = mk<C>(acc.x * inv, acc.y * inv);
  }
  const T sc = T(1) / (sigma * n2);
  C* db = dcol + (size_t)k2 * L * CP + k1;
#pragma unroll 2
  for (int l = 0; l < L; ++l) {
    C z[M];
    C d = load_b(l, z);
#pragma unroll
    for (int s = 0; s < M; ++s) {  // d -= conj(z_s) alpha_s
      d.x -= z[s].x * al[s].x + z[s].y * al[s].y;
      d.y -= z[s].x * al[s].y - z[s].y * al[s].x;
    }
    db[(size_t)l * CP] = mk<C>(d.x * sc, d.y * sc);
  }
}

// 1 / ||Q^T (d + e)|| per filter l = blockIdx.x (0 for a zero filter), formed before any block
// of the projection writes e.
template <typename T>
__global__ void __launch_bounds__(256) dl_norm_kernel(const T* __restrict__ d, const T* __restrict__ e,
                                                      T* __restrict__ inv, int N, int P) {
  __shared__ double red[8];
  const int l = blockIdx.x;
  const size_t plane = (size_t)N * N;
  const T* dl = d + (size_t)l * plane;
  const T* el = e + (size_t)l * plane;
  const int c = P / 2;
  double acc = 0.0;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    const int a = ((i / P - c) % N + N) % N, b = ((i % P - c) % N + N) % N;
    const size_t k = (size_t)a * N + b;
    const double v = (double)dl[k] + (double)el[k];
    acc += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    inv[l] = tot > 0.0 ? (T)(1.0 / sqrt(tot)) : T(0);
  }
}

// Eq. g_admm and Eq. h_admm (reading R22) for filter l = blockIdx.x over the chunk blockIdx.y of
// its N x N plane: g = Q Q^T (d + e) * inv_l, e <- e + d - g, and g - e for the next filter
// solve.  gs holds [g planes][g - e planes] (L each).
template <typename T>
__global__ void __launch_bounds__(256) dl_project_kernel(const T* __restrict__ d, T* __restrict__ e,
                                                         T* __restrict__ gs, const T* __restrict__ inv, int L, int N,
                                                         int P) {
  const int l = blockIdx.x;
  const size_t plane = (size_t)N * N;
  const T* dl = d + (size_t)l * plane;
  T* el = e + (size_t)l * plane;
  T* gl = gs + (size_t)l * plane;
  T* ql = gs + ((size_t)L + l) * plane;
  const int c = P / 2;
  const T s = inv[l];
  const size_t chunk = (plane + gridDim.y - 1) / gridDim.y;
  const size_t k0 = (size_t)blockIdx.y * chunk, k1 = min(plane, k0 + chunk);
  for (size_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int a = (int)(k / N), b = (int)(k - (size_t)a * N);
    const int ia = (a + c) % N, ib = (b + c) % N;  // position inside the P x P support if < P
    const bool in = ia < P && ib < P;
    const T v = dl[k] + el[k];
    const T gn = in ? v * s : T(0);
    const T en = v - gn;
    gl[k] = gn;
    el[k] = en;
    ql[k] = gn - en;
  }
}

// filters [L][P][P] (centre P/2) cropped from the N x N planes g
template <typename T>
__global__ void dl_crop_kernel(const T* __restrict__ g, T* __restrict__ out, int L, int N, int P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * P * P) return;
  const int l = idx / (P * P), r = idx - l * P * P;
  const int i = r / P, j = r - i * P;
  const int c = P / 2;
  const int a = ((i - c) % N + N) % N, b = ((j - c) % N + N) % N;
  out[idx] = g[((size_t)l * N + a) * N + b];
}

}  // namespace

template <typename T>
cudaError_t launch_dl_solve(const typename CT<T>::type* zcol, const typename CT<T>::type* xcol,
                            const typename CT<T>::type* gecol, int gep, typename CT<T>::type* dcol, int N, int M,
                            int L, double sigma, cudaStream_t s) {
  const dim3 grid((N + 63) / 64, N / 2 + 1), block(64);
  const T sg = (T)sigma;
  switch (M) {
#define DL_CASE(m) \
  case m: dl_solve_kernel<T, m><<<grid, block, 0, s>>>(zcol, xcol, gecol, gep, dcol, N, L, sg); break;
    DL_CASE(1) DL_CASE(2) DL_CASE(3) DL_CASE(4) DL_CASE(5) DL_CASE(6) DL_CASE(7) DL_CASE(8)
#undef DL_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_dl_norm(const T* d, const T* e, T* inv, int L, int N, int P, cudaStream_t s) {
  dl_norm_kernel<T><<<L, 256, 0, s>>>(d, e, inv, N, P);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dl_project(const T* d, T* e, T* gs, const T* inv, int L, int N, int P, cudaStream_t s) {
  const size_t plane = (size_t)N * N;
  const unsigned chunks = (unsigned)std::min<size_t>(64, std::max<size_t>(1, plane / 2048));
  dl_project_kernel<T><<<dim3(L, chunks), 256, 0, s>>>(d, e, gs, inv, L, N, P);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_dl_crop(const T* g, T* out, int L, int N, int P, cudaStream_t s) {
  const int n = L * P * P;
  dl_crop_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(g, out, L, N, P);
  return cudaGetLastError();
}
template cudaError_t launch_dl_solve<float>(const float2*, const float2*, const float2*, int, float2*, int, int, int,
                                            double, cudaStream_t);
template cudaError_t launch_dl_solve<double>(const double2*, const double2*, const double2*, int, double2*, int, int,
                                             int, double, cudaStream_t);
template cudaError_t launch_dl_norm<float>(const float*, const float*, float*, int, int, int, cudaStream_t);
template cudaError_t launch_dl_norm<double>(const double*, const double*, double*, int, int, int, cudaStream_t);
template cudaError_t launch_dl_project<float>(const float*, float*, float*, const float*, int, int, int, cudaStream_t);
template cudaError_t launch_dl_project<double>(const double*, double*, double*, const double*, int, int, int,
                                               cudaStream_t);
template cudaError_t launch_dl_crop<float>(const float*, float*, int, int, int, cudaStream_t);
template cudaError_t launch_dl_crop<double>(const double*, double*, int, int, int, cudaStream_t);

template <typename T>
cudaError_t launch_p_from_z(const typename CT<T>::type* zcol, const typename CT<T>::type* th,
                            typename CT<T>::type* p, int N, int M, int L, cudaStream_t s, double scale,
                            int th_planes) {
  dim3 grid((N + 127) / 128, N / 2 + 1, M);
  const T sc = scale > 0 ? (T)scale : T(1) / ((T)N * (T)N);
  p_from_z_kernel<T><<<grid, 128, 0, s>>>(zcol, th, p, N, M, L, th_planes > 0 ? th_planes : L, sc);
  return cudaGetLastError();
}
template cudaError_t launch_p_from_z<float>(const float2*, const float2*, float2*, int, int, int, cudaStream_t,
                                            double, int);
template cudaError_t launch_p_from_z<double>(const double2*, const double2*, double2*, int, int, int, cudaStream_t,
                                             double, int);

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
