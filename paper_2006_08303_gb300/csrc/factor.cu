// Setup kernels, all arithmetic in FP64:
//   * Psi(w) = rho g(w) I + beta Lambda(w)^H Lambda(w) at every half-spectrum
//     bin and its inverse (Alg. 1 line 2; Section IV-A, the inverse of Psi is
//     "computed only once").  Positive-definite bins use a Cholesky
//     factorisation L L^H and Psi^{-1} = L^{-H} L^{-1}; bins where g(w) = 0
//     (the DC bin of TV, singular when the PSFs have unit sum) or where the
//     factorisation fails get the min-norm pseudo-inverse from a cyclic
//     Jacobi eigendecomposition of the real 2M x 2M embedding of Psi
//     (eigenvalues below 1e-10 of the largest dropped).  Results are scaled by
//     1/N^2 (the inverse-DFT normalisation) and rounded once to the plan's
//     precision, packed as the upper triangle row by row.
//   * xb(w) = Psi^{-1}(w) beta Lambda(w)^H yhat(w) in FP64 (the constant data term).
//   * the deterministic reduction of the prior pass's residual partial sums.
#include "kernels.h"

namespace cip {

namespace {

constexpr int kMaxM = 16;

__device__ __forceinline__ void push_bin(int* list, int cap, int bin) {
  const int slot = atomicAdd(list, 1);
  if (slot < cap) list[1 + slot] = bin;
}

__device__ __forceinline__ double bin_g(const double* gs, int use_g, int k1, int k2) {
  return use_g ? gs[k1] + gs[k2] : 1.0;
}

// Psi_ij (i >= j) = rho g delta_ij + beta sum_k conj(Lam_{k,i}) Lam_{k,j}
__device__ __forceinline__ double2 psi_entry(const double2* lam, size_t off, size_t mplane, int K, int M, int i, int j,
                                             double rho_g, double beta) {
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < K; ++k) {
    const double2 a = lam[(size_t)(k * M + i) * mplane + off];
    const double2 b = lam[(size_t)(k * M + j) * mplane + off];
    cfmac(acc, a, b);
  }
  acc.x *= beta;
  acc.y *= beta;
  if (i == j) {
    acc.x += rho_g;
    acc.y = 0.0;
  }
  return acc;
}

template <typename Tout>
__global__ void __launch_bounds__(128) factor_kernel(const double2* __restrict__ lam, const double* __restrict__ gs,
                                                     int use_g, int K, int M, int N, double rho, double beta,
                                                     typename CT<Tout>::type* __restrict__ pinv,
                                                     double2* __restrict__ pinv64, int* list, int cap) {
  using C = typename CT<Tout>::type;
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const double g = bin_g(gs, use_g, k1, k2);
  if (g == 0.0) {
    push_bin(list, cap, bin);
    return;
  }
  double2 L[kMaxM][kMaxM];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j <= i; ++j) L[i][j] = psi_entry(lam, off, mplane, K, M, i, j, rho * g, beta);
  // Cholesky, lower, in place
  for (int j = 0; j < M; ++j) {
    double d = L[j][j].x;
    for (int k = 0; k < j; ++k) d -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
    if (!(d > 0.0)) {
      push_bin(list, cap, bin);
      return;
    }
    const double ljj = sqrt(d);
    L[j][j] = make_double2(ljj, 0.0);
    const double inv = 1.0 / ljj;
    for (int i = j + 1; i < M; ++i) {
      double2 s = L[i][j];
      for (int k = 0; k < j; ++k) {
        // s -= L[i][k] conj(L[j][k])
        const double2 a = L[i][k], b = L[j][k];
        s.x -= a.x * b.x + a.y * b.y;
        s.y -= a.y * b.x - a.x * b.y;
      }
      L[i][j] = make_double2(s.x * inv, s.y * inv);
    }
  }
  // W = L^{-1} (lower)
  double2 W[kMaxM][kMaxM];
  for (int i = 0; i < M; ++i) {
    const double inv = 1.0 / L[i][i].x;
    W[i][i] = make_double2(inv, 0.0);
    for (int j = 0; j < i; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = j; k < i; ++k) cfma(s, L[i][k], W[k][j]);
      W[i][j] = make_double2(-s.x * inv, -s.y * inv);
    }
  }
  // Psi^{-1} = W^H W, packed upper, scaled by 1/N^2; the plan-precision copy is
  // stored [k2][pk][k1] (contiguous bins along a column), the FP64 copy [pk][k1][P]
  const double sc = 1.0 / ((double)N * (double)N);
  const size_t colbase = (size_t)k2 * (M * (M + 1) / 2) * col_pitch(N) + k1;
  int pk = 0;
  for (int i = 0; i < M; ++i) {
    for (int j = i; j < M; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = j; k < M; ++k) cfmac(s, W[k][i], W[k][j]);
      if (i == j) s.y = 0.0;
      pinv[colbase + (size_t)pk * col_pitch(N)] = mk<C>(s.x * sc, s.y * sc);
      if (pinv64) pinv64[(size_t)pk * mplane + off] = make_double2(s.x * sc, s.y * sc);
      ++pk;
    }
  }
}

// Min-norm pseudo-inverse at the listed bins (one thread per bin).
template <typename Tout>
__global__ void factor_pinv_kernel(const double2* __restrict__ lam, const double* __restrict__ gs, int use_g, int K,
                                   int M, int N, double rho, double beta, typename CT<Tout>::type* __restrict__ pinv,
                                   double2* __restrict__ pinv64, const int* list, int cap) {
  using C = typename CT<Tout>::type;
  const int n = min(list[0], cap);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = list[1 + t];
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const double g = bin_g(gs, use_g, k1, k2);
  const int D = 2 * M;
  double A[2 * kMaxM][2 * kMaxM], V[2 * kMaxM][2 * kMaxM];
  for (int i = 0; i < M; ++i) {
    for (int j = 0; j <= i; ++j) {
      const double2 p = psi_entry(lam, off, mplane, K, M, i, j, rho * g, beta);
      // Psi_ij = p (i >= j), Psi_ji = conj(p); embedding [[B, -C], [C, B]]
      A[i][j] = p.x; A[M + i][M + j] = p.x; A[M + i][j] = p.y; A[i][M + j] = -p.y;
      A[j][i] = p.x; A[M + j][M + i] = p.x; A[M + j][i] = -p.y; A[j][M + i] = p.y;
    }
  }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) fro += A[i][j] * A[i][j];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off2 = 0.0;
    for (int p = 0; p < D; ++p)
      for (int q = p + 1; q < D; ++q) off2 += A[p][q] * A[p][q];
    if (off2 <= 1e-32 * fro || off2 == 0.0) break;
    for (int p = 0; p < D; ++p) {
      for (int q = p + 1; q < D; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < D; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < D; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < D; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
  double emax = 0.0;
  for (int i = 0; i < D; ++i) emax = fmax(emax, A[i][i]);
  const double cut = 1e-10 * emax;
  const double sc = 1.0 / ((double)N * (double)N);
  int pk = 0;
  for (int i = 0; i < M; ++i) {
    for (int j = i; j < M; ++j) {
      double re = 0.0, im = 0.0;
      for (int e = 0; e < D; ++e) {
        const double d = A[e][e];
        if (d > cut) {
          re += V[i][e] * V[j][e] / d;
          im += V[M + i][e] * V[j][e] / d;
        }
      }
      if (i == j) im = 0.0;
      pinv[((size_t)k2 * (M * (M + 1) / 2) + pk) * col_pitch(N) + k1] = mk<C>(re * sc, im * sc);
      if (pinv64) pinv64[(size_t)pk * mplane + off] = make_double2(re * sc, im * sc);
      ++pk;
    }
  }
}

// xb(w) = Psi^{-1}(w) / N^2 * beta Lambda(w)^H yhat(w), all in FP64, rounded once.
// This is the data term of Eq. solx_Trans_DFT; it does not change across
// iterations, so the ill-conditioned product with Psi^{-1} (cancellation at
// bins where the PSFs are nearly dependent) is taken once in FP64 and the
// per-iteration column pass only adds Psi^{-1} rho F T^H (t - u).
template <typename Tout>
__global__ void rhs_kernel(const double2* __restrict__ lam, const double2* __restrict__ yhat,
                           const double2* __restrict__ pinv64, int K, int M, int N, double beta,
                           typename CT<Tout>::type* __restrict__ xb) {
  using C = typename CT<Tout>::type;
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  double2 b[kMaxM], x[kMaxM];
  for (int m = 0; m < M; ++m) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < K; ++k) cfmac(acc, lam[(size_t)(k * M + m) * mplane + off], yhat[(size_t)k * mplane + off]);
    b[m] = make_double2(beta * acc.x, beta * acc.y);
    x[m] = make_double2(0.0, 0.0);
  }
  int pk = 0;
  for (int i = 0; i < M; ++i) {
    for (int j = i; j < M; ++j) {
      const double2 pij = pinv64[(size_t)pk * mplane + off];
      ++pk;
      cfma(x[i], pij, b[j]);
      if (j != i) cfmac(x[j], pij, b[i]);
    }
  }
  // stored [k2][m][k1]: the bins of one column are contiguous for the column pass
  for (int m = 0; m < M; ++m) xb[((size_t)k2 * M + m) * col_pitch(N) + k1] = mk<C>(x[m].x, x[m].y);
}

template <typename Tout>
__global__ void store_kernel(const double2* __restrict__ src, typename CT<Tout>::type* __restrict__ dst, size_t n) {
  using C = typename CT<Tout>::type;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = mk<C>(src[i].x, src[i].y);
}

__global__ void reduce_kernel(const double* __restrict__ partials, int nblocks, double rho, double tol,
                              double* __restrict__ out, int* conv) {
  __shared__ double sm[256][kNPart];
  const int tid = threadIdx.x;
  double acc[kNPart] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = tid; b < nblocks; b += 256)
    for (int i = 0; i < kNPart; ++i) acc[i] += partials[(size_t)b * kNPart + i];
  for (int i = 0; i < kNPart; ++i) sm[tid][i] = acc[i];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s)
      for (int i = 0; i < kNPart; ++i) sm[tid][i] += sm[tid + s][i];
    __syncthreads();
  }
  if (tid == 0) {
    for (int i = 0; i < kNPart; ++i) out[i] = sm[0][i];
    const double r = sqrt(sm[0][0]);
    const double den_r = fmax(fmax(sqrt(sm[0][1]), sqrt(sm[0][2])), 1e-300);
    const double s = rho * sqrt(sm[0][4]);
    const double den_s = fmax(rho * sqrt(sm[0][3]), 1e-300);
    out[kNPart] = r / den_r;
    out[kNPart + 1] = s / den_s;
    if (conv) *conv = (tol > 0.0 && out[kNPart] < tol && out[kNPart + 1] < tol) ? 1 : 0;
  }
}

}  // namespace

template <typename Tout>
cudaError_t launch_factor(const double2* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                          double beta, typename CT<Tout>::type* pinv, double2* pinv64, int* pinv_list, int list_cap,
                          cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const int nb = N * (N / 2 + 1);
  factor_kernel<Tout><<<(nb + 127) / 128, 128, 0, s>>>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list,
                                                       list_cap);
  return cudaGetLastError();
}

template <typename Tout>
cudaError_t launch_factor_pinv(const double2* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                               double beta, typename CT<Tout>::type* pinv, double2* pinv64, const int* pinv_list,
                               int list_cap, cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  factor_pinv_kernel<Tout><<<(list_cap + 31) / 32, 32, 0, s>>>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64,
                                                               pinv_list, list_cap);
  return cudaGetLastError();
}

template <typename Tout>
cudaError_t launch_rhs(const double2* lam, const double2* yhat, const double2* pinv64, int K, int M, int N,
                       double beta, typename CT<Tout>::type* xb, cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const int nb = N * (N / 2 + 1);
  rhs_kernel<Tout><<<(nb + 127) / 128, 128, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  return cudaGetLastError();
}

template <typename Tout>
cudaError_t launch_spectra_store(const double2* src, typename CT<Tout>::type* dst, size_t n, cudaStream_t s) {
  store_kernel<Tout><<<1024, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int nblocks, double rho, double tol, double* out, int* conv,
                                   cudaStream_t s) {
  reduce_kernel<<<1, 256, 0, s>>>(partials, nblocks, rho, tol, out, conv);
  return cudaGetLastError();
}

template cudaError_t launch_factor<float>(const double2*, const double*, int, int, int, int, double, double, float2*,
                                          double2*, int*, int, cudaStream_t);
template cudaError_t launch_factor<double>(const double2*, const double*, int, int, int, int, double, double,
                                           double2*, double2*, int*, int, cudaStream_t);
template cudaError_t launch_factor_pinv<float>(const double2*, const double*, int, int, int, int, double, double,
                                               float2*, double2*, const int*, int, cudaStream_t);
template cudaError_t launch_factor_pinv<double>(const double2*, const double*, int, int, int, int, double, double,
                                                double2*, double2*, const int*, int, cudaStream_t);
template cudaError_t launch_rhs<float>(const double2*, const double2*, const double2*, int, int, int, double,
                                       float2*, cudaStream_t);
template cudaError_t launch_rhs<double>(const double2*, const double2*, const double2*, int, int, int, double,
                                        double2*, cudaStream_t);
template cudaError_t launch_spectra_store<float>(const double2*, float2*, size_t, cudaStream_t);
template cudaError_t launch_spectra_store<double>(const double2*, double2*, size_t, cudaStream_t);

}  // namespace cip

// ---------------------------------------------------------------------------
// The plain FP32 method (comparison baseline for the mixed-precision path):
// Psi formed and inverted in FP32 (complex64 Cholesky) from the PSF spectra
// rounded to complex64, and b = beta Lambda^H yhat in FP32; the column pass
// then applies x = Psi^{-1} (b + Q) every iteration.
// ---------------------------------------------------------------------------
namespace cip {
namespace {

__global__ void __launch_bounds__(128) factor_fp32_kernel(const double2* __restrict__ lam, const double* __restrict__ gs,
                                                          int use_g, int K, int M, int N, float rho, float beta,
                                                          float2* __restrict__ pinv, int* list, int cap) {
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const float g = use_g ? (float)(gs[k1] + gs[k2]) : 1.0f;
  if (g == 0.0f) {
    push_bin(list, cap, bin);
    return;
  }
  float2 L[kMaxM][kMaxM];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j <= i; ++j) {
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < K; ++k) {
        const double2 a = lam[(size_t)(k * M + i) * mplane + off], b = lam[(size_t)(k * M + j) * mplane + off];
        cfmac(acc, make_float2((float)a.x, (float)a.y), make_float2((float)b.x, (float)b.y));
      }
      acc.x *= beta;
      acc.y *= beta;
      if (i == j) {
        acc.x += rho * g;
        acc.y = 0.f;
      }
      L[i][j] = acc;
    }
  for (int j = 0; j < M; ++j) {
    float d = L[j][j].x;
    for (int k = 0; k < j; ++k) d -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
    if (!(d > 0.f)) {
      push_bin(list, cap, bin);
      return;
    }
    const float ljj = sqrtf(d), inv = 1.0f / ljj;
    L[j][j] = make_float2(ljj, 0.f);
    for (int i = j + 1; i < M; ++i) {
      float2 s = L[i][j];
      for (int k = 0; k < j; ++k) {
        const float2 a = L[i][k], b = L[j][k];
        s.x -= a.x * b.x + a.y * b.y;
        s.y -= a.y * b.x - a.x * b.y;
      }
      L[i][j] = make_float2(s.x * inv, s.y * inv);
    }
  }
  float2 W[kMaxM][kMaxM];
  for (int i = 0; i < M; ++i) {
    const float inv = 1.0f / L[i][i].x;
    W[i][i] = make_float2(inv, 0.f);
    for (int j = 0; j < i; ++j) {
      float2 s = make_float2(0.f, 0.f);
      for (int k = j; k < i; ++k) cfma(s, L[i][k], W[k][j]);
      W[i][j] = make_float2(-s.x * inv, -s.y * inv);
    }
  }
  const float sc = 1.0f / ((float)N * (float)N);
  const size_t colbase = (size_t)k2 * (M * (M + 1) / 2) * col_pitch(N) + k1;
  int pk = 0;
  for (int i = 0; i < M; ++i)
    for (int j = i; j < M; ++j) {
      float2 s = make_float2(0.f, 0.f);
      for (int k = j; k < M; ++k) cfmac(s, W[k][i], W[k][j]);
      if (i == j) s.y = 0.f;
      pinv[colbase + (size_t)pk * col_pitch(N)] = make_float2(s.x * sc, s.y * sc);
      ++pk;
    }
}

__global__ void rhs_fp32_kernel(const double2* __restrict__ lam, const double2* __restrict__ yhat, int K, int M,
                                int N, float beta, float2* __restrict__ b) {
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  for (int m = 0; m < M; ++m) {
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      const double2 l = lam[(size_t)(k * M + m) * mplane + off], y = yhat[(size_t)k * mplane + off];
      cfmac(acc, make_float2((float)l.x, (float)l.y), make_float2((float)y.x, (float)y.y));
    }
    b[((size_t)k2 * M + m) * col_pitch(N) + k1] = make_float2(beta * acc.x, beta * acc.y);
  }
}

}  // namespace

cudaError_t launch_factor_fp32(const double2* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                               double beta, float2* pinv, int* pinv_list, int list_cap, cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const int nb = N * (N / 2 + 1);
  factor_fp32_kernel<<<(nb + 127) / 128, 128, 0, s>>>(lam, gs, use_g, K, M, N, (float)rho, (float)beta, pinv,
                                                     pinv_list, list_cap);
  return cudaGetLastError();
}

cudaError_t launch_rhs_fp32(const double2* lam, const double2* yhat, int K, int M, int N, double beta, float2* b,
                            cudaStream_t s) {
  const int nb = N * (N / 2 + 1);
  rhs_fp32_kernel<<<(nb + 255) / 256, 256, 0, s>>>(lam, yhat, K, M, N, (float)beta, b);
  return cudaGetLastError();
}

}  // namespace cip
