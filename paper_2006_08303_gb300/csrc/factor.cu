// Setup kernels:
//   * Psi(w) = rho g(w) I + beta Lambda(w)^H Lambda(w) at every half-spectrum
//     bin and its inverse (Alg. 1 line 2; Section IV-A, the inverse of Psi is
//     "computed only once").  Positive-definite bins use a Cholesky
//     factorisation L L^H and Psi^{-1} = L^{-H} L^{-1}, in the setup precision
//     (double-float, about 44 bits, for complex64 plans; FP64 for complex128
//     plans; square roots and reciprocals of the M pivots in FP64), with the
//     packed triangle of each bin in shared memory.  Bins where g(w) = 0 (the
//     DC bin of TV, singular when the PSFs have unit sum) or where the
//     factorisation fails get the min-norm pseudo-inverse from a cyclic Jacobi
//     eigendecomposition of the real 2M x 2M embedding of Psi in FP64
//     (eigenvalues below 1e-10 of the largest dropped).  Results are scaled by
//     1/N^2 (the inverse-DFT normalisation) and rounded once to the plan's
//     precision, packed as the upper triangle row by row; a setup-precision
//     copy is kept for the data term.
//   * xb(w) = Psi^{-1}(w) beta Lambda(w)^H yhat(w) in the setup precision (the constant data term).
//   * the deterministic reduction of the prior pass's residual partial sums.
// The PSF and measurement spectra arrive in the setup precision: complex
// double-float (cdf) for complex64 plans, complex FP64 for complex128 plans.
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

// Psi_ij (i >= j) = rho g delta_ij + beta sum_k conj(Lam_{k,i}) Lam_{k,j}, in FP64
template <typename S>
__device__ __forceinline__ double2 psi_entry(const S* lam, size_t off, size_t mplane, int K, int M, int i, int j,
                                             double rho_g, double beta) {
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < K; ++k) {
    const double2 a = cconv<double2>(lam[(size_t)(k * M + i) * mplane + off]);
    const double2 b = cconv<double2>(lam[(size_t)(k * M + j) * mplane + off]);
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

constexpr int kFacThreads = 64;
constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // packed lower triangle, i >= j

// One thread per bin; its packed triangle lives in shared memory as
// [entry][thread] (consecutive threads, consecutive 16-byte slots), so the
// factorisation keeps no matrix in registers or local memory.
template <typename Tout, int MMAX>
__global__ void __launch_bounds__(kFacThreads) factor_kernel(const SetupC<Tout>* __restrict__ lam,
                                                             const double* __restrict__ gs, int use_g, int K, int M,
                                                             int N, double rho, double beta,
                                                             typename CT<Tout>::type* __restrict__ pinv,
                                                             SetupC<Tout>* __restrict__ pinv64, int* list, int cap) {
  using C = typename CT<Tout>::type;
  using R = typename SetupReal<Tout>::type;
  using S = SetupC<Tout>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* sm = reinterpret_cast<S*>(smem_raw);
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * kFacThreads + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const double g = bin_g(gs, use_g, k1, k2);
  if (g == 0.0) {
    push_bin(list, cap, bin);
    return;
  }
  auto A = [&](int e) -> S& { return sm[e * kFacThreads + threadIdx.x]; };
  const S zero = mk<S>(0.0, 0.0);
  // Gram matrix, accumulated over the K measurement rows of Lambda
#pragma unroll
  for (int i = 0; i < MMAX; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      if (i < M) A(tri(i, j)) = zero;
  for (int k = 0; k < K; ++k) {
    S l[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < M) l[i] = lam[(size_t)(k * M + i) * mplane + off];
#pragma unroll
    for (int i = 0; i < MMAX; ++i) {
      if (i < M) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          S a = A(tri(i, j));
          cfmac(a, l[i], l[j]);
          A(tri(i, j)) = a;
        }
      }
    }
  }
  const R bd(beta), rg(rho * g);
#pragma unroll
  for (int i = 0; i < MMAX; ++i) {
    if (i < M) {
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        S a = A(tri(i, j));
        a.x = a.x * bd;
        a.y = a.y * bd;
        if (i == j) {
          a.x = a.x + rg;
          a.y = R(0.0f);
        }
        A(tri(i, j)) = a;
      }
    }
  }
  // Cholesky L L^H, lower, in place; square roots and reciprocals of the pivots in FP64.
  // The diagonal slot keeps 1/L_jj, which is also the diagonal of W = L^{-1}.
  for (int j = 0; j < M; ++j) {
    R d = A(tri(j, j)).x;
    for (int k = 0; k < j; ++k) {
      const S a = A(tri(j, k));
      d = d - dfma(a.x, a.x, a.y * a.y);
    }
    const double dd = to_double(d);
    if (!(dd > 0.0)) {
      push_bin(list, cap, bin);
      return;
    }
    const R inv(1.0 / sqrt(dd));
    A(tri(j, j)) = cmk(inv, R(0.0f));
    for (int i = j + 1; i < M; ++i) {
      S t = A(tri(i, j));
      for (int k = 0; k < j; ++k) {
        // t -= L_ik conj(L_jk)
        const S a = A(tri(i, k)), b = A(tri(j, k));
        t.x = t.x - dfma(a.x, b.x, a.y * b.y);
        t.y = t.y - dfma(a.y, b.x, -(a.x * b.y));
      }
      A(tri(i, j)) = cmk(t.x * inv, t.y * inv);
    }
  }
  // W = L^{-1} in place, row by row: W_ij = -W_ii sum_{k=j}^{i-1} L_ik W_kj, for ascending j
  // (reads L_ik with k >= j of the row being rewritten and the finished rows above it)
  for (int i = 1; i < M; ++i) {
    const R wii = A(tri(i, i)).x;
    for (int j = 0; j < i; ++j) {
      S t = zero;
      for (int k = j; k < i; ++k) cfma(t, A(tri(i, k)), A(tri(k, j)));
      A(tri(i, j)) = cmk(-(t.x * wii), -(t.y * wii));
    }
  }
  // Psi^{-1} = W^H W, packed upper, scaled by 1/N^2 (exact: N is a power of two); the
  // plan-precision copy is stored blocked by 32 bins of a column (binp), the setup-precision
  // copy [pk][k1][P]
  const float sc = 1.0f / ((float)N * (float)N);
  const int npk = M * (M + 1) / 2;
  int pk = 0;
  for (int i = 0; i < M; ++i) {
    for (int j = i; j < M; ++j) {
      S t = zero;
      for (int k = j; k < M; ++k) cfmac(t, A(tri(k, i)), A(tri(k, j)));
      if (i == j) t.y = R(0.0f);
      t = cscale_pow2(t, sc);
      pinv[binp(k2, pk, k1, npk, N)] = cconv<C>(t);
      if (pinv64) pinv64[(size_t)pk * mplane + off] = t;
      ++pk;
    }
  }
}

// The same factorisation with one warp per bin (kFacWarps consecutive bins per CTA), used for
// M > 12: a bin's M x M work is spread over 32 lanes and an SM keeps up to 64 bins in flight
// (one thread per bin above holds the whole packed triangle in shared memory, which caps an SM at
// 2 warps for M = 16).  Every sum is taken in the same order as above:
//   Gram: lanes own entries of the packed triangle and accumulate them over the K measurement
//         rows, whose M spectra are staged per row for the CTA's bins (consecutive bins: one
//         128-byte load per plane);
//   Cholesky: step j's pivot by lane 0, the rows i > j of column j by lanes;
//   W = L^{-1}: row by row, the entries of a row by lanes (they read only L values of that row and
//         finished rows above);
//   Psi^{-1} = W^H W: entries by lanes, staged in shared memory and written out per entry for
//         the CTA's bins together.
constexpr int kFacWarps = 8;
template <int MMAX> constexpr int fac_epl() { return (MMAX * (MMAX + 1) / 2 + 31) / 32; }  // entries per lane

template <typename Tout, int MMAX>
__global__ void __launch_bounds__(32 * kFacWarps) factor_warp_kernel(const SetupC<Tout>* __restrict__ lam,
                                                                    const double* __restrict__ gs, int use_g, int K,
                                                                    int M, int N, double rho, double beta,
                                                                    typename CT<Tout>::type* __restrict__ pinv,
                                                                    SetupC<Tout>* __restrict__ pinv64, int* list,
                                                                    int cap) {
  using C = typename CT<Tout>::type;
  using R = typename SetupReal<Tout>::type;
  using S = SetupC<Tout>;
  constexpr int NT = MMAX * (MMAX + 1) / 2, EPL = fac_epl<MMAX>();
  __shared__ S tri_s[kFacWarps][NT];   // each warp's packed triangle (lower), later Psi^{-1} (packed upper)
  __shared__ S lrow[MMAX][kFacWarps];  // spectra of one measurement row for the CTA's bins
  __shared__ int skip[kFacWarps];
  const int H = N / 2 + 1, P = half_pitch(N), nb = N * H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bin0 = blockIdx.x * kFacWarps, bin = bin0 + warp;
  const bool valid = bin < nb;
  const int k1 = valid ? bin / H : 0, k2 = valid ? bin - k1 * H : 0;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const double g = valid ? bin_g(gs, use_g, k1, k2) : 1.0;
  if (lane == 0) {
    skip[warp] = (!valid || g == 0.0) ? 1 : 0;
    if (valid && g == 0.0) push_bin(list, cap, bin);
  }
  S* A = tri_s[warp];
  const S zero = mk<S>(0.0, 0.0);
  // entries of this lane in the packed lower triangle: e = lane + 32 q -> (i, j), i >= j
  int ei[EPL], ej[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int e = lane + 32 * q;
    int i = 0;
    while (i + 1 < MMAX && tri(i + 1, 0) <= e) ++i;
    ei[q] = i;
    ej[q] = e - tri(i, 0);
  }
  // Gram over the K measurement rows
  S acc[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) acc[q] = zero;
  for (int k = 0; k < K; ++k) {
    __syncthreads();  // the previous row is consumed
    for (int t = threadIdx.x; t < M * kFacWarps; t += 32 * kFacWarps) {
      const int i = t / kFacWarps, w = t - i * kFacWarps, bw = bin0 + w;
      S v = zero;
      if (bw < nb) {
        const int a1 = bw / H, a2 = bw - a1 * H;
        v = lam[(size_t)(k * M + i) * mplane + (size_t)a1 * P + a2];
      }
      lrow[i][w] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPL; ++q)
      if (ei[q] < M && lane + 32 * q < NT) cfmac(acc[q], lrow[ei[q]][warp], lrow[ej[q]][warp]);
  }
  const R bd(beta), rg(rho * g);
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    if (ei[q] < M && lane + 32 * q < NT) {
      S a = acc[q];
      a.x = a.x * bd;
      a.y = a.y * bd;
      if (ei[q] == ej[q]) {
        a.x = a.x + rg;
        a.y = R(0.0f);
      }
      A[tri(ei[q], ej[q])] = a;
    }
  }
  __syncwarp();
  bool ok = skip[warp] == 0;
  // Cholesky L L^H, lower, in place; the diagonal slot keeps 1/L_jj (= W_jj)
  for (int j = 0; j < M && ok; ++j) {
    double dd = 0.0;
    if (lane == 0) {
      R d = A[tri(j, j)].x;
      for (int k = 0; k < j; ++k) {
        const S a = A[tri(j, k)];
        d = d - dfma(a.x, a.x, a.y * a.y);
      }
      dd = to_double(d);
    }
    dd = __shfl_sync(0xffffffffu, dd, 0);
    if (!(dd > 0.0)) {
      if (lane == 0) push_bin(list, cap, bin);
      ok = false;
      break;
    }
    const R inv(1.0 / sqrt(dd));
    for (int i = j + 1 + lane; i < M; i += 32) {
      S t = A[tri(i, j)];
      for (int k = 0; k < j; ++k) {
        const S a = A[tri(i, k)], b = A[tri(j, k)];
        t.x = t.x - dfma(a.x, b.x, a.y * b.y);
        t.y = t.y - dfma(a.y, b.x, -(a.x * b.y));
      }
      A[tri(i, j)] = cmk(t.x * inv, t.y * inv);
    }
    if (lane == 0) A[tri(j, j)] = cmk(inv, R(0.0f));
    __syncwarp();
  }
  if (ok) {
    // W = L^{-1}: row i from the L values of row i and the finished rows above
    for (int i = 1; i < M; ++i) {
      const R wii = A[tri(i, i)].x;
      S t = zero;
      const int j = lane;
      if (j < i)
        for (int k = j; k < i; ++k) cfma(t, A[tri(i, k)], A[tri(k, j)]);
      __syncwarp();
      if (j < i) A[tri(i, j)] = cmk(-(t.x * wii), -(t.y * wii));
      __syncwarp();
    }
    // Psi^{-1} = W^H W, packed upper row by row, scaled by 1/N^2; kept in registers, then in the
    // warp's triangle slot (entry pk), once every lane has read W
    const float sc = 1.0f / ((float)N * (float)N);
    const int npk = M * (M + 1) / 2;
    S res[EPL];
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int pk = lane + 32 * q;
      if (pk < npk) {
        int i = 0, rem = pk;
        while (rem >= M - i) {
          rem -= M - i;
          ++i;
        }
        const int j = i + rem;
        S t = zero;
        for (int k = j; k < M; ++k) cfmac(t, A[tri(k, i)], A[tri(k, j)]);
        if (i == j) t.y = R(0.0f);
        res[q] = cscale_pow2(t, sc);
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < EPL; ++q)
      if (lane + 32 * q < npk) A[lane + 32 * q] = res[q];
  }
  if (lane == 0 && !ok) skip[warp] = 1;
  __syncthreads();
  // write-out: entry pk of the CTA's bins together
  const int npk = M * (M + 1) / 2;
  for (int t = threadIdx.x; t < npk * kFacWarps; t += 32 * kFacWarps) {
    const int pk = t / kFacWarps, w = t - pk * kFacWarps, bw = bin0 + w;
    if (skip[w]) continue;
    const int a1 = bw / H, a2 = bw - a1 * H;
    const S v = tri_s[w][pk];
    pinv[binp(a2, pk, a1, npk, N)] = cconv<C>(v);
    if (pinv64) pinv64[(size_t)pk * mplane + (size_t)a1 * P + a2] = v;
  }
}

// Min-norm pseudo-inverse at the listed bins (one thread per bin).
template <typename Tout>
__global__ void factor_pinv_kernel(const SetupC<Tout>* __restrict__ lam, const double* __restrict__ gs, int use_g,
                                   int K, int M, int N, double rho, double beta,
                                   typename CT<Tout>::type* __restrict__ pinv, SetupC<Tout>* __restrict__ pinv64,
                                   const int* list, int cap) {
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
      pinv[binp(k2, pk, k1, M * (M + 1) / 2, N)] = mk<C>(re * sc, im * sc);
      if (pinv64) pinv64[(size_t)pk * mplane + off] = cconv<SetupC<Tout>>(make_double2(re * sc, im * sc));
      ++pk;
    }
  }
}

// xb(w) = Psi^{-1}(w) / N^2 * beta Lambda(w)^H yhat(w) in the setup precision, rounded
// once.  This is the data term of Eq. solx_Trans_DFT; it does not change across
// iterations, so the ill-conditioned product with Psi^{-1} (cancellation at
// bins where the PSFs are nearly dependent) is taken once at high precision and
// the per-iteration column pass only adds Psi^{-1} rho F T^H (t - u).
template <typename Tout, int MMAX>
__global__ void __launch_bounds__(128) rhs_kernel(const SetupC<Tout>* __restrict__ lam,
                                                  const SetupC<Tout>* __restrict__ yhat,
                                                  const SetupC<Tout>* __restrict__ pinv64, int K, int M, int N,
                                                  double beta, typename CT<Tout>::type* __restrict__ xb) {
  using C = typename CT<Tout>::type;
  using R = typename SetupReal<Tout>::type;
  using S = SetupC<Tout>;
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  const R bd(beta);
  const S zero = mk<S>(0.0, 0.0);
  S b[MMAX], x[MMAX];
#pragma unroll
  for (int m = 0; m < MMAX; ++m) {
    b[m] = zero;
    x[m] = zero;
  }
  for (int k = 0; k < K; ++k) {
    const S yk = yhat[(size_t)k * mplane + off];
#pragma unroll
    for (int m = 0; m < MMAX; ++m)
      if (m < M) cfmac(b[m], lam[(size_t)(k * M + m) * mplane + off], yk);
  }
#pragma unroll
  for (int m = 0; m < MMAX; ++m) {
    b[m].x = b[m].x * bd;
    b[m].y = b[m].y * bd;
  }
  int pk = 0;
#pragma unroll
  for (int i = 0; i < MMAX; ++i) {
    if (i < M) {
#pragma unroll
      for (int j = i; j < MMAX; ++j) {
        if (j < M) {
          const S pij = pinv64[(size_t)pk * mplane + off];
          ++pk;
          cfma(x[i], pij, b[j]);
          if (j != i) cfmac(x[j], pij, b[i]);
        }
      }
    }
  }
  // stored blocked by 32 bins of a column (binp), as the factor
#pragma unroll
  for (int m = 0; m < MMAX; ++m)
    if (m < M) xb[binp(k2, m, k1, M, N)] = cconv<C>(x[m]);
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

template <typename Tout, int MMAX>
cudaError_t launch_factor_m(const SetupC<Tout>* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                            double beta, typename CT<Tout>::type* pinv, SetupC<Tout>* pinv64, int* pinv_list,
                            int list_cap, cudaStream_t s) {
  const int nb = N * (N / 2 + 1);
  if constexpr (MMAX > 12) {
    // warp per bin: the one-thread form's triangle (2.2 KB per bin) would leave 2 warps per SM
    factor_warp_kernel<Tout, MMAX><<<(nb + kFacWarps - 1) / kFacWarps, 32 * kFacWarps, 0, s>>>(
        lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list, list_cap);
    return cudaGetLastError();
  }
  // thread per bin: for M <= 12 it issues fewer instructions than a warp whose lanes are mostly
  // idle in the short per-bin loops (measured at 512 x 512 x 10: setup 1.37 ms against 3.0 ms)
  const size_t sm = (size_t)(M * (M + 1) / 2) * kFacThreads * sizeof(SetupC<Tout>);
  auto k = factor_kernel<Tout, MMAX>;
  static PerDeviceOnce once;
  const int most = MMAX * (MMAX + 1) / 2 * kFacThreads * (int)sizeof(SetupC<Tout>);
  cudaError_t e = once([&] { return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, most); });
  if (e != cudaSuccess) return e;
  k<<<(nb + kFacThreads - 1) / kFacThreads, kFacThreads, sm, s>>>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64,
                                                                  pinv_list, list_cap);
  return cudaGetLastError();
}

template <typename Tout>
cudaError_t launch_factor(const SetupC<Tout>* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                          double beta, typename CT<Tout>::type* pinv, SetupC<Tout>* pinv64, int* pinv_list,
                          int list_cap, cudaStream_t s) {
  if (M <= 4) return launch_factor_m<Tout, 4>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list, list_cap, s);
  if (M <= 8) return launch_factor_m<Tout, 8>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list, list_cap, s);
  if (M <= 12)
    return launch_factor_m<Tout, 12>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list, list_cap, s);
  if (M <= kMaxM)
    return launch_factor_m<Tout, 16>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64, pinv_list, list_cap, s);
  return cudaErrorInvalidValue;
}

template <typename Tout>
cudaError_t launch_factor_pinv(const SetupC<Tout>* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                               double beta, typename CT<Tout>::type* pinv, SetupC<Tout>* pinv64, const int* pinv_list,
                               int list_cap, cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  factor_pinv_kernel<Tout><<<(list_cap + 31) / 32, 32, 0, s>>>(lam, gs, use_g, K, M, N, rho, beta, pinv, pinv64,
                                                               pinv_list, list_cap);
  return cudaGetLastError();
}

template <typename Tout>
cudaError_t launch_rhs(const SetupC<Tout>* lam, const SetupC<Tout>* yhat, const SetupC<Tout>* pinv64, int K, int M,
                       int N, double beta, typename CT<Tout>::type* xb, cudaStream_t s) {
  const int nb = N * (N / 2 + 1);
  const dim3 grid((nb + 127) / 128), block(128);
  if (M <= 4) rhs_kernel<Tout, 4><<<grid, block, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  else if (M <= 8) rhs_kernel<Tout, 8><<<grid, block, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  else if (M <= 10) rhs_kernel<Tout, 10><<<grid, block, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  else if (M <= 12) rhs_kernel<Tout, 12><<<grid, block, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  else if (M <= kMaxM) rhs_kernel<Tout, 16><<<grid, block, 0, s>>>(lam, yhat, pinv64, K, M, N, beta, xb);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
__global__ void scale_kernel(T* __restrict__ a, size_t n, T f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] *= f;
}

template <typename T> cudaError_t launch_scale(T* a, size_t n, T f, cudaStream_t s) {
  scale_kernel<T><<<1216, 256, 0, s>>>(a, n, f);
  return cudaGetLastError();
}
template cudaError_t launch_scale<float>(float*, size_t, float, cudaStream_t);
template cudaError_t launch_scale<double>(double*, size_t, double, cudaStream_t);

cudaError_t launch_reduce_partials(const double* partials, int nblocks, double rho, double tol, double* out, int* conv,
                                   cudaStream_t s) {
  return launch_plain(reduce_kernel, dim3(1), dim3(256), 0, s, partials, nblocks, rho, tol, out, conv);
}

template cudaError_t launch_factor<float>(const cdf*, const double*, int, int, int, int, double, double, float2*,
                                          cdf*, int*, int, cudaStream_t);
template cudaError_t launch_factor<double>(const double2*, const double*, int, int, int, int, double, double,
                                           double2*, double2*, int*, int, cudaStream_t);
template cudaError_t launch_factor_pinv<float>(const cdf*, const double*, int, int, int, int, double, double, float2*,
                                               cdf*, const int*, int, cudaStream_t);
template cudaError_t launch_factor_pinv<double>(const double2*, const double*, int, int, int, int, double, double,
                                                double2*, double2*, const int*, int, cudaStream_t);
template cudaError_t launch_rhs<float>(const cdf*, const cdf*, const cdf*, int, int, int, double, float2*,
                                       cudaStream_t);
template cudaError_t launch_rhs<double>(const double2*, const double2*, const double2*, int, int, int, double,
                                        double2*, cudaStream_t);

}  // namespace cip

// ---------------------------------------------------------------------------
// The plain FP32 method (comparison baseline for the mixed-precision path):
// Psi formed and inverted in FP32 (complex64 Cholesky) from the PSF spectra
// rounded to complex64, and b = beta Lambda^H yhat in FP32; the column pass
// then applies x = Psi^{-1} (b + Q) every iteration.
// ---------------------------------------------------------------------------
namespace cip {
namespace {

__global__ void __launch_bounds__(128) factor_fp32_kernel(const cdf* __restrict__ lam, const double* __restrict__ gs,
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
        cfmac(acc, cconv<float2>(lam[(size_t)(k * M + i) * mplane + off]),
              cconv<float2>(lam[(size_t)(k * M + j) * mplane + off]));
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
  const int npk = M * (M + 1) / 2;
  int pk = 0;
  for (int i = 0; i < M; ++i)
    for (int j = i; j < M; ++j) {
      float2 s = make_float2(0.f, 0.f);
      for (int k = j; k < M; ++k) cfmac(s, W[k][i], W[k][j]);
      if (i == j) s.y = 0.f;
      pinv[binp(k2, pk, k1, npk, N)] = make_float2(s.x * sc, s.y * sc);
      ++pk;
    }
}

__global__ void rhs_fp32_kernel(const cdf* __restrict__ lam, const cdf* __restrict__ yhat, int K, int M,
                                int N, float beta, float2* __restrict__ b) {
  const int H = N / 2 + 1, P = half_pitch(N);
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= N * H) return;
  const int k1 = bin / H, k2 = bin - k1 * H;
  const size_t off = (size_t)k1 * P + k2, mplane = (size_t)N * P;
  for (int m = 0; m < M; ++m) {
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      cfmac(acc, cconv<float2>(lam[(size_t)(k * M + m) * mplane + off]), cconv<float2>(yhat[(size_t)k * mplane + off]));
    }
    b[binp(k2, m, k1, M, N)] = make_float2(beta * acc.x, beta * acc.y);
  }
}

}  // namespace

cudaError_t launch_factor_fp32(const cdf* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                               double beta, float2* pinv, int* pinv_list, int list_cap, cudaStream_t s) {
  if (M > kMaxM) return cudaErrorInvalidValue;
  const int nb = N * (N / 2 + 1);
  factor_fp32_kernel<<<(nb + 127) / 128, 128, 0, s>>>(lam, gs, use_g, K, M, N, (float)rho, (float)beta, pinv,
                                                     pinv_list, list_cap);
  return cudaGetLastError();
}

cudaError_t launch_rhs_fp32(const cdf* lam, const cdf* yhat, int K, int M, int N, double beta, float2* b,
                            cudaStream_t s) {
  const int nb = N * (N / 2 + 1);
  rhs_fp32_kernel<<<(nb + 255) / 256, 256, 0, s>>>(lam, yhat, K, M, N, (float)beta, b);
  return cudaGetLastError();
}

}  // namespace cip
