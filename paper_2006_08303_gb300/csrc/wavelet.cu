// Kronecker analysis prior T = W (x) C (Section V): W the 2D periodic Symmlet-8 wavelet transform
// of every channel (Mallat levels down to a 16 x 16 coarse band), C the orthonormal DCT-II along
// the channels.  T is orthonormal, so the x-update is that of Eq. solx_Trans_DFT with g = 1 and the
// t-update is the soft threshold of Eq. solt_trans on the coefficients.
//
// The prior pass for this T is a chain of kernels over [M][N][N] planes (x from the row spectra,
// the wavelet levels, the per-pixel channel DCT with shrinkage and dual update, the inverse levels,
// the row spectra of q), because the wavelet is not local to a row tile.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "kernels.h"

namespace cip {

// ---------------------------------------------------------------------------------------------
// Host: the Symmlet lowpass filter from its definition (Daubechies' spectral factorisation)
// ---------------------------------------------------------------------------------------------
namespace {

using cd = std::complex<double>;

// roots of sum_k a[k] y^k (a[deg] != 0) by the Aberth-Ehrlich simultaneous iteration
std::vector<cd> poly_roots(const std::vector<double>& a) {
  const int n = (int)a.size() - 1;
  std::vector<cd> z(n);
  if (n < 1) return z;
  double rad = 0;  // Cauchy bound on the root moduli
  for (int k = 0; k < n; ++k) rad = std::max(rad, std::abs(a[k] / a[n]));
  rad = 1 + rad;
  for (int k = 0; k < n; ++k) z[k] = std::polar(0.5 * rad, 2 * M_PI * (k + 0.25) / n);
  for (int it = 0; it < 500; ++it) {
    double moved = 0;
    for (int k = 0; k < n; ++k) {
      cd p = a[n], dp = 0;
      for (int j = n - 1; j >= 0; --j) {
        dp = dp * z[k] + p;
        p = p * z[k] + a[j];
      }
      const cd ratio = p / dp;
      cd s = 0;
      for (int j = 0; j < n; ++j)
        if (j != k) s += 1.0 / (z[k] - z[j]);
      const cd step = ratio / (1.0 - ratio * s);
      z[k] -= step;
      moved = std::max(moved, std::abs(step) / std::max(1.0, std::abs(z[k])));
    }
    if (moved < 1e-15) break;
  }
  return z;
}

std::vector<cd> poly_mul_linear(const std::vector<cd>& q, cd c0, cd c1) {  // q(w) * (c0 + c1 w)
  std::vector<cd> r(q.size() + 1, cd(0));
  for (size_t i = 0; i < q.size(); ++i) {
    r[i] += q[i] * c0;
    r[i + 1] += q[i] * c1;
  }
  return r;
}

}  // namespace

// Orthonormal lowpass of 2p taps with p vanishing moments and the most nearly linear phase:
// |m0|^2 = cos^{2p}(w/2) P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k; every root y of P gives
// the pair z, 1/z of z^2 - 2(1 - 2y) z + 1 = 0, one of which is kept (conjugate y together); of all
// choices the one whose factor Q(e^{iw}) = prod (1 - z e^{-iw}) has the smallest least-squares
// deviation of its unwrapped phase from a line on [0, pi] (513 samples) is taken, and of the two
// mirror images the one with the smaller energy centroid.  Returns false for p outside [1, 8].
bool symlet_lowpass(int p, double* h) {
  if (p < 1 || p > 8) return false;
  std::vector<double> a(p);
  double binom = 1;  // C(p-1+k, k)
  for (int k = 0; k < p; ++k) {
    if (k > 0) binom = binom * (p - 1 + k) / k;
    a[k] = binom;
  }
  const std::vector<cd> ys = poly_roots(a);
  std::vector<std::vector<cd>> groups;
  std::vector<bool> used(ys.size(), false);
  for (size_t i = 0; i < ys.size(); ++i) {
    if (used[i]) continue;
    used[i] = true;
    const cd w = 1.0 - 2.0 * ys[i];
    cd z = w + std::sqrt(w * w - 1.0);
    if (std::abs(z) >= 1) z = 1.0 / z;
    if (std::abs(ys[i].imag()) <= 1e-9 * std::max(1.0, std::abs(ys[i]))) {
      groups.push_back({cd(z.real(), 0)});
    } else {
      size_t j = ys.size();
      double best = 1e300;
      for (size_t k = 0; k < ys.size(); ++k)
        if (!used[k] && std::abs(ys[k] - std::conj(ys[i])) < best) {
          best = std::abs(ys[k] - std::conj(ys[i]));
          j = k;
        }
      if (j == ys.size()) return false;
      used[j] = true;
      groups.push_back({z, std::conj(z)});
    }
  }
  const int L = 2 * p, K = 512;
  double best_dev = 1e300, best_cen = 1e300;
  std::vector<double> best_h(L);
  for (int pick = 0; pick < (1 << groups.size()); ++pick) {
    std::vector<cd> roots;
    for (size_t b = 0; b < groups.size(); ++b)
      for (const cd& z : groups[b]) roots.push_back(((pick >> b) & 1) ? 1.0 / z : z);
    // h(w) = prod (1 - r w) (1 + w)^p in powers of w = z^-1, scaled to sum sqrt(2)
    std::vector<cd> q{cd(1)};
    for (const cd& r : roots) q = poly_mul_linear(q, 1.0, -r);
    for (int k = 0; k < p; ++k) q = poly_mul_linear(q, 1.0, 1.0);
    double sum = 0;
    for (const cd& c : q) sum += c.real();
    std::vector<double> hh(L);
    for (int n = 0; n < L; ++n) hh[n] = q[n].real() * std::sqrt(2.0) / sum;
    // unwrapped phase of Q on [0, pi] and its deviation from the least-squares line
    std::vector<double> om(K + 1), ph(K + 1);
    for (int k = 0; k <= K; ++k) {
      om[k] = M_PI * k / K;
      cd Q = 1;
      for (const cd& r : roots) Q *= 1.0 - r * std::polar(1.0, -om[k]);
      double v = std::arg(Q);
      if (k > 0) {
        while (v - ph[k - 1] > M_PI) v -= 2 * M_PI;
        while (v - ph[k - 1] < -M_PI) v += 2 * M_PI;
      }
      ph[k] = v;
    }
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int k = 0; k <= K; ++k) {
      sx += om[k];
      sy += ph[k];
      sxx += om[k] * om[k];
      sxy += om[k] * ph[k];
    }
    const double n1 = K + 1, slope = (n1 * sxy - sx * sy) / (n1 * sxx - sx * sx), icpt = (sy - slope * sx) / n1;
    double dev = 0, cen = 0;
    for (int k = 0; k <= K; ++k) dev += (ph[k] - icpt - slope * om[k]) * (ph[k] - icpt - slope * om[k]);
    for (int n = 0; n < L; ++n) cen += n * hh[n] * hh[n];
    const bool tie = std::abs(dev - best_dev) <= 1e-6 * std::max(1.0, best_dev);
    if ((!tie && dev < best_dev) || (tie && cen < best_cen)) {
      best_dev = tie ? std::min(dev, best_dev) : dev;
      best_cen = cen;
      best_h = hh;
    }
  }
  for (int n = 0; n < L; ++n) h[n] = best_h[n];
  return true;
}

// ---------------------------------------------------------------------------------------------
// Device: one level of the periodic 2D DWT (rows then columns of the n x n band) per launch
// ---------------------------------------------------------------------------------------------
namespace {

// Forward level: a CTA makes the 16 x 16 tile (i0, j0) of each of the four subbands from the
// 46 x 46 input tile starting at (2 i0, 2 j0) (periodic in n): a_i = sum_k h_k x[(2i + k) mod n]
// along the rows into shared memory, then the same along the columns.  The three detail subbands
// go to det (Mallat positions of the band, pitch N, plane N^2); the LL subband to ll.
template <typename T>
__global__ void __launch_bounds__(256) dwt2_fwd_kernel(const T* __restrict__ in, int in_pitch, size_t in_plane,
                                                       T* __restrict__ det, int N, T* __restrict__ ll, int ll_pitch,
                                                       size_t ll_plane, int n, WaveFilt<T> f) {
  __shared__ T S[46][47];
  __shared__ T R[46][33];
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16, ch = blockIdx.z;
  const int tid = threadIdx.x;
  const T* src = in + (size_t)ch * in_plane;
  for (int idx = tid; idx < 46 * 46; idx += 256) {
    const int r = idx / 46, c = idx - r * 46;
    S[r][c] = src[(size_t)((2 * i0 + r) & (n - 1)) * in_pitch + ((2 * j0 + c) & (n - 1))];
  }
  __syncthreads();
  // rows: a thread makes the low and high outputs 2q and 2q + 1 of row r, which read the 18
  // inputs 4q .. 4q + 17 (four outputs per 18 shared-memory loads instead of one per 16)
  for (int it = tid; it < 46 * 8; it += 256) {
    const int r = it >> 3, q = it & 7;
    T x[18];
#pragma unroll
    for (int m = 0; m < 18; ++m) x[m] = S[r][4 * q + m];
    T l0 = T(0), h0 = T(0), l1 = T(0), h1 = T(0);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      l0 = fma(f.h[k], x[k], l0);
      h0 = fma(f.g[k], x[k], h0);
      l1 = fma(f.h[k], x[k + 2], l1);
      h1 = fma(f.g[k], x[k + 2], h1);
    }
    R[r][2 * q] = l0;
    R[r][2 * q + 1] = l1;
    R[r][16 + 2 * q] = h0;
    R[r][16 + 2 * q + 1] = h1;
  }
  __syncthreads();
  // columns: the same on the output rows 2q, 2q + 1 of column o (one item per thread)
  const int half = n / 2;
  {
    const int q = tid >> 5, o = tid & 31;
    T x[18];
#pragma unroll
    for (int m = 0; m < 18; ++m) x[m] = R[4 * q + m][o];
    T v[4] = {T(0), T(0), T(0), T(0)};  // low 2q, low 2q + 1, high 2q, high 2q + 1
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      v[0] = fma(f.h[k], x[k], v[0]);
      v[1] = fma(f.h[k], x[k + 2], v[1]);
      v[2] = fma(f.g[k], x[k], v[2]);
      v[3] = fma(f.g[k], x[k + 2], v[3]);
    }
    const int cb = o >> 4, col = j0 + (o & 15);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int rb = e >> 1, row = i0 + 2 * q + (e & 1);
      if (rb == 0 && cb == 0) ll[(size_t)ch * ll_plane + (size_t)row * ll_pitch + col] = v[e];
      else det[(size_t)ch * N * N + (size_t)(rb * half + row) * N + cb * half + col] = v[e];
    }
  }
}

// Inverse level (the transpose): a CTA makes the 32 x 32 output tile (y0, x0) of the n x n band
// from the 23 x 23 coefficient tiles of the four subbands starting at (y0/2 - 7, x0/2 - 7)
// (periodic in n/2): x_j = sum over k = j mod 2 of h_k a_i + g_k d_i, i = (j - k)/2, first along
// the columns, then along the rows.  LL comes from ll, the details from det (Mallat positions).
template <typename T>
__global__ void __launch_bounds__(256) dwt2_inv_kernel(const T* __restrict__ ll, int ll_pitch, size_t ll_plane,
                                                       const T* __restrict__ det, int N, T* __restrict__ out,
                                                       int out_pitch, size_t out_plane, int n, WaveFilt<T> f) {
  __shared__ T C[4][23][24];  // subband rb * 2 + cb
  __shared__ T V[2][32][24];  // after the column inverse: [cb][output row][coefficient column]
  const int y0 = blockIdx.y * 32, x0 = blockIdx.x * 32, ch = blockIdx.z;
  const int tid = threadIdx.x, half = n / 2;
  for (int idx = tid; idx < 4 * 23 * 23; idx += 256) {
    const int sb = idx / 529, rem = idx - sb * 529, a = rem / 23, b = rem - a * 23;
    const int ri = (y0 / 2 - 7 + a + half) & (half - 1), ci = (x0 / 2 - 7 + b + half) & (half - 1);
    const int rb = sb >> 1, cb = sb & 1;
    C[sb][a][b] = sb == 0 ? ll[(size_t)ch * ll_plane + (size_t)ri * ll_pitch + ci]
                          : det[(size_t)ch * N * N + (size_t)(rb * half + ri) * N + cb * half + ci];
  }
  __syncthreads();
  // columns: a thread makes the outputs jj = 4p .. 4p + 3 of coefficient column b, which read the
  // coefficient rows a = 2p .. 2p + 8 of both subbands (four outputs per 18 loads instead of 16 each)
  for (int it = tid; it < 2 * 8 * 23; it += 256) {
    const int cb = it / (8 * 23), rem = it - cb * 8 * 23, p = rem / 23, b = rem - p * 23;
    T cl[9], chh[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      cl[m] = C[cb][2 * p + m][b];
      chh[m] = C[2 + cb][2 * p + m][b];
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T acc = T(0);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int k = e + 2 * t, m = d + 7 - t;  // a = 2p + d - t + 7
          acc = fma(f.h[k], cl[m], acc);
          acc = fma(f.g[k], chh[m], acc);
        }
        V[cb][4 * p + 2 * d + e][b] = acc;
      }
    }
  }
  __syncthreads();
  // rows: the same along the row, outputs xx = 4p .. 4p + 3 of output row jj (one item per thread)
  {
    const int jj = tid >> 3, p = tid & 7;
    T v0[9], v1[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      v0[m] = V[0][jj][2 * p + m];
      v1[m] = V[1][jj][2 * p + m];
    }
    T* o = out + (size_t)ch * out_plane + (size_t)(y0 + jj) * out_pitch + x0 + 4 * p;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T acc = T(0);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int k = e + 2 * t, m = d + 7 - t;
          acc = fma(f.h[k], v0[m], acc);
          acc = fma(f.g[k], v1[m], acc);
        }
        o[2 * d + e] = acc;
      }
    }
  }
}

// Every level of a band of side n0 <= wave_fuse_n<T>() in one CTA per channel, in shared memory:
// the band (rows then columns per level, periodic in the current side n), its LL quadrant kept for
// the next level, the detail subbands to their Mallat positions in A (pitch N), the final 16 x 16
// LL to A's corner.  The same filtering as dwt2_fwd_kernel; only the tiling differs.
template <typename T>
__global__ void __launch_bounds__(512) dwt2_fwd_fused_kernel(const T* __restrict__ in, int in_pitch, size_t in_plane,
                                                             T* __restrict__ A, int N, int n0, WaveFilt<T> f) {
  extern __shared__ __align__(16) unsigned char wsm[];
  const int pp = n0 + 1;
  T* X = reinterpret_cast<T*>(wsm);  // [n0][n0 + 1]: the band of the current level
  T* R = X + (size_t)n0 * pp;          // [n0][n0 + 1]: after the row filters
  const int ch = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const T* src = in + (size_t)ch * in_plane;
  T* dst = A + (size_t)ch * N * N;
  for (int idx = tid; idx < n0 * n0; idx += nth) {
    const int r = idx / n0, c = idx - r * n0;
    X[r * pp + c] = src[(size_t)r * in_pitch + c];
  }
  __syncthreads();
  for (int n = n0; n >= 32; n >>= 1) {
    const int half = n / 2, qn = half / 2;
    // rows: low and high outputs 2q, 2q + 1 of row r from the inputs 4q .. 4q + 17 (mod n)
    for (int it = tid; it < n * qn; it += nth) {
      const int r = it / qn, q = it - r * qn;
      T x[18];
#pragma unroll
      for (int m = 0; m < 18; ++m) x[m] = X[r * pp + ((4 * q + m) & (n - 1))];
      T l0 = T(0), h0 = T(0), l1 = T(0), h1 = T(0);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        l0 = fma(f.h[k], x[k], l0);
        h0 = fma(f.g[k], x[k], h0);
        l1 = fma(f.h[k], x[k + 2], l1);
        h1 = fma(f.g[k], x[k + 2], h1);
      }
      R[r * pp + 2 * q] = l0;
      R[r * pp + 2 * q + 1] = l1;
      R[r * pp + half + 2 * q] = h0;
      R[r * pp + half + 2 * q + 1] = h1;
    }
    __syncthreads();
    // columns: the same on the output rows 2q, 2q + 1 of column o
    for (int it = tid; it < qn * n; it += nth) {
      const int q = it / n, o = it - q * n;
      T x[18];
#pragma unroll
      for (int m = 0; m < 18; ++m) x[m] = R[((4 * q + m) & (n - 1)) * pp + o];
      T v[4] = {T(0), T(0), T(0), T(0)};  // low 2q, low 2q + 1, high 2q, high 2q + 1
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        v[0] = fma(f.h[k], x[k], v[0]);
        v[1] = fma(f.h[k], x[k + 2], v[1]);
        v[2] = fma(f.g[k], x[k], v[2]);
        v[3] = fma(f.g[k], x[k + 2], v[3]);
      }
      const int cb = o < half ? 0 : 1, col = o & (half - 1);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int rb = e >> 1, ii = 2 * q + (e & 1);
        if (rb == 0 && cb == 0) {
          if (half == 16) dst[(size_t)ii * N + col] = v[e];
          else X[ii * pp + col] = v[e];
        } else {
          dst[(size_t)(rb * half + ii) * N + cb * half + col] = v[e];
        }
      }
    }
    __syncthreads();
  }
}

// The inverse of dwt2_fwd_fused_kernel: from the 16 x 16 LL in A's corner and the detail subbands
// (Mallat positions, pitch N) up to the band of side n0, in one CTA per channel: per level the
// column inverse then the row inverse of dwt2_inv_kernel over the whole band; the result of the
// last level goes to out (pitch out_pitch), the others stay in shared memory as the next LL.
template <typename T>
__global__ void __launch_bounds__(512) dwt2_inv_fused_kernel(const T* __restrict__ A, int N, T* __restrict__ out,
                                                             int out_pitch, size_t out_plane, int n0, WaveFilt<T> f) {
  extern __shared__ __align__(16) unsigned char wsm[];
  const int q0 = n0 / 2, qp = q0 + 1;
  T* C = reinterpret_cast<T*>(wsm);  // [4][q0][q0 + 1]: subband rb * 2 + cb of the current level
  T* V = C + (size_t)4 * q0 * qp;      // [2][n0][q0 + 1]: after the column inverse
  const int ch = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const T* a = A + (size_t)ch * N * N;
  for (int idx = tid; idx < 16 * 16; idx += nth) C[(idx >> 4) * qp + (idx & 15)] = a[(size_t)(idx >> 4) * N + (idx & 15)];
  for (int n = 32; n <= n0; n <<= 1) {
    const int half = n / 2, hh = half * half;
    for (int idx = tid; idx < 3 * hh; idx += nth) {
      const int sb = 1 + idx / hh, rem = idx - (sb - 1) * hh, r = rem / half, c = rem - r * half;
      const int rb = sb >> 1, cb = sb & 1;
      C[((size_t)sb * q0 + r) * qp + c] = a[(size_t)(rb * half + r) * N + cb * half + c];
    }
    __syncthreads();
    // columns: outputs j = 4p .. 4p + 3 of coefficient column b from the coefficient rows
    // 2p - 7 .. 2p + 1 (mod half) of both subbands
    const int pn = n / 4;
    for (int it = tid; it < 2 * pn * half; it += nth) {
      const int cb = it / (pn * half), rem = it - cb * pn * half, p = rem / half, b = rem - p * half;
      T cl[9], chh[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const int ai = (2 * p + m - 7) & (half - 1);
        cl[m] = C[((size_t)cb * q0 + ai) * qp + b];
        chh[m] = C[((size_t)(2 + cb) * q0 + ai) * qp + b];
      }
#pragma unroll
      for (int d = 0; d < 2; ++d) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          T acc = T(0);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            acc = fma(f.h[e + 2 * t], cl[d + 7 - t], acc);
            acc = fma(f.g[e + 2 * t], chh[d + 7 - t], acc);
          }
          V[((size_t)cb * n0 + 4 * p + 2 * d + e) * qp + b] = acc;
        }
      }
    }
    __syncthreads();
    // rows: outputs x = 4p .. 4p + 3 of output row j
    for (int it = tid; it < n * pn; it += nth) {
      const int j = it / pn, p = it - j * pn;
      T v0[9], v1[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const int bb = (2 * p + m - 7) & (half - 1);
        v0[m] = V[(size_t)j * qp + bb];
        v1[m] = V[((size_t)n0 + j) * qp + bb];
      }
#pragma unroll
      for (int d = 0; d < 2; ++d) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          T acc = T(0);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            acc = fma(f.h[e + 2 * t], v0[d + 7 - t], acc);
            acc = fma(f.g[e + 2 * t], v1[d + 7 - t], acc);
          }
          const int x = 4 * p + 2 * d + e;
          if (n == n0) out[(size_t)ch * out_plane + (size_t)j * out_pitch + x] = acc;
          else C[(size_t)j * qp + x] = acc;
        }
      }
    }
    __syncthreads();
  }
}

// Per pixel over the M channels: w = C c (channel DCT), then Eq. solt_trans / Eq. subu_trans on
// w (or t = t_imp in import mode), q = t - u', and c <- C^T q in place.  Residual partial sums
// per block (the same five sums and order as the other prior passes) into partials[block].
template <typename T, int M>
__global__ void __launch_bounds__(256) wdct_shrink_kernel(T* __restrict__ coef, const ChanDCT<T> cmat,
                                                          const T* __restrict__ u_in, T* __restrict__ u_out,
                                                          T* __restrict__ tprev, const T* __restrict__ t_imp,
                                                          double* __restrict__ partials, int N, T tau, int flags) {
  __shared__ double red[8][kNPart];
  const T* cv = cmat.c;  // kernel parameter: constant-bank operands, the same for every thread
  const bool import_mode = (flags & PA_IMPORT) != 0;
  const bool resid = (flags & PA_RESID) != 0;
  const bool store_t = (flags & PA_STORE_T) != 0;
  const size_t plane = (size_t)N * N;
  T part[kNPart] = {T(0), T(0), T(0), T(0), T(0)};
  for (size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x; pix < plane; pix += (size_t)gridDim.x * blockDim.x) {
    T cin[M], q[M];
#pragma unroll
    for (int m = 0; m < M; ++m) cin[m] = import_mode ? T(0) : coef[(size_t)m * plane + pix];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      {
        T w = T(0);
#pragma unroll
        for (int m = 0; m < M; ++m) w = fma((T)cv[k * M + m], cin[m], w);
        const size_t g = (size_t)k * plane + pix;
        const T uo = u_in[g];
        T t, un;
        if (import_mode) {
          t = t_imp[g];
          un = uo;
          w = T(0);
        } else {
          const T v = w + uo;
          t = v > tau ? v - tau : (v < -tau ? v + tau : T(0));
          un = uo + w - t;
        }
        u_out[g] = un;
        if (resid) {
          const T r = w - t;
          part[0] = fma(r, r, part[0]);
          part[1] = fma(w, w, part[1]);
          part[2] = fma(t, t, part[2]);
          part[3] = fma(un, un, part[3]);
          const T dt = t - tprev[g];
          part[4] = fma(dt, dt, part[4]);
        }
        if (store_t) tprev[g] = t;
        q[k] = t - un;
      }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      T x = T(0);
#pragma unroll
      for (int k = 0; k < M; ++k) x = fma((T)cv[k * M + m], q[k], x);
      coef[(size_t)m * plane + pix] = x;
    }
  }
  if (!resid) return;
  double s[kNPart];
#pragma unroll
  for (int i = 0; i < kNPart; ++i) {
    s[i] = (double)part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < kNPart; ++i) red[warp][i] = s[i];
  __syncthreads();
  if (threadIdx.x < kNPart) {
    double acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    partials[(size_t)blockIdx.x * kNPart + threadIdx.x] = acc;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_dwt2_fwd(const T* in, int in_pitch, size_t in_plane, T* det, int N, T* ll, int ll_pitch,
                            size_t ll_plane, int n, int M, const WaveFilt<T>& f, cudaStream_t s) {
  if (n < 32 || n > N || (n & (n - 1))) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)(n / 32), (unsigned)(n / 32), (unsigned)M);
  dwt2_fwd_kernel<T><<<grid, 256, 0, s>>>(in, in_pitch, in_plane, det, N, ll, ll_pitch, ll_plane, n, f);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dwt2_inv(const T* ll, int ll_pitch, size_t ll_plane, const T* det, int N, T* out, int out_pitch,
                            size_t out_plane, int n, int M, const WaveFilt<T>& f, cudaStream_t s) {
  if (n < 32 || n > N || (n & (n - 1))) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)(n / 32), (unsigned)(n / 32), (unsigned)M);
  dwt2_inv_kernel<T><<<grid, 256, 0, s>>>(ll, ll_pitch, ll_plane, det, N, out, out_pitch, out_plane, n, f);
  return cudaGetLastError();
}

template <typename T> int wave_fuse_band(int N) { return N < wave_fuse_n<T>() ? N : wave_fuse_n<T>(); }

template <typename T>
cudaError_t launch_dwt2_fwd_fused(const T* in, int in_pitch, size_t in_plane, T* A, int N, int n0, int M,
                                  const WaveFilt<T>& f, cudaStream_t s) {
  if (n0 < 32 || n0 > wave_fuse_n<T>() || n0 > N || (n0 & (n0 - 1))) return cudaErrorInvalidValue;
  const size_t sm = 2 * (size_t)n0 * (n0 + 1) * sizeof(T);
  static PerDeviceOnce once;
  cudaError_t e = once([&] {
    return cudaFuncSetAttribute(dwt2_fwd_fused_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * (size_t)wave_fuse_n<T>() * (wave_fuse_n<T>() + 1) * sizeof(T)));
  });
  if (e != cudaSuccess) return e;
  dwt2_fwd_fused_kernel<T><<<M, 512, sm, s>>>(in, in_pitch, in_plane, A, N, n0, f);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dwt2_inv_fused(const T* A, int N, T* out, int out_pitch, size_t out_plane, int n0, int M,
                                  const WaveFilt<T>& f, cudaStream_t s) {
  if (n0 < 32 || n0 > wave_fuse_n<T>() || n0 > N || (n0 & (n0 - 1))) return cudaErrorInvalidValue;
  const size_t sm = 8 * (size_t)(n0 / 2) * (n0 / 2 + 1) * sizeof(T);  // C: 4 q (q + 1), V: 2 n0 (q + 1)
  static PerDeviceOnce once;
  cudaError_t e = once([&] {
    const int q = wave_fuse_n<T>() / 2;
    return cudaFuncSetAttribute(dwt2_inv_fused_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(8 * (size_t)q * (q + 1) * sizeof(T)));
  });
  if (e != cudaSuccess) return e;
  dwt2_inv_fused_kernel<T><<<M, 512, sm, s>>>(A, N, out, out_pitch, out_plane, n0, f);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wdct_shrink(T* coef, const ChanDCT<T>& cmat, const T* u_in, T* u_out, T* tprev, const T* t_imp,
                               double* partials, int blocks, int N, int M, T tau, int flags, cudaStream_t s) {
  if (blocks < 1) return cudaErrorInvalidValue;
  switch (M) {
#define WS_CASE(m)                                                                                              \
  case m:                                                                                                      \
    wdct_shrink_kernel<T, m><<<blocks, 256, 0, s>>>(coef, cmat, u_in, u_out, tprev, t_imp, partials, N, tau, flags); \
    break;
    WS_CASE(1) WS_CASE(2) WS_CASE(3) WS_CASE(4) WS_CASE(5) WS_CASE(6) WS_CASE(7) WS_CASE(8)
    WS_CASE(9) WS_CASE(10) WS_CASE(11) WS_CASE(12) WS_CASE(13) WS_CASE(14) WS_CASE(15) WS_CASE(16)
#undef WS_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_dwt2_fwd<float>(const float*, int, size_t, float*, int, float*, int, size_t, int, int,
                                            const WaveFilt<float>&, cudaStream_t);
template cudaError_t launch_dwt2_fwd<double>(const double*, int, size_t, double*, int, double*, int, size_t, int, int,
                                             const WaveFilt<double>&, cudaStream_t);
template cudaError_t launch_dwt2_inv<float>(const float*, int, size_t, const float*, int, float*, int, size_t, int,
                                            int, const WaveFilt<float>&, cudaStream_t);
template cudaError_t launch_dwt2_inv<double>(const double*, int, size_t, const double*, int, double*, int, size_t,
                                             int, int, const WaveFilt<double>&, cudaStream_t);
template int wave_fuse_band<float>(int);
template int wave_fuse_band<double>(int);
template cudaError_t launch_dwt2_fwd_fused<float>(const float*, int, size_t, float*, int, int, int,
                                                  const WaveFilt<float>&, cudaStream_t);
template cudaError_t launch_dwt2_fwd_fused<double>(const double*, int, size_t, double*, int, int, int,
                                                   const WaveFilt<double>&, cudaStream_t);
template cudaError_t launch_dwt2_inv_fused<float>(const float*, int, float*, int, size_t, int, int,
                                                  const WaveFilt<float>&, cudaStream_t);
template cudaError_t launch_dwt2_inv_fused<double>(const double*, int, double*, int, size_t, int, int,
                                                   const WaveFilt<double>&, cudaStream_t);
template cudaError_t launch_wdct_shrink<float>(float*, const ChanDCT<float>&, const float*, float*, float*, const float*,
                                               double*, int, int, int, float, int, cudaStream_t);
template cudaError_t launch_wdct_shrink<double>(double*, const ChanDCT<double>&, const double*, double*, double*,
                                                const double*, double*, int, int, int, double, int, cudaStream_t);

}  // namespace cip
