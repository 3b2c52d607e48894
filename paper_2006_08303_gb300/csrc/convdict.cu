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
//
// State between steps: theta = F g and F(g - e) (spectra of the filters on the torus and of the
// filters minus the scaled dual), and g itself on its P x P support.  One step:
//   dl_solve  per bin: d-hat from the normal equation summed over the channels, w = d-hat + e-hat
//             with e-hat = theta - F(g - e); per column, Y(a, k2) = sum_k1 w exp(2 pi i k1 a / N)
//             for the P support rows a (so that d + e at the support points is a short sum over k2)
//   dl_filter per filter: v = d + e on the support, g = v / ||v|| (Eq. g_admm), the partial DFT
//             G(a, k2) = sum_b g(a, b) exp(-2 pi i k2 b / N)
//   dl_spec   per bin: g-hat = sum_a exp(-2 pi i k1 a / N) G(a, k2); e-hat <- w - g-hat (Eq.
//             h_admm, reading R22), so F(g - e) = 2 g-hat - w; theta = g-hat; p = sum_l theta_l z_l
// The spatial d and e off the support are never formed: g is zero there and e is only ever needed
// through its spectrum.

// exp(-2 pi i j / N) (SIGN < 0) or exp(+2 pi i j / N) (SIGN > 0) for any integer j (N a power of
// two: j mod N is j & (N - 1) in two's complement)
template <int SIGN, typename C>
__device__ __forceinline__ C tw_at(const C* __restrict__ tw, int j, int N) {
  const int r = j & (N - 1);
  C t = ldg_tw(&tw[r * (kTwN / N)]);
  if (SIGN > 0) t.y = -t.y;
  return t;
}

// Warp reduce-scatter by recursive halving over PM entries per lane (PM a power of two <= 32): at
// xor distance O a lane keeps one half of its LIVE entries (the upper half when bit O of the lane
// is set) and adds its partner's copy of that half.  Afterwards v[0] of lane i holds the warp's sum
// of entry i >> log2(32 / PM), after PM - 1 + log2(32 / PM) exchanges (5 PM for separate sums).
template <int LIVE, int O, int PM, typename C>
__device__ __forceinline__ void reduce_scatter(C (&v)[PM], int lane) {
  if constexpr (LIVE > 1) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < LIVE / 2; ++i) {
      const C lo = v[i], hi = v[i + LIVE / 2];
      C keep = up ? hi : lo;
      const C send = up ? lo : hi;
      keep.x += __shfl_xor_sync(0xffffffffu, send.x, O);
      keep.y += __shfl_xor_sync(0xffffffffu, send.y, O);
      v[i] = keep;
    }
    reduce_scatter<LIVE / 2, O / 2>(v, lane);
  } else if constexpr (O >= 1) {
    v[0].x += __shfl_xor_sync(0xffffffffu, v[0].x, O);
    v[0].y += __shfl_xor_sync(0xffffffffu, v[0].y, O);
    reduce_scatter<1, O / 2>(v, lane);
  }
}

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// block sum of one double per thread (blockDim a multiple of 32, <= 1024; red holds a value per
// warp); every thread gets it
__device__ __forceinline__ double block_sum256(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read from a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Per frequency, one thread (k1 = block offset + thread, k2 = blockIdx.y, so that the warps read
// the column layout contiguously): the filter normal equation summed over the M channels,
// (sigma I + W W^H) d = b with W = [conj(zhat_{l,s})] (L x M) and b = W xhat + sigma F(g - e), by
// the Woodbury identity d = (b - W alpha) / sigma, (sigma I_M + W^H W) alpha = W^H b.  The L
// filters are streamed twice: once to accumulate W^H W and W^H b, once to form d; the M x M system
// is solved by Cholesky in registers.  Then w = d + e-hat is stored and its partial inverse DFT
// along k1 at the P support rows is summed over the CTA's bins (reduce-scatter across each warp);
// the last CTA of a column to finish adds the column's CTA sums in a fixed order, so the result
// does not depend on the order in which CTAs run.
template <typename T, int M, int PM>
__global__ void __launch_bounds__(kDLBlock) dl_solve_kernel(const DLArgs<T> a) {
  using C = typename CT<T>::type;
  static_assert(kDLBlock == 64, "two warps per CTA");
  const int N = a.N, L = a.L, P = a.P;
  const int CP = col_pitch(N), H = N / 2 + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kb = blockIdx.x, nkb = gridDim.x;
  const int k1 = kb * kDLBlock + tid, k2 = blockIdx.y;
  const T n2 = (T)N * (T)N;
  const T sigma = a.sigma;
  const C* zb = a.zcol + (size_t)k2 * M * L * CP + k1;  // z_{l,s} at zb[(s L + l) CP]
  const C* th = a.spec + (size_t)k2 * 2 * L * CP + k1;  // theta_l at th[l CP], F(g - e)_l at th[(L + l) CP]
  C x[M], c[M], G[M][M];
#pragma unroll
  for (int s = 0; s < M; ++s) {
    const C v = a.xcol[((size_t)k2 * M + s) * CP + k1];
    x[s] = mk<C>(v.x * n2, v.y * n2);
    c[s] = mk<C>(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < M; ++t) G[s][t] = mk<C>(0.0, 0.0);
  }
  // b_l = sigma F(g - e)_l + sum_s conj(z_{l,s}) x_s
  auto load_b = [&](int l, C (&z)[M]) {
    const C ge = __ldg(th + (size_t)(L + l) * CP);
    C b = mk<C>(sigma * ge.x, sigma * ge.y);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const C v = __ldg(zb + ((size_t)s * L + l) * CP);
      z[s] = mk<C>(v.x * n2, v.y * n2);
      cfmac(b, z[s], x[s]);
    }
    return b;
  };
#pragma unroll 4
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
        const C u = G[i][k], v = G[j][k];
        acc.x -= u.x * v.x + u.y * v.y;
        acc.y -= u.y * v.x - u.x * v.y;
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
  // exp(+2 pi i k1 (a - P/2) / N) for the support rows a < P (zero beyond P)
  const int cen = P / 2;
  C wa[PM];
#pragma unroll
  for (int i = 0; i < PM; ++i) wa[i] = i < P ? tw_at<+1>(a.tw, k1 * (i - cen), N) : mk<C>(0.0, 0.0);
  __shared__ C red[2][32][PM];  // [warp][l][a]
  constexpr int SH = ilog2c(32 / PM);
  const T isg = T(1) / sigma;
  C* wb = a.wcol + (size_t)k2 * L * CP + k1;
  // the operands of filter l + 1 are loaded while filter l is processed (one thread per bin leaves
  // few warps per SM, so the loads in flight per thread set the bandwidth)
  C zn[M], gen, tn;
  auto load_l = [&](int l) {
#pragma unroll
    for (int s = 0; s < M; ++s) zn[s] = __ldg(zb + ((size_t)s * L + l) * CP);
    gen = __ldg(th + (size_t)(L + l) * CP);
    tn = __ldg(th + (size_t)l * CP);
  };
  load_l(0);
#pragma unroll 1
  for (int l = 0; l < L; ++l) {
    C z[M];
#pragma unroll
    for (int s = 0; s < M; ++s) z[s] = mk<C>(zn[s].x * n2, zn[s].y * n2);
    const C ge = gen, t = tn;
    if (l + 1 < L) load_l(l + 1);
    // b_l = sigma F(g - e)_l + sum_s conj(z_{l,s}) x_s, then d -= conj(z_s) alpha_s
    C d = mk<C>(sigma * ge.x, sigma * ge.y);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      cfmac(d, z[s], x[s]);
      d.x -= z[s].x * al[s].x + z[s].y * al[s].y;
      d.y -= z[s].x * al[s].y - z[s].y * al[s].x;
    }
    // w = d-hat + e-hat, e-hat = theta - F(g - e)
    const C wl = mk<C>(fma(d.x, isg, t.x - ge.x), fma(d.y, isg, t.y - ge.y));
    wb[(size_t)l * CP] = wl;
    C v[PM];
#pragma unroll
    for (int i = 0; i < PM; ++i) v[i] = cmul(wl, wa[i]);
    reduce_scatter<PM, 16>(v, lane);
    if ((lane & ((1 << SH) - 1)) == 0) red[warp][l][lane >> SH] = v[0];
  }
  __syncthreads();
  C* yp = a.ypart + ((size_t)k2 * nkb + kb) * L * P;
  for (int i = tid; i < L * P; i += kDLBlock) {
    const int l = i / P, ai = i - l * P;
    const C s0 = red[0][l][ai], s1 = red[1][l][ai];
    yp[i] = mk<C>(s0.x + s1.x, s0.y + s1.y);
  }
  __shared__ int last;
  __threadfence();  // this CTA's sums are visible device-wide before it is counted
  __syncthreads();
  if (tid == 0) last = atomicAdd(&a.cnt[k2], 1) == nkb - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    const C* y0 = a.ypart + (size_t)k2 * nkb * L * P;
    for (int i = tid; i < L * P; i += kDLBlock) {
      C acc = mk<C>(0.0, 0.0);
      for (int b = 0; b < nkb; ++b) {
        const C v = __ldcg(y0 + (size_t)b * L * P + i);
        acc.x += v.x;
        acc.y += v.y;
      }
      const int l = i / P, ai = i - l * P;
      a.yfull[((size_t)l * P + ai) * H + k2] = acc;
    }
    if (tid == 0) a.cnt[k2] = 0;  // ready for the next step (stream order)
  }
}

// Per filter l = blockIdx.x: v = d + e at the P x P support points,
//   v(a, b) = N^-2 sum_k2 c_k2 Re[Y(a, k2) exp(2 pi i k2 (b - P/2) / N)]
// (c_k2 = 1 at k2 = 0 and N/2, 2 otherwise: the half spectrum of a real map); g = v / ||v||
// (Eq. g_admm: support and unit norm, reading R22); ||g - g_prev||^2 when a check follows; then the
// partial DFT G(a, k2) = sum_b g(a, b) exp(-2 pi i k2 (b - P/2) / N) for every k2.  Y of all
// support rows and the twiddles of every (k2, b) are staged in shared memory for `chunk` columns
// at a time (all H at once where they fit); kFiltSplit threads per output each take every
// kFiltSplit-th column, their partial sums added in a fixed order.
constexpr int kFiltThreads = 512, kFiltSplit = 4;
constexpr size_t kFiltSmem = 96 * 1024;
template <typename T> int filt_chunk(int N, int P) {
  const int H = N / 2 + 1;
  const int c = (int)(kFiltSmem / (2 * (size_t)P * sizeof(typename CT<T>::type)));
  return c < H ? c : H;
}
template <typename T>
__global__ void __launch_bounds__(kFiltThreads) dl_filter_kernel(const DLArgs<T> a, int chunk) {
  using C = typename CT<T>::type;
  const int N = a.N, L = a.L, P = a.P, H = N / 2 + 1, PP = P * P, cen = P / 2;
  const int l = blockIdx.x, tid = threadIdx.x;
  extern __shared__ __align__(16) unsigned char fsm[];
  C* ys = reinterpret_cast<C*>(fsm);  // [P][chunk]: Y(a, k2) of the chunk
  C* ws = ys + (size_t)P * chunk;       // [P][chunk]: exp(-2 pi i k2 (b - P/2) / N)
  __shared__ T vs[kDLMaxP * kDLMaxP];
  __shared__ T part[kFiltSplit][kFiltThreads / kFiltSplit];
  __shared__ double red[kFiltThreads / 32];
  const T inv_n = T(1) / ((T)N * (T)N);
  const C* Y = a.yfull + (size_t)l * P * H;
  const int sub = tid % kFiltSplit, o0 = tid / kFiltSplit;
  constexpr int OSTEP = kFiltThreads / kFiltSplit;
  auto stage = [&](int c0, int nc, bool with_y) {
    __syncthreads();  // the previous chunk is consumed
    for (int i = tid; i < P * nc; i += kFiltThreads) {
      const int r = i / nc, c = i - r * nc;
      if (with_y) ys[(size_t)r * chunk + c] = Y[(size_t)r * H + c0 + c];
      ws[(size_t)r * chunk + c] = tw_at<-1>(a.tw, (c0 + c) * (r - cen), N);
    }
    __syncthreads();
  };
  for (int ob = 0; ob < PP; ob += OSTEP) {  // outputs ob .. ob + OSTEP - 1 (one pass for P <= 11)
    const int o = ob + o0;
    const int ai = o < PP ? o / P : 0, bi = o < PP ? o - ai * P : 0;
    T acc = T(0);
    for (int c0 = 0; c0 < H; c0 += chunk) {
      const int nc = H - c0 < chunk ? H - c0 : chunk;
      if (ob == 0 || nc < H) stage(c0, nc, true);  // a single chunk is staged once
      if (o < PP) {
        for (int c = sub; c < nc; c += kFiltSplit) {
          const C y = ys[(size_t)ai * chunk + c], t = ws[(size_t)bi * chunk + c];  // Re(y conj(t))
          const int k2 = c0 + c;
          const T w = (k2 == 0 || k2 == N / 2) ? T(1) : T(2);
          acc = fma(w, fma(y.x, t.x, y.y * t.y), acc);
        }
      }
    }
    if (o < PP) part[sub][o0] = acc;
    __syncthreads();
    if (sub == 0 && o < PP) vs[o] = (((part[0][o0] + part[1][o0]) + part[2][o0]) + part[3][o0]) * inv_n;
    __syncthreads();
  }
  double nn = 0.0;
  for (int o = tid; o < PP; o += kFiltThreads) nn += (double)vs[o] * (double)vs[o];
  nn = block_sum256(nn, red);
  const T inv = nn > 0.0 ? (T)(1.0 / sqrt(nn)) : T(0);
  T* g = a.gs + (size_t)l * PP;
  double ds = 0.0;
  for (int o = tid; o < PP; o += kFiltThreads) {
    const T gn = vs[o] * inv;
    const double dg = (double)gn - (double)g[o];
    ds += dg * dg;
    g[o] = gn;
    vs[o] = gn;
  }
  if (a.check) {
    ds = block_sum256(ds, red);
    if (tid == 0) a.spart[l] = ds;
  }
  // G(a, k2) = sum_b g(a, b) ws[b][k2] over the same chunks (twiddles staged again when chunked)
  for (int c0 = 0; c0 < H; c0 += chunk) {
    const int nc = H - c0 < chunk ? H - c0 : chunk;
    if (nc < H) stage(c0, nc, false);
    else __syncthreads();  // vs is final
    for (int o = tid; o < P * nc; o += kFiltThreads) {
      const int ai = o / nc, c = o - ai * nc;
      C acc = mk<C>(0.0, 0.0);
      for (int bi = 0; bi < P; ++bi) {
        const T gv = vs[ai * P + bi];
        const C t = ws[(size_t)bi * chunk + c];
        acc.x = fma(gv, t.x, acc.x);
        acc.y = fma(gv, t.y, acc.y);
      }
      a.gfac[((size_t)(c0 + c) * L + l) * P + ai] = acc;
    }
  }
}

// Per frequency: g-hat_l = sum_a exp(-2 pi i k1 (a - P/2) / N) G_l(a, k2) = theta_l of the new
// filters; the dual update e-hat <- e-hat + d-hat - g-hat = w - g-hat (Eq. h_admm), stored as
// F(g - e) = 2 g-hat - w; p = sum_l theta_l z_l for the next x-update; and, before a check, the
// primal residual |F(d - g)|^2 = |w - e-hat_old - g-hat|^2 (Parseval on the half spectrum).
template <typename T, int M, int PM>
__global__ void __launch_bounds__(kDLBlock) dl_spec_kernel(const DLArgs<T> a) {
  using C = typename CT<T>::type;
  const int N = a.N, L = a.L, P = a.P, CP = col_pitch(N);
  const int tid = threadIdx.x;
  const int k1 = blockIdx.x * kDLBlock + tid, k2 = blockIdx.y;
  __shared__ C gk[32][PM];
  __shared__ double red[8];
  for (int i = tid; i < 32 * PM; i += kDLBlock) {
    const int l = i / PM, ai = i - l * PM;
    gk[l][ai] = (l < L && ai < P) ? a.gfac[((size_t)k2 * L + l) * P + ai] : mk<C>(0.0, 0.0);
  }
  __syncthreads();
  const int cen = P / 2;
  C wa[PM];
#pragma unroll
  for (int i = 0; i < PM; ++i) wa[i] = i < P ? tw_at<-1>(a.tw, k1 * (i - cen), N) : mk<C>(0.0, 0.0);
  C pm[M];
#pragma unroll
  for (int m = 0; m < M; ++m) pm[m] = mk<C>(0.0, 0.0);
  T r2 = T(0);
  C* th = a.spec + (size_t)k2 * 2 * L * CP + k1;
  const C* wb = a.wcol + (size_t)k2 * L * CP + k1;
  const C* zb = a.zcol + (size_t)k2 * M * L * CP + k1;
  // operands of filter l + 1 loaded while filter l is processed
  C wn = wb[0], zn[M];
#pragma unroll
  for (int m = 0; m < M; ++m) zn[m] = zb[(size_t)m * L * CP];
#pragma unroll 1
  for (int l = 0; l < L; ++l) {
    C gh = mk<C>(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < PM; ++i) cfma(gh, wa[i], gk[l][i]);
    const C w = wn;
    C z[M];
#pragma unroll
    for (int m = 0; m < M; ++m) z[m] = zn[m];
    if (l + 1 < L) {
      wn = wb[(size_t)(l + 1) * CP];
#pragma unroll
      for (int m = 0; m < M; ++m) zn[m] = zb[((size_t)m * L + l + 1) * CP];
    }
    if (a.check) {
      const C t0 = th[(size_t)l * CP], ge0 = th[(size_t)(L + l) * CP];
      const T dx = w.x - t0.x + ge0.x - gh.x, dy = w.y - t0.y + ge0.y - gh.y;
      r2 = fma(dx, dx, fma(dy, dy, r2));
    }
    th[(size_t)l * CP] = gh;
    th[(size_t)(L + l) * CP] = mk<C>(T(2) * gh.x - w.x, T(2) * gh.y - w.y);
#pragma unroll
    for (int m = 0; m < M; ++m) cfma(pm[m], gh, z[m]);
  }
#pragma unroll
  for (int m = 0; m < M; ++m) a.p_out[((size_t)k2 * M + m) * CP + k1] = pm[m];
  if (a.check) {
    const double wgt = (k2 == 0 || k2 == N / 2) ? 1.0 : 2.0;
    double v = wgt * (double)r2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) a.rpart[(size_t)k2 * gridDim.x + blockIdx.x] = red[0] + red[1];
  }
}

template <typename T>
__global__ void dl_rescale_kernel(typename CT<T>::type* __restrict__ spec, int L, int N, T f) {
  using C = typename CT<T>::type;
  const int CP = col_pitch(N), H = N / 2 + 1;
  const size_t total = (size_t)H * L * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % N);
    const size_t r = i / N;
    const int l = (int)(r % L);
    const size_t k2 = r / L;
    C* th = spec + (k2 * 2 * L + l) * CP + k1;
    const C t = th[0], ge = th[(size_t)L * CP];
    th[(size_t)L * CP] = mk<C>(t.x - (t.x - ge.x) * f, t.y - (t.y - ge.y) * f);
  }
}

template <typename T, int PM> cudaError_t dl_by_m(const DLArgs<T>& a, bool spec, cudaStream_t s) {
  const dim3 grid(a.N / kDLBlock, a.N / 2 + 1);
  switch (a.M) {
#define DL_CASE(m)                                                          \
  case m:                                                                   \
    if (spec) dl_spec_kernel<T, m, PM><<<grid, kDLBlock, 0, s>>>(a);        \
    else dl_solve_kernel<T, m, PM><<<grid, kDLBlock, 0, s>>>(a);            \
    break;
    DL_CASE(1) DL_CASE(2) DL_CASE(3) DL_CASE(4) DL_CASE(5) DL_CASE(6) DL_CASE(7) DL_CASE(8)
#undef DL_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template <typename T> bool dl_args_ok(const DLArgs<T>& a) {
  return a.N % kDLBlock == 0 && a.N <= kTwN && a.L >= 1 && a.L <= 32 && a.P >= 1 && a.P <= kDLMaxP &&
         a.P <= a.N && a.M >= 1 && a.M <= 8;
}

}  // namespace

template <typename T> cudaError_t launch_dl_solve(const DLArgs<T>& a, cudaStream_t s) {
  if (!dl_args_ok(a)) return cudaErrorInvalidValue;
  return a.P <= 16 ? dl_by_m<T, 16>(a, false, s) : dl_by_m<T, 32>(a, false, s);
}
template <typename T> cudaError_t launch_dl_filter(const DLArgs<T>& a, cudaStream_t s) {
  if (!dl_args_ok(a)) return cudaErrorInvalidValue;
  const int chunk = filt_chunk<T>(a.N, a.P);
  const size_t sm = 2 * (size_t)a.P * chunk * sizeof(typename CT<T>::type);
  static PerDeviceOnce once;
  cudaError_t e = once([&] {
    return cudaFuncSetAttribute(dl_filter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFiltSmem);
  });
  if (e != cudaSuccess) return e;
  dl_filter_kernel<T><<<a.L, kFiltThreads, sm, s>>>(a, chunk);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_dl_spec(const DLArgs<T>& a, cudaStream_t s) {
  if (!dl_args_ok(a)) return cudaErrorInvalidValue;
  return a.P <= 16 ? dl_by_m<T, 16>(a, true, s) : dl_by_m<T, 32>(a, true, s);
}
template <typename T>
cudaError_t launch_dl_rescale(typename CT<T>::type* spec, int L, int N, T f, cudaStream_t s) {
  dl_rescale_kernel<T><<<4 * 152, 256, 0, s>>>(spec, L, N, f);
  return cudaGetLastError();
}
template cudaError_t launch_dl_solve<float>(const DLArgs<float>&, cudaStream_t);
template cudaError_t launch_dl_solve<double>(const DLArgs<double>&, cudaStream_t);
template cudaError_t launch_dl_filter<float>(const DLArgs<float>&, cudaStream_t);
template cudaError_t launch_dl_filter<double>(const DLArgs<double>&, cudaStream_t);
template cudaError_t launch_dl_spec<float>(const DLArgs<float>&, cudaStream_t);
template cudaError_t launch_dl_spec<double>(const DLArgs<double>&, cudaStream_t);
template cudaError_t launch_dl_rescale<float>(float2*, int, int, float, cudaStream_t);
template cudaError_t launch_dl_rescale<double>(double2*, int, int, double, cudaStream_t);

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
