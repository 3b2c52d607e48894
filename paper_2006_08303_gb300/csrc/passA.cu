// Pass A: the fused prior pass of one ADMM iteration (Alg. 1 lines 5-6 and
// the T^H (t - u) term of the next x-update, Eq. solx_Trans_DFT).
//
// One CTA owns R consecutive image rows of one channel (plus one halo row on
// each side for TV).  It
//   1. loads the row half-spectra of x (written by pass B) and inverts the row
//      DFT two rows at a time (one complex FFT for two real rows);
//   2. applies the analysis operator T (anisotropic TV differences, 8x8
//      orthonormal block DCT, or identity), the soft-threshold t-update
//      (Eq. solt_trans) and the dual update (Eq. subu_trans), writing u;
//   3. forms q = (rho/2) T^T (t - u) and takes its forward row DFT, writing
//      the row half-spectra that pass B turns into the full 2D DFT.
// Optionally it stores t (for the next iteration's dual residual) and writes
// per-CTA partial sums of the residual norms (Eq. paramS quantities).
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

template <typename T>
__device__ __forceinline__ void block_reduce_store(const double (&v)[kNPart], double* out) {
  __shared__ double red[32][kNPart];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s[kNPart];
#pragma unroll
  for (int i = 0; i < kNPart; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    s[i] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kNPart; ++i) red[warp][i] = s[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < kNPart; ++i) {
      double acc = 0.0;
      for (int w = 0; w < nw; ++w) acc += red[w][i];
      out[i] = acc;
    }
  }
}

template <typename T> struct PA {
  using C = typename CT<T>::type;
};

// rows per tile and smem size
template <typename T> constexpr int rows_for(int N, int prior) {
  if (prior != PRIOR_TV) return 8;
  using C = typename CT<T>::type;
  for (int R = 8; R >= 2; R /= 2) {
    size_t zs = (size_t)spad(N);
    size_t sm = (size_t)((R + 2) / 2) * zs * sizeof(C) + (size_t)(2 * R + 1) * N * sizeof(T);
    if (sm <= 200 * 1024) return R;
  }
  return 2;
}

template <typename T> size_t smem_for(int N, int prior, int R) {
  using C = typename CT<T>::type;
  const int halo = prior == PRIOR_TV ? 1 : 0;
  size_t sm = (size_t)((R + 2 * halo) / 2) * spad(N) * sizeof(C);
  if (prior == PRIOR_TV) sm += (size_t)(2 * R + 1) * N * sizeof(T);
  return sm;
}

template <typename T>
__device__ __forceinline__ T zget(const typename CT<T>::type* zb, int ZS, int j, int c) {
  const typename CT<T>::type& v = zb[(j >> 1) * ZS + spad(c)];
  return (j & 1) ? v.y : v.x;
}
template <typename T>
__device__ __forceinline__ void zset(typename CT<T>::type* zb, int ZS, int j, int c, T val) {
  typename CT<T>::type& v = zb[(j >> 1) * ZS + spad(c)];
  if (j & 1) v.y = val; else v.x = val;
}

// 8-point orthonormal DCT-II (FWD) or its inverse, matrix dct[k*8+n]
template <typename T, bool FWD>
__device__ __forceinline__ void dct8(const T* __restrict__ d, const T (&in)[8], T (&out)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    T acc = T(0);
#pragma unroll
    for (int n = 0; n < 8; ++n) acc = fma(FWD ? d[k * 8 + n] : d[n * 8 + k], in[n], acc);
    out[k] = acc;
  }
}

template <typename T, int LOGN, int PRIOR, int R>
__global__ void __launch_bounds__(512) passA_kernel(const PassAArgs<T> a) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int P = half_pitch(N);
  constexpr int HALO = PRIOR == PRIOR_TV ? 1 : 0;
  constexpr int ROWS = R + 2 * HALO;
  constexpr int NPIN = ROWS / 2;
  constexpr int NPOUT = R / 2;
  constexpr int ZS = spad(N);
  constexpr int TEAM = N / 16;
  constexpr int NCOMP = PRIOR == PRIOR_TV ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* zb = reinterpret_cast<C*>(smem_raw);
  T* ah = reinterpret_cast<T*>(zb + NPIN * ZS);  // TV only: [R][N]
  T* av = ah + R * N;                             // TV only: [R+1][N]

  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  const int m = blockIdx.y;
  const int r0 = blockIdx.x * R;
  const bool import_mode = (a.flags & PA_IMPORT) != 0;
  const bool resid = (a.flags & PA_RESID) != 0;
  const bool store_t = (a.flags & PA_STORE_T) != 0;
  const T tau = a.tau;
  const size_t plane = (size_t)N * N;
  const T* u_in = a.u_in + (size_t)m * NCOMP * plane;
  T* u_out = a.u_out + (size_t)m * NCOMP * plane;
  T* tprev = a.tprev ? a.tprev + (size_t)m * NCOMP * plane : nullptr;
  const T* timp = a.t_imp ? a.t_imp + (size_t)m * NCOMP * plane : nullptr;
  double part[kNPart] = {0.0, 0.0, 0.0, 0.0, 0.0};

  auto grow = [&](int j) { return (r0 - HALO + j) & (N - 1); };

  if (!import_mode) {
    // 1. load row half-spectra (two rows per complex FFT) and invert the row DFT
    const C* xh = a.xh + (size_t)m * N * P;
    for (int idx = tid; idx < NPIN * H; idx += nth) {
      const int p = idx / H, k = idx - p * H;
      const C xa = xh[(size_t)grow(2 * p) * P + k];
      const C xb = xh[(size_t)grow(2 * p + 1) * P + k];
      pair_spectrum_put(zb + p * ZS, N, k, xa, xb);
    }
    __syncthreads();
    {
      const int team = tid / TEAM;
      if (team < NPIN) fft_team<C, LOGN, 1, 16, +1>(zb + team * ZS, tid % TEAM, a.tw, make_team_sync(team, TEAM));
    }
    __syncthreads();
  }

  // 2. analysis operator, shrinkage, dual update; 3. q = qscale T^T (t - u')
  if constexpr (PRIOR == PRIOR_TV) {
    const T* uh_in = u_in;
    const T* uv_in = u_in + plane;
    for (int idx = tid; idx < (R + 1) * N; idx += nth) {
      const int j = idx / N, c = idx - j * N;
      const size_t g = (size_t)grow(j) * N + c;
      T x0 = T(0), wv = T(0), wh = T(0);
      if (!import_mode) {
        x0 = zget<T>(zb, ZS, j, c);
        wv = zget<T>(zb, ZS, j + 1, c) - x0;
      }
      // vertical component (rows j = 0..R; j = 0 is the halo row, not written)
      T tv, uvn;
      if (import_mode) {
        tv = timp[plane + g];
        uvn = uv_in[g];
      } else {
        const T uv = uv_in[g];
        tv = soft(wv + uv, tau);
        uvn = uv + wv - tv;
      }
      av[j * N + c] = tv - uvn;
      if (j >= 1) {
        u_out[plane + g] = uvn;
        T th, uhn;
        if (import_mode) {
          th = timp[g];
          uhn = uh_in[g];
        } else {
          wh = zget<T>(zb, ZS, j, (c + 1) & (N - 1)) - x0;
          const T uh = uh_in[g];
          th = soft(wh + uh, tau);
          uhn = uh + wh - th;
        }
        ah[(j - 1) * N + c] = th - uhn;
        u_out[g] = uhn;
        if (resid) {
          part[0] += (double)(wh - th) * (double)(wh - th) + (double)(wv - tv) * (double)(wv - tv);
          part[1] += (double)wh * wh + (double)wv * wv;
          part[2] += (double)th * th + (double)tv * tv;
          part[3] += (double)uhn * uhn + (double)uvn * uvn;
          if (tprev) {
            const T dh = th - tprev[g], dv = tv - tprev[plane + g];
            part[4] += (double)dh * dh + (double)dv * dv;
          }
        }
        if (store_t) {
          tprev[g] = th;
          tprev[plane + g] = tv;
        }
      }
    }
    __syncthreads();
    for (int idx = tid; idx < R * N; idx += nth) {
      const int jj = idx / N, c = idx - jj * N;
      const T q = ah[jj * N + ((c - 1) & (N - 1))] - ah[jj * N + c] + av[jj * N + c] - av[(jj + 1) * N + c];
      zset<T>(zb, ZS, jj, c, q * a.qscale);
    }
  } else if constexpr (PRIOR == PRIOR_DCT8) {
    if (!import_mode) {
      // row DCT of every 8-sample segment, in place (each thread owns its 8 slots)
      for (int idx = tid; idx < R * (N / 8); idx += nth) {
        const int j = idx / (N / 8), c0 = (idx - j * (N / 8)) * 8;
        T v[8], o[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) v[n] = zget<T>(zb, ZS, j, c0 + n);
        dct8<T, true>(a.dct, v, o);
#pragma unroll
        for (int n = 0; n < 8; ++n) zset<T>(zb, ZS, j, c0 + n, o[n]);
      }
      __syncthreads();
    }
    // column DCT -> coefficients w; shrink; dual; inverse column DCT of (t - u')
    for (int idx = tid; idx < (R / 8) * N; idx += nth) {
      const int br = idx / N, c = idx - br * N;
      T v[8], w[8], d[8];
      if (!import_mode) {
#pragma unroll
        for (int n = 0; n < 8; ++n) v[n] = zget<T>(zb, ZS, br * 8 + n, c);
        dct8<T, true>(a.dct, v, w);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const size_t g = (size_t)(r0 + br * 8 + k) * N + c;
        T t, un;
        if (import_mode) {
          t = timp[g];
          un = u_in[g];
        } else {
          const T u = u_in[g];
          t = soft(w[k] + u, tau);
          un = u + w[k] - t;
        }
        u_out[g] = un;
        d[k] = t - un;
        if (resid) {
          part[0] += (double)(w[k] - t) * (double)(w[k] - t);
          part[1] += (double)w[k] * w[k];
          part[2] += (double)t * t;
          part[3] += (double)un * un;
          if (tprev) {
            const T dt = t - tprev[g];
            part[4] += (double)dt * dt;
          }
        }
        if (store_t) tprev[g] = t;
      }
      dct8<T, false>(a.dct, d, v);
#pragma unroll
      for (int n = 0; n < 8; ++n) zset<T>(zb, ZS, br * 8 + n, c, v[n]);
    }
    __syncthreads();
    for (int idx = tid; idx < R * (N / 8); idx += nth) {
      const int j = idx / (N / 8), c0 = (idx - j * (N / 8)) * 8;
      T v[8], o[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) v[n] = zget<T>(zb, ZS, j, c0 + n);
      dct8<T, false>(a.dct, v, o);
#pragma unroll
      for (int n = 0; n < 8; ++n) zset<T>(zb, ZS, j, c0 + n, o[n] * a.qscale);
    }
  } else {  // PRIOR_L1: T = I
    for (int idx = tid; idx < R * N; idx += nth) {
      const int j = idx / N, c = idx - j * N;
      const size_t g = (size_t)(r0 + j) * N + c;
      T w = T(0), t, un;
      if (import_mode) {
        t = timp[g];
        un = u_in[g];
      } else {
        w = zget<T>(zb, ZS, j, c);
        const T u = u_in[g];
        t = soft(w + u, tau);
        un = u + w - t;
      }
      u_out[g] = un;
      if (resid) {
        part[0] += (double)(w - t) * (double)(w - t);
        part[1] += (double)w * w;
        part[2] += (double)t * t;
        part[3] += (double)un * un;
        if (tprev) {
          const T dt = t - tprev[g];
          part[4] += (double)dt * dt;
        }
      }
      if (store_t) tprev[g] = t;
      zset<T>(zb, ZS, j, c, (t - un) * a.qscale);
    }
  }
  __syncthreads();

  // 4. forward row DFT of q (two rows per FFT), 5. store row half-spectra
  {
    const int team = tid / TEAM;
    if (team < NPOUT) fft_team<C, LOGN, 1, 16, -1>(zb + team * ZS, tid % TEAM, a.tw, make_team_sync(team, TEAM));
  }
  __syncthreads();
  C* qh = a.qh + (size_t)m * N * P;
  for (int idx = tid; idx < NPOUT * H; idx += nth) {
    const int p = idx / H, k = idx - p * H;
    C qa, qb;
    pair_spectrum_get(zb + p * ZS, N, k, qa, qb);
    qh[(size_t)(r0 + 2 * p) * P + k] = qa;
    qh[(size_t)(r0 + 2 * p + 1) * P + k] = qb;
  }
  if (resid) block_reduce_store<T>(part, a.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNPart);
}

template <typename T, int LOGN, int PRIOR>
cudaError_t launchA(const PassAArgs<T>& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  constexpr int R = rows_for<T>(N, PRIOR);
  constexpr int HALO = PRIOR == PRIOR_TV ? 1 : 0;
  constexpr int NPIN = (R + 2 * HALO) / 2;
  constexpr int TEAM = N / 16;
  int nth = NPIN * TEAM;
  nth = ((nth + 31) / 32) * 32;
  if (nth < 128) nth = 128;
  const size_t sm = smem_for<T>(N, PRIOR, R);
  auto kern = passA_kernel<T, LOGN, PRIOR, R>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(N / R, a.M);
  kern<<<grid, nth, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int PRIOR>
cudaError_t dispatchA(const PassAArgs<T>& a, int N, cudaStream_t s) {
  switch (N) {
    case 64: return launchA<T, 6, PRIOR>(a, s);
    case 128: return launchA<T, 7, PRIOR>(a, s);
    case 256: return launchA<T, 8, PRIOR>(a, s);
    case 512: return launchA<T, 9, PRIOR>(a, s);
    case 1024: return launchA<T, 10, PRIOR>(a, s);
    case 2048: return launchA<T, 11, PRIOR>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T> int passA_rows(int N, int prior) { return rows_for<T>(N, prior); }
template <typename T> size_t passA_smem(int N, int prior) { return smem_for<T>(N, prior, rows_for<T>(N, prior)); }

template <typename T> cudaError_t launch_passA(const PassAArgs<T>& a, int N, int prior, cudaStream_t s) {
  switch (prior) {
    case PRIOR_TV: return dispatchA<T, PRIOR_TV>(a, N, s);
    case PRIOR_DCT8: return dispatchA<T, PRIOR_DCT8>(a, N, s);
    case PRIOR_L1: return dispatchA<T, PRIOR_L1>(a, N, s);
    default: return cudaErrorInvalidValue;
  }
}

template int passA_rows<float>(int, int);
template int passA_rows<double>(int, int);
template size_t passA_smem<float>(int, int);
template size_t passA_smem<double>(int, int);
template cudaError_t launch_passA<float>(const PassAArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_passA<double>(const PassAArgs<double>&, int, int, cudaStream_t);

}  // namespace cip
