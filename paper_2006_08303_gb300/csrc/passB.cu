// Pass B: column DFT, per-frequency solve and inverse column DFT, fused
// (the x-update of Eq. solx_Trans_DFT).
//
// A thread-block cluster of M CTAs owns CC adjacent half-spectrum columns k2;
// CTA m of the cluster holds channel m's N x CC tile in its shared memory.
//   1. every CTA loads its channel's row-domain half spectra q and runs the
//      forward column DFTs of its CC columns (interleaved in smem);
//   2. cluster barrier; the bins of the tile are split over the M CTAs and
//      for each bin the thread reads the M channel values from the M CTAs'
//      shared memory (distributed shared memory), forms
//        X(w) = xb(w) + Psi^{-1}(w)/N^2 Q(w)
//      with the packed Hermitian M x M factor and the FP64-formed data term
//      xb = Psi^{-1} beta Lambda^H F y / N^2 (the same x-update by linearity),
//      and writes the M results back into the owners' shared memory;
//   3. cluster barrier; every CTA runs the inverse column DFTs and writes its
//      channel's row-domain half spectra of the new x.
// Each channel value of a bin is read from HBM once and written once; the
// factor and the data term are stored column-major per bin plane
// ([k2][plane][k1]) so that the bins of one column are contiguous.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace cip {

namespace {

template <typename T> constexpr int elems_for() { return sizeof(T) == 4 ? 8 : 16; }

template <typename T> int cols_for(int N, int M) {
  (void)M;
  if (N <= 128) return 4;
  if (N >= 2048) return 2;  // keeps the CTA at <= 512 threads
  return sizeof(T) == 4 ? 4 : 2;
}

#ifndef PASSB_RT
#define PASSB_RT 80
#endif

// register budget: at most ~PASSB_RT registers per thread so that several CTAs share an SM
constexpr int minblocks_b(int nt) {
  const int b = 65536 / (nt * PASSB_RT);
  return b < 1 ? 1 : (b > 32 ? 32 : b);
}

template <typename T, int LOGN, int CC, int MMAX>
__global__ void __launch_bounds__((1 << LOGN) * CC / elems_for<T>(),
                                  minblocks_b((1 << LOGN) * CC / elems_for<T>()))
    passB_kernel(const PassBArgs<T> a) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int P = half_pitch(N);
  constexpr int E = elems_for<T>();
  constexpr int NT = N * CC / E;  // threads = one team
  constexpr int CP = col_pitch(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int M = a.M;
  const int m = blockIdx.x;  // channel == rank in the cluster
  const int tid = threadIdx.x;
  const int c0 = blockIdx.y * CC;
  const size_t mplane = (size_t)N * P;
  const C* qh = a.qh + (size_t)m * mplane;

  // this CTA's share of the tile's bins, and an L2 prefetch of the factor and
  // data-term columns it will read in the solve (overlaps the forward FFT)
  const int nbins = N * CC;
  const int per = (nbins + M - 1) / M;
  const int b0 = m * per;
  const int b1 = min(nbins, b0 + per);
  const int npk = M * (M + 1) / 2;
  if (b1 > b0) {
    const int k1lo = b0 / CC, k1hi = (b1 - 1) / CC + 1;
    const size_t len = (size_t)(k1hi - k1lo) * sizeof(C);
    for (int s = tid; s < CC * (npk + M); s += NT) {
      const int c = s % CC, j = s / CC;
      const int k2 = c0 + c;
      if (k2 >= H) continue;
      const C* base = (j < npk) ? a.pinv + ((size_t)k2 * npk + j) * CP + k1lo
                                : a.bhat + ((size_t)k2 * M + (j - npk)) * CP + k1lo;
      prefetch_l2(base, len);
    }
  }

  grid_dep_wait();  // q of the preceding prior pass is complete from here on
  grid_dep_launch();
  for (int idx = tid; idx < N * CC; idx += NT) {
    const int n1 = idx / CC, c = idx - n1 * CC;
    const int k2 = c0 + c;
    buf[spad(idx)] = (k2 < H) ? qh[(size_t)n1 * P + k2] : mk<C>(0.0, 0.0);
  }
  TeamSync ts;
  ts.bar_id = 0;
  ts.nthreads = NT;
  ts.mask = 0xffffffffu;
  ts.cta = false;
  __syncthreads();
  fft_team<C, LOGN, CC, E, -1>(buf, tid, a.tw, ts);
  cluster.sync();

  // per-frequency solve over this CTA's share of the tile's bins
  for (int b = b0 + tid; b < b1; b += NT) {
    const int k1 = b / CC, c = b - k1 * CC;
    const int k2 = c0 + c;
    if (k2 >= H) continue;
    const C* pcol = a.pinv + ((size_t)k2 * npk) * CP + k1;  // plane stride CP
    const C* xcol = a.bhat + ((size_t)k2 * M) * CP + k1;
    C r[MMAX], x[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i) {
      if (i < M) {
        const C* peer = cluster.map_shared_rank(buf, i);
        r[i] = peer[spad(b)];
        x[i] = xcol[(size_t)i * CP];
        if (a.plain) {  // plain FP32 method: X = Pinv (b + Q)
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
            const C pij = pcol[(size_t)pk * CP];
            ++pk;
            cfma(x[i], pij, r[j]);
            if (j != i) cfmac(x[j], pij, r[i]);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < MMAX; ++i) {
      if (i < M) {
        C* peer = cluster.map_shared_rank(buf, i);
        peer[spad(b)] = x[i];
      }
    }
  }
  cluster.sync();
  fft_team<C, LOGN, CC, E, +1>(buf, tid, a.tw, ts);
  __syncthreads();
  C* xh = a.xh + (size_t)m * mplane;
  for (int idx = tid; idx < N * CC; idx += NT) {
    const int n1 = idx / CC, c = idx - n1 * CC;
    const int k2 = c0 + c;
    if (k2 < H) xh[(size_t)n1 * P + k2] = buf[spad(idx)];
  }
}

template <typename T, int LOGN, int CC, int MMAX>
cudaError_t launchB(const PassBArgs<T>& a, cudaStream_t s) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int NT = N * CC / elems_for<T>();
  const size_t sm = (size_t)spad(N * CC) * sizeof(C);
  auto kern = passB_kernel<T, LOGN, CC, MMAX>;
  static PerDeviceOnce once;
  cudaError_t e = once([&] {
    if (sm > 48 * 1024) {
      cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (r != cudaSuccess) return r;
    }
    return cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(a.M, (N / 2 + 1 + CC - 1) / CC, 1), dim3(NT), sm, s, (unsigned)a.M, a);
}

template <typename T, int LOGN, int CC>
cudaError_t dispatchB_m(const PassBArgs<T>& a, cudaStream_t s) {
  if (a.M <= 4) return launchB<T, LOGN, CC, 4>(a, s);
  if (sizeof(T) == 4) {
    if (a.M <= 8) return launchB<T, LOGN, CC, 8>(a, s);
    if (a.M <= 10) return launchB<T, LOGN, CC, 10>(a, s);
    if (a.M <= 12) return launchB<T, LOGN, CC, 12>(a, s);
  }
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
  (void)M;
  return (size_t)spad(N * cc) * sizeof(typename CT<T>::type);
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
