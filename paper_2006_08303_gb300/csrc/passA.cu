// Pass A: the fused prior pass of one ADMM iteration (Alg. 1 lines 5-6 and
// the T^H (t - u) term of the next x-update, Eq. solx_Trans_DFT).
//
// One CTA owns R consecutive image rows of one channel (plus one halo row on
// each side for TV).  It
//   1. loads the row half-spectra of x (written by pass B) and inverts the row
//      DFT two rows at a time (one complex FFT z = x_a + i x_b for two real
//      rows, so shared memory holds the tile as row pairs);
//   2. applies the analysis operator T (anisotropic TV differences, 8x8
//      orthonormal block DCT, or identity), the soft-threshold t-update
//      (Eq. solt_trans) and the dual update (Eq. subu_trans), writing u; every
//      thread works on both rows of a pair, so shared-memory accesses are
//      whole 8- or 16-byte pairs;
//   3. forms q = (rho/2) T^T (t - u) and takes its forward row DFT, writing
//      the row half-spectra that pass B turns into the full 2D DFT.
// Optionally it stores t (for the next iteration's dual residual) and writes
// per-CTA partial sums of the residual norms (Eq. paramS quantities).
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

#ifndef PASSA_RT32
#define PASSA_RT32 48
#endif

template <typename T>
__device__ __forceinline__ void block_reduce_store(const T (&v)[kNPart], double* out) {
  __shared__ double red[32][kNPart];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s[kNPart];
#pragma unroll
  for (int i = 0; i < kNPart; ++i) {
    double x = (double)v[i];
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

// FFT elements per thread: 8 for complex64 up to N = 1024 (more warps per
// tile), 16 otherwise (keeps the CTA within 1024 threads).
// (complex64 DCT / l1 tiles at N = 512 take 16: one warp per row-pair FFT, whose stage
// barriers are then warp syncs, while TV, which needs more registers for its halo rows,
// takes 8.)  Variant V = 1 of a complex64 iteration kernel at N = 256 .. 1024 takes the other
// of 8 and 16; the plan's autotuner times both inside whole iterations and keeps the faster.
template <typename T> constexpr int elems_a(int N, int prior, int V = 0) {
  const int e = (sizeof(T) == 4 && N <= 1024) ? ((N == 512 && !prior_is_tv(prior)) ? 16 : 8) : 16;
  return V == 1 ? 24 - e : e;
}
template <typename T> constexpr bool has_variant(int N, int prior) {
  return sizeof(T) == 4 && N >= 256 && N <= 1024 && prior < ROWS_OUT && prior != PRIOR_WDCT;
}

// Pitch of the row-pair FFT buffers (complex elements): the padded FFT layout plus 4 slots from
// N = 256 on, so that the 4 or 5 buffers a warp writes at once (pair p, consecutive columns k,
// when the column-layout spectra are gathered or scattered) start in different bank groups.
constexpr int zs_of(int N) { return spad(N) + (N >= 256 ? 4 : 0); }

// rows per tile
template <typename T> constexpr int rows_for(int N, int prior) {
  if (!prior_is_tv(prior)) return 8;
  using C = typename CT<T>::type;
  for (int R = 8; R >= 2; R /= 2) {
    size_t zs = (size_t)zs_of(N);
    size_t sm = (size_t)((R + 2) / 2) * zs * sizeof(C) + (size_t)(2 * R + 1) * N * sizeof(T);
    if (sm <= 200 * 1024) return R;
  }
  return 2;
}

// DCT and l1 tiles stage their R rows of u in shared memory with one TMA bulk
// copy issued before the grid dependency (u does not depend on the preceding
// column pass), when the staging area keeps the CTA within ~100 KB
template <typename T> constexpr bool u_staged(int N, int prior, int R) {
  using C = typename CT<T>::type;
  return !prior_is_tv(prior) && prior < ROWS_OUT &&
         (size_t)(R / 2) * zs_of(N) * sizeof(C) + (size_t)R * N * sizeof(T) <= 100 * 1024;
}

template <typename T> constexpr size_t smem_for(int N, int prior, int R) {
  using C = typename CT<T>::type;
  const int halo = prior_is_tv(prior) ? 1 : 0;
  size_t sm = (size_t)((R + 2 * halo) / 2) * zs_of(N) * sizeof(C);
  if (prior_is_tv(prior)) sm += (size_t)(2 * R + 1) * N * sizeof(T);
  if (u_staged<T>(N, prior, R)) sm += (size_t)R * N * sizeof(T);
  return sm;
}

template <typename T> constexpr int threads_for(int N, int prior, int R, int V = 0) {
  const int npin = (R + (prior_is_tv(prior) ? 2 : 0)) / 2;
  const int n = npin * (N / elems_a<T>(N, prior, V));
  return ((n + 31) / 32) * 32;
}

// CTAs per SM the register budget is cut for: as many as shared memory and the
// thread limit allow, at <= ~48 registers per thread for complex64 (so that a
// 10-channel 512 x 512 prior pass runs as one wave) and <= ~168 for complex128
// (whose 16-element FFT registers would otherwise spill).
template <typename T> constexpr int minblocks_for(int nth, size_t smem) {
  const int by_regs = 65536 / (nth * (sizeof(T) == 4 ? PASSA_RT32 : 168));
  const int by_smem = (int)((227 * 1024) / (smem + 1024));
  const int by_thr = 2048 / nth;
  int b = by_regs < by_smem ? by_regs : by_smem;
  b = b < by_thr ? b : by_thr;
  b = b < 16 ? b : 16;  // small tiles (N <= 128): no point in squeezing registers further
  return b < 1 ? 1 : b;
}

// 8-point orthonormal DCT-II and its inverse through the even/odd split of
// the basis (row k of the matrix d[k*8+n] is symmetric in n <-> 7-n for even
// k and antisymmetric for odd k; rows 0, 4 are also symmetric and rows 2, 6
// antisymmetric in n <-> 3-n): 36 operations per transform instead of 64.
template <typename T>
__device__ __forceinline__ void dct8_fwd(const T* __restrict__ d, const T (&x)[8], T (&X)[8]) {
  T s[4], df[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    s[n] = x[n] + x[7 - n];
    df[n] = x[n] - x[7 - n];
  }
  const T s03 = s[0] + s[3], s12 = s[1] + s[2], e0 = s[0] - s[3], e1 = s[1] - s[2];
  X[0] = d[0] * (s03 + s12);
  X[4] = d[32] * (s03 - s12);
  X[2] = fma(d[16], e0, d[17] * e1);
  X[6] = fma(d[48], e0, d[49] * e1);
#pragma unroll
  for (int k = 1; k < 8; k += 2) {
    T acc = d[k * 8] * df[0];
#pragma unroll
    for (int n = 1; n < 4; ++n) acc = fma(d[k * 8 + n], df[n], acc);
    X[k] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void dct8_inv(const T* __restrict__ d, const T (&X)[8], T (&x)[8]) {
  const T a = d[0] * X[0], b = d[32] * X[4];
  const T A = a + b, B = a - b;
  const T C0 = fma(d[16], X[2], d[48] * X[6]), C1 = fma(d[17], X[2], d[49] * X[6]);
  const T e[4] = {A + C0, B + C1, B - C1, A - C0};
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    T o = d[8 + n] * X[1];
    o = fma(d[24 + n], X[3], o);
    o = fma(d[40 + n], X[5], o);
    o = fma(d[56 + n], X[7], o);
    x[n] = e[n] + o;
    x[7 - n] = e[n] - o;
  }
}

// the same on the two rows of a pair (real and imaginary parts)
template <typename T, bool FWD, typename C>
__device__ __forceinline__ void dct8_pair(const T* __restrict__ d, const C (&in)[8], C (&out)[8]) {
  T a[8], b[8], ra[8], rb[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    a[n] = in[n].x;
    b[n] = in[n].y;
  }
  if (FWD) {
    dct8_fwd(d, a, ra);
    dct8_fwd(d, b, rb);
  } else {
    dct8_inv(d, a, ra);
    dct8_inv(d, b, rb);
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) out[n] = mk<C>(ra[n], rb[n]);
}

template <typename T>
__device__ __forceinline__ void shrink(T w, T u, T tau, T& t, T& un) {
  t = soft(w + u, tau);
  un = u + w - t;
}

template <typename T>
__device__ __forceinline__ void acc_resid(T (&part)[kNPart], T w, T t, T un, const T* tprev, size_t g) {
  // a thread sums a few dozen terms at most, so the plan's precision suffices here; the
  // block and grid reductions run in double (FP64 issue is scarce on this part)
  const T r = w - t;
  part[0] = fma(r, r, part[0]);
  part[1] = fma(w, w, part[1]);
  part[2] = fma(t, t, part[2]);
  part[3] = fma(un, un, part[3]);
  if (tprev) {
    const T dt = t - tprev[g];
    part[4] = fma(dt, dt, part[4]);
  }
}

template <typename T, int LOGN, int PRIOR, int R, int V>
__global__ void __launch_bounds__(threads_for<T>(1 << LOGN, PRIOR, R, V),
                                  minblocks_for<T>(threads_for<T>(1 << LOGN, PRIOR, R, V),
                                                   smem_for<T>(1 << LOGN, PRIOR, R)))
    passA_kernel(const PassAArgs<T> a) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int HALO = prior_is_tv(PRIOR) ? 1 : 0;
  constexpr int ROWS = R + 2 * HALO;
  constexpr int NPIN = ROWS / 2;
  constexpr int NPOUT = R / 2;
  constexpr int ZS = zs_of(N);
  constexpr int CP = col_pitch(N);
  constexpr int E = elems_a<T>(N, PRIOR, V);
  constexpr int TEAM = N / E;
  constexpr int NCOMP = prior_is_tv(PRIOR) ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* zb = reinterpret_cast<C*>(smem_raw);
  T* ah = reinterpret_cast<T*>(zb + NPIN * ZS);  // TV only: [R][N], a_h at tile rows 1..R
  T* av = ah + R * N;                             // TV only: [R+1][N], a_v at tile rows 0..R
  constexpr bool USTAGE = u_staged<T>(N, PRIOR, R);
  static_assert(!USTAGE || (NPIN * ZS * sizeof(C)) % 16 == 0, "the TMA destination must be 16-byte aligned");
  T* us = reinterpret_cast<T*>(zb + NPIN * ZS);   // DCT / l1 with USTAGE: [R][N] rows r0.. of u_in
  __shared__ unsigned long long ubar;

  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  const int m = blockIdx.y;
  const int r0 = blockIdx.x * R;
  constexpr bool ROWXF = PRIOR >= ROWS_OUT;  // row transform only (read-back, wavelet chain)
  const bool import_mode = PRIOR == ROWS_IN || (a.flags & PA_IMPORT) != 0;
  const bool resid = (a.flags & PA_RESID) != 0;
  const bool store_t = (a.flags & PA_STORE_T) != 0;
  const T tau = a.tau;
  const size_t plane = (size_t)N * N;
  const T* u_in = a.u_in ? a.u_in + (size_t)m * NCOMP * plane : nullptr;
  T* u_out = a.u_out ? a.u_out + (size_t)m * NCOMP * plane : nullptr;
  T* tprev = a.tprev ? a.tprev + (size_t)m * NCOMP * plane : nullptr;
  const T* timp = a.t_imp ? a.t_imp + (size_t)m * NCOMP * plane : nullptr;
  const T* tprev_rd = resid ? tprev : nullptr;
  T part[kNPart] = {T(0), T(0), T(0), T(0), T(0)};
  // false when this thread's bounded wait for the staged u rows gave up: it then reads u from
  // global memory (the same values), never the shared-memory rows the copy may not have written
  bool u_ok = true;

  auto grow = [&](int j) { return (r0 - HALO + j) & (N - 1); };

  if constexpr (USTAGE) {
    // u rows r0 .. r0+R-1 of this channel: one contiguous block (16-byte aligned: r0 is a
    // multiple of 8 and N >= 64), fetched by the TMA unit while the previous kernel drains
    if (tid == 0) {
      constexpr unsigned bytes = (unsigned)(R * N * sizeof(T));
      if (a.test_fault == 1) {
        // test of the bounded wait: two arrivals expected, one given, no copy issued, so the
        // phase never completes and nothing is in flight when the wait gives up
        mbar_init(&ubar, 2);
        mbar_arrive(&ubar);
      } else {
        mbar_init(&ubar, 1);
        mbar_arrive_expect_tx(&ubar, bytes);
        bulk_copy_g2s(us, u_in + (size_t)r0 * N, bytes, &ubar);
      }
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
  }
  // L2 prefetch of the u rows (and t_prev rows) read after the inverse FFT
  if (!ROWXF && tid < 2 * NCOMP && !(USTAGE && (tid & 1) == 0)) {
    const T* src = (tid & 1) ? tprev_rd : u_in;
    if (src) {
      const size_t comp = (size_t)(tid >> 1) * plane;
      prefetch_l2(src + comp + (size_t)r0 * N, (size_t)R * N * sizeof(T));
      if (HALO) prefetch_l2(src + comp + (size_t)grow(0) * N, (size_t)N * sizeof(T));
    }
  }

  grid_dep_wait();  // x (and u, t) of the previous kernels are complete from here on
  grid_dep_launch();
  if (!import_mode) {
    // 1. gather the row half-spectra of the tile (two rows per complex FFT) from the column
    //    layout and invert the row DFT; thread = (pair p, column k) with p fastest, so that a warp
    //    reads the contiguous row segments of a few columns
    const C* xh = a.xh + (size_t)m * CP;
    const size_t kstride = (size_t)a.M * CP;
    for (int idx = tid; idx < NPIN * H; idx += nth) {
      const int p = idx % NPIN, k = idx / NPIN;
      const C* col = xh + (size_t)k * kstride;
      C xa, xb;
      if constexpr (sizeof(C) == 8 && !HALO) {
        // rows r0 + 2p, r0 + 2p + 1: adjacent, 16-byte aligned (r0 even, CP even)
        const float4 v = *reinterpret_cast<const float4*>(col + r0 + 2 * p);
        xa = mk<C>(v.x, v.y);
        xb = mk<C>(v.z, v.w);
      } else {
        xa = col[grow(2 * p)];
        xb = col[grow(2 * p + 1)];
      }
      pair_spectrum_put(zb + p * ZS, N, k, xa, xb);
    }
    __syncthreads();
    {
      const int team = tid / TEAM;
      const TeamSync ts = make_team_sync(team, TEAM);
      if (ts.cta || team < NPIN)
        fft_team<C, LOGN, 1, E, +1>(zb + (team < NPIN ? team : 0) * ZS, tid % TEAM, a.tw, ts, team < NPIN);
    }
    __syncthreads();
  }
  if constexpr (PRIOR == ROWS_OUT) {
    // x rows r0 .. r0 + R - 1 of map m into u_out ([maps][N][N])
    for (int idx = tid; idx < NPIN * N; idx += nth) {
      const int p = idx / N, n = idx - p * N;
      const C z = zb[p * ZS + spad(n)];
      u_out[(size_t)(r0 + 2 * p) * N + n] = z.x;
      u_out[(size_t)(r0 + 2 * p + 1) * N + n] = z.y;
    }
    return;
  }

  // 2. analysis operator, shrinkage, dual update; 3. q = qscale T^T (t - u')
  if constexpr (prior_is_tv(PRIOR)) {
    // a_v at tile rows 0..R, a_h at tile rows 1..R; thread = (row pair p, column c)
    for (int idx = tid; idx < NPIN * N; idx += nth) {
      const int p = idx / N, c = idx - p * N;
      C z0 = mk<C>(0.0, 0.0), zr = z0, zd = z0;
      if (!import_mode) {
        z0 = zb[p * ZS + spad(c)];
        zr = zb[p * ZS + spad((c + 1) & (N - 1))];
        if (p + 1 < NPIN) zd = zb[(p + 1) * ZS + spad(c)];
      }
      const T x0[2] = {z0.x, z0.y};
      const T wv[2] = {z0.y - z0.x, zd.x - z0.y};
      const T wh[2] = {zr.x - z0.x, zr.y - z0.y};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j = 2 * p + s;
        if (j > R) continue;  // row R+1: neither component needed
        const size_t g = (size_t)grow(j) * N + c;
        T tv, uvn, th = T(0), uhn = T(0);
        if (import_mode) {
          tv = timp[plane + g];
          uvn = u_in[plane + g];
          if (j >= 1) {
            th = timp[g];
            uhn = u_in[g];
          }
        } else if constexpr (PRIOR == PRIOR_TV_ISO) {
          // isotropic TV: the pixel's two components shrink together (group soft threshold);
          // the halo row needs its horizontal component too, for the vertical one
          const T vh = wh[s] + u_in[g], vv = wv[s] + u_in[plane + g];
          const T nrm = sqrt(vh * vh + vv * vv);
          const T f = nrm > tau ? T(1) - tau / nrm : T(0);
          th = vh * f;
          tv = vv * f;
          uhn = vh - th;
          uvn = vv - tv;
        } else {
          shrink(wv[s], u_in[plane + g], tau, tv, uvn);
          if (j >= 1) shrink(wh[s], u_in[g], tau, th, uhn);
        }
        av[j * N + c] = tv - uvn;
        if (j >= 1) {
          u_out[plane + g] = uvn;
          ah[(j - 1) * N + c] = th - uhn;
          u_out[g] = uhn;
          if (resid) {
            acc_resid(part, wh[s], th, uhn, tprev_rd, g);
            acc_resid(part, wv[s], tv, uvn, tprev_rd ? tprev_rd + plane : nullptr, g);
          }
          if (store_t) {
            tprev[g] = th;
            tprev[plane + g] = tv;
          }
        }
        (void)x0;
      }
    }
    __syncthreads();
    // q at output rows jj = 0..R-1 (tile rows jj+1), written as row pairs
    for (int idx = tid; idx < NPOUT * N; idx += nth) {
      const int p = idx / N, c = idx - p * N;
      const int cm = (c - 1) & (N - 1);
      T q[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int jj = 2 * p + s;
        q[s] = (ah[jj * N + cm] - ah[jj * N + c] + av[jj * N + c] - av[(jj + 1) * N + c]) * a.qscale;
      }
      zb[p * ZS + spad(c)] = mk<C>(q[0], q[1]);
    }
    // Row frequencies k2 = 0 and 1 (kLowK = 2) of the two components of a = t - u' on the output
    // rows, as direct sums with the exact table twiddle exp(-2 pi i c / N), for the low-column
    // correction of the x-update (launch_passB_split): near DC the FP32 transforms of q = D^T a
    // carry a uniform rounding error that Psi^{-1} amplifies by ~1/g, while transforms of a itself
    // do not.  One warp per (row, component), lanes over the columns; layout [comp][k2][map][CP].
    static_assert(kLowK == 2, "the sums below form k2 = 0 and 1");
    if (a.lowbuf) {
      const int nw = nth >> 5, wid = tid >> 5, lane = tid & 31;
      for (int o = wid; o < R * 2; o += nw) {
        const int jj = o >> 1, comp = o & 1;
        const T* src = comp == 0 ? ah + jj * N : av + (jj + 1) * N;
        T s0 = T(0), re = T(0), im = T(0);
        for (int c = lane; c < N; c += 32) {
          const T v = src[c];
          const C w = ldg_tw(&a.tw[c * (kTwN / N)]);
          s0 += v;
          re = fma(v, (T)w.x, re);
          im = fma(v, (T)w.y, im);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s0 += __shfl_down_sync(0xffffffffu, s0, off);
          re += __shfl_down_sync(0xffffffffu, re, off);
          im += __shfl_down_sync(0xffffffffu, im, off);
        }
        if (lane == 0) {
          a.lowbuf[((size_t)(comp * kLowK + 0) * a.M + m) * CP + r0 + jj] = mk<C>(s0, 0.0);
          a.lowbuf[((size_t)(comp * kLowK + 1) * a.M + m) * CP + r0 + jj] = mk<C>(re, im);
        }
      }
    }
  } else if constexpr (PRIOR == PRIOR_DCT8) {
    if (!import_mode) {
      // row DCT of every 8-sample segment of both rows of a pair, in place
      for (int idx = tid; idx < NPOUT * (N / 8); idx += nth) {
        const int p = idx / (N / 8), c0 = (idx - p * (N / 8)) * 8;
        C v[8], o[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) v[n] = zb[p * ZS + spad(c0 + n)];
        dct8_pair<T, true>(a.dct, v, o);
#pragma unroll
        for (int n = 0; n < 8; ++n) zb[p * ZS + spad(c0 + n)] = o[n];
      }
      __syncthreads();
    }
    if constexpr (USTAGE) u_ok = mbar_wait_bounded(&ubar, 0, a.err, a.test_fault ? 64 : (1 << 22));
    // column DCT -> coefficients w; shrink; dual; inverse column DCT of (t - u')
    for (int idx = tid; idx < (R / 8) * N; idx += nth) {
      const int br = idx / N, c = idx - br * N;
      T v[8], w[8], d[8];
      if (!import_mode) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const C z = zb[(br * 4 + q) * ZS + spad(c)];
          v[2 * q] = z.x;
          v[2 * q + 1] = z.y;
        }
        dct8_fwd(a.dct, v, w);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const size_t g = (size_t)(r0 + br * 8 + k) * N + c;
        const T uo = (USTAGE && u_ok) ? us[(br * 8 + k) * N + c] : u_in[g];
        T t, un;
        if (import_mode) {
          t = timp[g];
          un = uo;
          w[k] = T(0);
        } else {
          shrink(w[k], uo, tau, t, un);
        }
        u_out[g] = un;
        d[k] = t - un;
        if (resid) acc_resid(part, w[k], t, un, tprev_rd, g);
        if (store_t) tprev[g] = t;
      }
      dct8_inv(a.dct, d, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) zb[(br * 4 + q) * ZS + spad(c)] = mk<C>(v[2 * q], v[2 * q + 1]);
    }
    __syncthreads();
    for (int idx = tid; idx < NPOUT * (N / 8); idx += nth) {
      const int p = idx / (N / 8), c0 = (idx - p * (N / 8)) * 8;
      C v[8], o[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) v[n] = zb[p * ZS + spad(c0 + n)];
      dct8_pair<T, false>(a.dct, v, o);
#pragma unroll
      for (int n = 0; n < 8; ++n) zb[p * ZS + spad(c0 + n)] = mk<C>(o[n].x * a.qscale, o[n].y * a.qscale);
    }
  } else if constexpr (PRIOR == ROWS_IN) {
    // q rows from real rows: zb = qscale (u_in[r0 + 2p], u_in[r0 + 2p + 1])
    for (int idx = tid; idx < NPOUT * N; idx += nth) {
      const int p = idx / N, n = idx - p * N;
      zb[p * ZS + spad(n)] = mk<C>(u_in[(size_t)(r0 + 2 * p) * N + n] * a.qscale,
                                   u_in[(size_t)(r0 + 2 * p + 1) * N + n] * a.qscale);
    }
  } else {  // PRIOR_L1: T = I
    if constexpr (USTAGE) u_ok = mbar_wait_bounded(&ubar, 0, a.err, a.test_fault ? 64 : (1 << 22));
    for (int idx = tid; idx < NPOUT * N; idx += nth) {
      const int p = idx / N, c = idx - p * N;
      const C z = zb[p * ZS + spad(c)];
      const T w[2] = {z.x, z.y};
      T q[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const size_t g = (size_t)(r0 + 2 * p + s) * N + c;
        const T uo = (USTAGE && u_ok) ? us[(2 * p + s) * N + c] : u_in[g];
        T t, un;
        if (import_mode) {
          t = timp[g];
          un = uo;
        } else {
          shrink(w[s], uo, tau, t, un);
        }
        u_out[g] = un;
        if (resid) acc_resid(part, import_mode ? T(0) : w[s], t, un, tprev_rd, g);
        if (store_t) tprev[g] = t;
        q[s] = (t - un) * a.qscale;
      }
      zb[p * ZS + spad(c)] = mk<C>(q[0], q[1]);
    }
  }
  __syncthreads();

  // 4. forward row DFT of q (two rows per FFT), 5. store row half-spectra
  {
    const int team = tid / TEAM;
    const TeamSync ts = make_team_sync(team, TEAM);
    if (ts.cta || team < NPOUT)
      fft_team<C, LOGN, 1, E, -1>(zb + (team < NPOUT ? team : 0) * ZS, tid % TEAM, a.tw, ts, team < NPOUT);
  }
  __syncthreads();
  // 5. scatter the row half-spectra of q into the column layout: rows r0 + 2p, r0 + 2p + 1 of
  //    column k are adjacent (one 16-byte store for complex64)
  C* qh = a.qh + (size_t)m * CP;
  const size_t qstride = (size_t)a.M * CP;
  for (int idx = tid; idx < NPOUT * H; idx += nth) {
    const int p = idx % NPOUT, k = idx / NPOUT;
    C qa, qb;
    pair_spectrum_get(zb + p * ZS, N, k, qa, qb);
    C* col = qh + (size_t)k * qstride + r0 + 2 * p;
    if constexpr (sizeof(C) == 8) {
      *reinterpret_cast<float4*>(col) = make_float4(qa.x, qa.y, qb.x, qb.y);
    } else {
      col[0] = qa;
      col[1] = qb;
    }
  }
  if (resid) block_reduce_store<T>(part, a.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNPart);
  if constexpr (USTAGE) {
    // a copy that was only late must not write this CTA's shared memory after the CTA ends
    if (tid == 0 && !u_ok && a.test_fault == 0) mbar_wait_bounded(&ubar, 0, a.err);
  }
}

template <typename T, int LOGN, int PRIOR, int V>
cudaError_t launchA(const PassAArgs<T>& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  constexpr int R = rows_for<T>(N, PRIOR);
  constexpr int nth = threads_for<T>(N, PRIOR, R, V);
  constexpr size_t sm = smem_for<T>(N, PRIOR, R);
  auto kern = passA_kernel<T, LOGN, PRIOR, R, V>;
  static PerDeviceOnce once;
  cudaError_t e = once([&] {
    if (sm > 48 * 1024) {
      cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (r != cudaSuccess) return r;
    }
    // the largest shared-memory carveout, so that the register-bound CTA count is reached
    return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
  });
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(N / R, a.M), dim3(nth), sm, s, 0, a);
}

template <typename T, int PRIOR>
cudaError_t dispatchA(const PassAArgs<T>& a, int N, cudaStream_t s) {
  if constexpr (has_variant<T>(256, PRIOR)) {
    if (a.variant == 1) {
      switch (N) {
        case 256: return launchA<T, 8, PRIOR, 1>(a, s);
        case 512: return launchA<T, 9, PRIOR, 1>(a, s);
        case 1024: return launchA<T, 10, PRIOR, 1>(a, s);
        default: break;
      }
    }
  }
  switch (N) {
    case 64: return launchA<T, 6, PRIOR, 0>(a, s);
    case 128: return launchA<T, 7, PRIOR, 0>(a, s);
    case 256: return launchA<T, 8, PRIOR, 0>(a, s);
    case 512: return launchA<T, 9, PRIOR, 0>(a, s);
    case 1024: return launchA<T, 10, PRIOR, 0>(a, s);
    case 2048: return launchA<T, 11, PRIOR, 0>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T> int passA_rows(int N, int prior) { return rows_for<T>(N, prior); }
template <typename T> size_t passA_smem(int N, int prior) { return smem_for<T>(N, prior, rows_for<T>(N, prior)); }

template <typename T> cudaError_t launch_passA(const PassAArgs<T>& a, int N, int prior, cudaStream_t s) {
  switch (prior) {
    case PRIOR_TV: return dispatchA<T, PRIOR_TV>(a, N, s);
    case PRIOR_TV_ISO: return dispatchA<T, PRIOR_TV_ISO>(a, N, s);
    case PRIOR_DCT8: return dispatchA<T, PRIOR_DCT8>(a, N, s);
    case PRIOR_L1: return dispatchA<T, PRIOR_L1>(a, N, s);
    case ROWS_OUT: return dispatchA<T, ROWS_OUT>(a, N, s);
    case ROWS_IN: return dispatchA<T, ROWS_IN>(a, N, s);
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
