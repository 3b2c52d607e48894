// Column pass on the column-contiguous spectrum layout (the x-update of
// Eq. solx_Trans_DFT: column DFT, per-frequency M x M solve, inverse column DFT).
//
// Between the two passes of an iteration the row-domain half spectra are kept
// as [k2][map][CP]: for each half-spectrum column k2 the N values of every map
// (channel) are contiguous, so that everything the column pass needs for one
// column -- q-hat of all channels, the packed factor Psi^{-1} and the data
// term xb, both already stored per column as [k2][plane][CP] -- is a handful
// of long contiguous runs.  The prior pass reads and writes that layout in
// R-row segments.
//
// Fused form (colpass_fused_kernel): one CTA per column k2.
//   * a producer warp streams the factor and data term of the column through a
//     ring of shared-memory stages (32 bins x (npk + M) planes per stage: two
//     bulk copies, since both are stored blocked by 32 bins of a column, see
//     binp), completed on mbarriers; the first stages, and the rest of the
//     column into L2, are requested before the grid dependency, since they do
//     not depend on the preceding prior pass;
//   * after the dependency it fetches q-hat of the M channels (one bulk copy
//     per channel) into the channel slots of the tile;
//   * one team per channel runs the forward column FFT in shared memory (first
//     stage straight from the bulk-copied data);
//   * every consumer warp solves 32 bins per ring stage, X = xb + Psi^{-1} Q
//     with the packed Hermitian factor, reading the M channel values of a bin
//     from the tile and writing the results back in place, then frees the
//     stage;
//   * one team per channel runs the inverse column FFT; its last stage writes
//     the natural-order results straight to global memory.
// Every channel value of a frequency is read from HBM once and written once,
// and the factor is read once (north of 60% of the iteration's bytes).
//
// Split form (colfft_cols_kernel + the per-bin solve of colsplit.cu): for
// tiles that do not fit in shared memory.
#include "fft.cuh"
#include "kernels.h"

namespace cip {

namespace {

// FFT elements per thread of one column FFT: one warp per FFT of 256..1024
// points in complex64 (so that the stage barriers are warp barriers), two warps
// at 2048; complex128 keeps 16 elements (register budget).
template <typename T> constexpr int cp_elems(int N) {
  if (sizeof(T) == 4) return N <= 256 ? 8 : (N == 512 ? 16 : 32);
  return N <= 128 ? 8 : 16;
}
template <typename T> constexpr int cp_team(int N) { return N / cp_elems<T>(N); }

// Channel slot stride of the fused tile (complex elements): the padded FFT
// layout, rounded to 16 bytes.
template <typename T> constexpr int cp_slot(int N) {
  return sizeof(T) == 4 ? ((spad(N) + 1) & ~1) : spad(N);
}

constexpr int kStageBins = 32;  // bins per ring stage (one warp, one bin per lane)
constexpr int kConsBar = 15;    // named barrier of the consumer warps

// Team barrier: a masked warp barrier for teams inside one warp, a named
// barrier (id 1 + team) for teams of several warps.
struct ColSync {
  int id, n;
  unsigned mask;
  __device__ __forceinline__ void operator()() const {
    if (n > 32) asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    else __syncwarp(mask);
  }
};
__device__ __forceinline__ ColSync col_sync(int team, int tt) {
  ColSync s;
  s.n = tt;
  s.id = 1 + team;
  if (tt >= 32) s.mask = 0xffffffffu;
  else s.mask = ((tt == 32) ? 0xffffffffu : ((1u << tt) - 1u)) << ((team * tt) & 31);
  return s;
}

__device__ __forceinline__ void consumer_bar(int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"n"(kConsBar), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// Column FFTs on the column layout: every (k2, map) column of N contiguous
// values is transformed in place or out of place (src may equal dst).  One
// team per column; the first stage reads global memory, the last writes it.
// Columns past ncols come from a second range (src2 -> dst2, ncols2 columns).
// ---------------------------------------------------------------------------
constexpr int kColThreads = 256;

template <typename T, int LOGN, int SIGN>
__global__ void __launch_bounds__(kColThreads) colfft_cols_kernel(const typename CT<T>::type* src,
                                                                  typename CT<T>::type* dst,
                                                                  const typename CT<T>::type* __restrict__ tw,
                                                                  int ncols, const typename CT<T>::type* src2,
                                                                  typename CT<T>::type* dst2, int ncols2) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN, E = cp_elems<T>(N), TT = N / E, TEAMS = kColThreads / TT;
  constexpr int CP = col_pitch(N), ZS = spad(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* zb = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x, team = tid / TT, tt = tid % TT;
  const int col = blockIdx.x * TEAMS + team;
  grid_dep_wait();
  grid_dep_launch();
  // idle teams (past the last column) still take part in the CTA-wide barriers of wide teams
  const bool active = col < ncols + ncols2;
  const bool second = active && col >= ncols;
  const C* s = second ? src2 + (size_t)(col - ncols) * CP : src + (size_t)(active ? col : 0) * CP;
  C* d = second ? dst2 + (size_t)(col - ncols) * CP : dst + (size_t)(active ? col : 0) * CP;
  C* buf = zb + team * ZS;
  const ColSync cs = col_sync(team, TT);
  auto in0 = [&](int i0, int off) { return s[i0 + off]; };
  auto outL = [&](int i0, int off, C v) {
    if (active) d[i0 + off] = v;
  };
  fft_team_io<C, LOGN, E, SIGN, false>(buf, tt, tw, cs, in0, outL);
}

template <typename T, int LOGN, int SIGN>
cudaError_t launch_cols(const typename CT<T>::type* src, typename CT<T>::type* dst, const typename CT<T>::type* tw,
                        int ncols, cudaStream_t s, const typename CT<T>::type* src2, typename CT<T>::type* dst2,
                        int ncols2) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN, TT = cp_team<T>(N), TEAMS = kColThreads / TT;
  const size_t sm = (size_t)TEAMS * spad(N) * sizeof(C);
  auto k = colfft_cols_kernel<T, LOGN, SIGN>;
  static PerDeviceOnce once;
  if (sm > 48 * 1024) {
    cudaError_t e = once([&] { return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); });
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k, dim3((ncols + ncols2 + TEAMS - 1) / TEAMS), dim3(kColThreads), sm, s, 0, src, dst, tw, ncols,
                    src2, dst2, ncols2);
}

// ---------------------------------------------------------------------------
// Fused column pass.
// ---------------------------------------------------------------------------
template <typename T> struct FusedShape {
  int N, M, npk, slot, cons_warps, threads, nstage, stages_per_col;
  size_t tile_bytes, stage_bytes, smem;
};

// shared-memory budget of one CTA: two CTAs per SM when the tile is small,
// else one with the largest ring that fits
template <typename T> FusedShape<T> fused_shape(int N, int M, size_t smem_cap) {
  using C = typename CT<T>::type;
  FusedShape<T> f{};
  f.N = N;
  f.M = M;
  f.npk = M * (M + 1) / 2;
  f.slot = cp_slot<T>(N);
  const int tt = cp_team<T>(N);
  f.cons_warps = (M * tt + 31) / 32;
  f.threads = 32 * (f.cons_warps + 1);
  f.stages_per_col = N / kStageBins;
  f.tile_bytes = (size_t)M * f.slot * sizeof(C);
  f.stage_bytes = (size_t)(f.npk + M) * kStageBins * sizeof(C);
  const size_t bars = 1024;  // mbarriers and alignment slack
  const size_t half = 110 * 1024;
  size_t budget = (f.tile_bytes + 2 * f.stage_bytes + bars <= half) ? half : smem_cap;
  int ns = (int)((budget - f.tile_bytes - bars) / f.stage_bytes);
  if (f.tile_bytes + bars > budget) ns = 0;
  if (ns > 8) ns = 8;
  if (ns > f.stages_per_col) ns = f.stages_per_col;
  f.nstage = ns;
  f.smem = f.tile_bytes + (size_t)ns * f.stage_bytes + bars;
  return f;
}

template <typename T> struct FusedArgs {
  using C = typename CT<T>::type;
  const C* qh;    // [H][S][CP] q-hat row spectra (column layout)
  C* xh;          // [H][S][CP] x-hat row spectra (column layout)
  const C* pinv;  // packed Psi^{-1} / N^2, blocked by 32 bins (binp, npk planes)
  const C* xb;    // data term / N^2 (or b for the plain FP32 method), blocked by 32 bins (M planes)
  const C* tw;
  int* err;       // set to 1 when a bounded wait gives up
  int M, S, npk, nstage, plain;
};

// threads of the fused kernel for up to MMAX channels (capped at the CTA limit; larger shapes
// are not launched), and two CTAs per SM for complex64 tiles up to 512 points
template <typename T, int LOGN, int MMAX> constexpr int fused_threads() {
  const int t = 32 * ((MMAX * cp_team<T>(1 << LOGN) + 31) / 32 + 1);
  return t < 1024 ? t : 1024;
}
template <typename T, int LOGN, int MMAX> constexpr int fused_minblocks() {
  return (sizeof(T) == 4 && LOGN <= 9 && MMAX <= 12) ? 2 : 1;
}

template <typename T, int LOGN, int MMAX>
__global__ void __launch_bounds__(fused_threads<T, LOGN, MMAX>(), fused_minblocks<T, LOGN, MMAX>())
    colpass_fused_kernel(const FusedArgs<T> a) {
  using C = typename CT<T>::type;
  constexpr int N = 1 << LOGN, E = cp_elems<T>(N), TT = N / E;
  constexpr int CP = col_pitch(N), SLOT = cp_slot<T>(N);
  constexpr int NSC = N / kStageBins;  // ring stages per column
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int M = a.M, npk = a.npk, NS = a.nstage;
  const int planes = npk + M;
  C* tile = reinterpret_cast<C*>(smem_raw);
  C* ring = tile + (size_t)M * SLOT;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + (size_t)NS * planes * kStageBins);
  unsigned long long* tfull = bars;
  unsigned long long* full = bars + 1;
  unsigned long long* empty = bars + 1 + NS;
  // failure flag of the CTA (a bounded wait gave up), in the dynamic area so that the kernel has
  // no static shared memory and the whole opt-in size is available to the tile and the ring
  volatile int& s_fail = *reinterpret_cast<volatile int*>(bars + 1 + 2 * NS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cons_warps = (M * TT + 31) / 32;
  const int k2 = blockIdx.x;
  if (tid == 0) {
    s_fail = 0;
    mbar_init(tfull, 1);
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
  }
  __syncthreads();

  if (warp == cons_warps) {
    // ---------------- producer warp ----------------
    // stage s = bin block s of the column: its npk factor planes and M data-term planes are two
    // contiguous runs of the blocked layouts, fetched by two bulk copies
    const unsigned fbytes = (unsigned)(npk * kStageBins * sizeof(C)), xbytes = (unsigned)(M * kStageBins * sizeof(C));
    auto issue_stage = [&](int s) {
      const int slot = s % NS;
      C* dstg = ring + (size_t)slot * planes * kStageBins;
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[slot], fbytes + xbytes);
        bulk_copy_g2s(dstg, a.pinv + binp(k2, 0, s * kStageBins, npk, N), fbytes, &full[slot]);
        bulk_copy_g2s(dstg + (size_t)npk * kStageBins, a.xb + binp(k2, 0, s * kStageBins, M, N), xbytes, &full[slot]);
      }
      __syncwarp();
    };
    int s = 0;
    for (; s < NS && s < NSC; ++s) issue_stage(s);  // independent of the preceding kernel
    // The rest of the column's factor and data term into L2 as well: the preceding prior pass is
    // compute-bound and leaves HBM bandwidth unused while this CTA waits for it (one contiguous
    // run each in the blocked layout; requests of at most 64 KB)
    if (lane == 0 && NSC > NS) {
      const size_t f0 = binp(k2, 0, NS * kStageBins, npk, N), f1 = binp(k2, 0, 0, npk, N) + (size_t)N * npk;
      const size_t x0 = binp(k2, 0, NS * kStageBins, M, N), x1 = binp(k2, 0, 0, M, N) + (size_t)N * M;
      for (size_t o = f0; o < f1; o += 8192) prefetch_l2(a.pinv + o, (f1 - o < 8192 ? f1 - o : 8192) * sizeof(C));
      for (size_t o = x0; o < x1; o += 8192) prefetch_l2(a.xb + o, (x1 - o < 8192 ? x1 - o : 8192) * sizeof(C));
    }
    grid_dep_wait();
    grid_dep_launch();
    if (lane == 0) mbar_arrive_expect_tx(tfull, (unsigned)(M * N * sizeof(C)));
    __syncwarp();
    for (int m = lane; m < M; m += 32)
      bulk_copy_g2s(tile + (size_t)m * SLOT, a.qh + ((size_t)k2 * a.S + m) * CP, N * sizeof(C), tfull);
    for (; s < NSC; ++s) {
      const int slot = s % NS;
      // one decision for the whole warp (s_fail may change while the lanes read it)
      const bool failed = __any_sync(0xffffffffu, s_fail != 0);
      if (failed || !mbar_wait_warp(&empty[slot], ((s / NS) - 1) & 1, a.err)) {
        if (lane == 0) s_fail = 1;
        break;  // nothing more is issued; the copies already issued are waited for below
      }
      issue_stage(s);
    }
    // every copy this warp issued has landed before the warp leaves (the CTA's shared memory
    // stays allocated while the consumers run; this keeps no copy in flight past a failure)
    const int issued = s;
    if (lane == 0) {
      for (int sl = 0; sl < NS && sl < issued; ++sl) {
        const int last = sl + ((issued - 1 - sl) / NS) * NS;  // last stage issued into slot sl
        mbar_wait_bounded(&full[sl], (last / NS) & 1, a.err);
      }
      mbar_wait_bounded(tfull, 0, a.err);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  grid_dep_wait();  // x-hat is read by the preceding prior pass: written only after it completed
  grid_dep_launch();
  const int ncons = cons_warps * 32;
  const int team = tid / TT, tt = tid % TT;
  const bool in_team = team < M;
  const ColSync cs = col_sync(team, TT);
  const bool have_q = mbar_wait_warp(tfull, 0, a.err);
  if (!have_q) s_fail = 1;
  // 1. forward column DFT of each channel slot (in place; first stage reads the bulk-copied data)
  if (in_team && have_q) {
    C* buf = tile + (size_t)team * SLOT;
    auto in0 = [&](int i0, int off) { return buf[i0 + off]; };
    auto outL = [&](int i0, int off, C v) { buf[i0 + off] = v; };
    fft_team_io<C, LOGN, E, -1, true>(buf, tt, a.tw, cs, in0, outL);
  }
  consumer_bar(ncons);
  // 2. per-frequency solve, 32 bins per ring stage.  Every ring slot has one owning warp, which
  //    consumes the slot's stages in order: a warp never waits on a phase of its slot while the
  //    one before it is outstanding, so the parity of the wait names exactly one phase.
  const int solvers = cons_warps < NS ? cons_warps : NS;
  if (warp < solvers) {
    for (int s = 0; s < NSC; ++s) {
      const int slot = s % NS;
      if (slot % solvers != warp) continue;
      const bool failed = __any_sync(0xffffffffu, s_fail != 0);  // uniform over the warp
      const bool ok = !failed && mbar_wait_warp(&full[slot], (s / NS) & 1, a.err);
      if (ok && have_q) {
        const C* stg = ring + (size_t)slot * planes * kStageBins + lane;
        const int k1 = s * kStageBins + lane;
        C r[MMAX], x[MMAX];
#pragma unroll
        for (int i = 0; i < MMAX; ++i) {
          if (i < M) {
            r[i] = tile[(size_t)i * SLOT + k1];
            x[i] = stg[(size_t)(npk + i) * kStageBins];
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
                const C pij = stg[(size_t)pk * kStageBins];
                ++pk;
                cfma(x[i], pij, r[j]);
                if (j != i) cfmac(x[j], pij, r[i]);
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < MMAX; ++i)
          if (i < M) tile[(size_t)i * SLOT + k1] = x[i];
      } else if (!ok) {
        s_fail = 1;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
  }
  consumer_bar(ncons);
  if (s_fail) return;
  // 3. inverse column DFT; the last stage writes x-hat of this column straight to global memory
  if (in_team) {
    C* buf = tile + (size_t)team * SLOT;
    C* dst = a.xh + ((size_t)k2 * a.S + team) * CP;
    auto in0 = [&](int i0, int off) { return buf[i0 + off]; };
    auto outL = [&](int i0, int off, C v) { dst[i0 + off] = v; };
    fft_team_io<C, LOGN, E, +1, false>(buf, tt, a.tw, cs, in0, outL);
  }
}

template <typename T, int LOGN, int MMAX>
cudaError_t launch_fused_m(const FusedArgs<T>& a, const FusedShape<T>& f, cudaStream_t s) {
  auto k = colpass_fused_kernel<T, LOGN, MMAX>;
  static PerDeviceOnce once;
  // the attribute is set to the largest size any shape of this instantiation may ask for
  cudaError_t e = once([&] {
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  });
  if (e != cudaSuccess) return e;
  return launch_pdl(k, dim3(f.N / 2 + 1), dim3(f.threads), f.smem, s, 0, a);
}

template <typename T, int LOGN>
cudaError_t launch_fused_n(const FusedArgs<T>& a, const FusedShape<T>& f, cudaStream_t s) {
  if (a.M <= 4) return launch_fused_m<T, LOGN, 4>(a, f, s);
  if (a.M <= 8) return launch_fused_m<T, LOGN, 8>(a, f, s);
  if (a.M <= 10) return launch_fused_m<T, LOGN, 10>(a, f, s);
  if (a.M <= 12) return launch_fused_m<T, LOGN, 12>(a, f, s);
  if (a.M <= 16) return launch_fused_m<T, LOGN, 16>(a, f, s);
  return cudaErrorInvalidValue;
}

size_t optin_smem() {
  int dev = 0, cap = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cap > 0 ? (size_t)cap : (size_t)227 * 1024;
}

}  // namespace

template <typename T> bool colpass_fused_fits(int N, int M) {
  const FusedShape<T> f = fused_shape<T>(N, M, optin_smem());
  return f.nstage >= 2 && f.smem <= optin_smem() && f.threads <= 1024;
}

template <typename T> size_t colpass_fused_smem(int N, int M) { return fused_shape<T>(N, M, optin_smem()).smem; }

template <typename T> cudaError_t launch_colpass_fused(const PassBArgs<T>& b, int S, int* err, cudaStream_t s) {
  const FusedShape<T> f = fused_shape<T>(b.N, b.M, optin_smem());
  if (f.smem > optin_smem()) return cudaErrorInvalidConfiguration;
  if (f.nstage < 2 || f.threads > 1024) return cudaErrorInvalidConfiguration;
  FusedArgs<T> a;
  a.qh = b.qh;
  a.xh = b.xh;
  a.pinv = b.pinv;
  a.xb = b.bhat;
  a.tw = b.tw;
  a.err = err;
  a.M = b.M;
  a.S = S;
  a.npk = f.npk;
  a.nstage = f.nstage;
  a.plain = b.plain;
  switch (b.N) {
    case 64: return launch_fused_n<T, 6>(a, f, s);
    case 128: return launch_fused_n<T, 7>(a, f, s);
    case 256: return launch_fused_n<T, 8>(a, f, s);
    case 512: return launch_fused_n<T, 9>(a, f, s);
    case 1024: return launch_fused_n<T, 10>(a, f, s);
    case 2048: return launch_fused_n<T, 11>(a, f, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_cols_fft(const typename CT<T>::type* src, typename CT<T>::type* dst,
                            const typename CT<T>::type* tw, int N, int maps, int sign, cudaStream_t s,
                            const typename CT<T>::type* src2, typename CT<T>::type* dst2, int ncols2) {
  const int ncols = (N / 2 + 1) * maps;
#define CIP_COLS(L) \
  return sign < 0 ? launch_cols<T, L, -1>(src, dst, tw, ncols, s, src2, dst2, ncols2) \
                  : launch_cols<T, L, 1>(src, dst, tw, ncols, s, src2, dst2, ncols2)
  switch (N) {
    case 64: CIP_COLS(6);
    case 128: CIP_COLS(7);
    case 256: CIP_COLS(8);
    case 512: CIP_COLS(9);
    case 1024: CIP_COLS(10);
    case 2048: CIP_COLS(11);
    default: return cudaErrorInvalidValue;
  }
#undef CIP_COLS
}

template bool colpass_fused_fits<float>(int, int);
template bool colpass_fused_fits<double>(int, int);
template size_t colpass_fused_smem<float>(int, int);
template size_t colpass_fused_smem<double>(int, int);
template cudaError_t launch_colpass_fused<float>(const PassBArgs<float>&, int, int*, cudaStream_t);
template cudaError_t launch_colpass_fused<double>(const PassBArgs<double>&, int, int*, cudaStream_t);
template cudaError_t launch_cols_fft<float>(const float2*, float2*, const float2*, int, int, int, cudaStream_t,
                                            const float2*, float2*, int);
template cudaError_t launch_cols_fft<double>(const double2*, double2*, const double2*, int, int, int, cudaStream_t,
                                             const double2*, double2*, int);

}  // namespace cip
