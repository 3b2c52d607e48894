// Shared-memory Stockham FFT for power-of-two lengths 64..2048 (sm_103a).
//
// The 2D DFTs of Section IV-A (F_2D on every slice, Eq. solx_Trans_DFT) are
// done as a row pass and a column pass; both run this 1D routine on data a
// CTA has staged in shared memory.  A "team" of NTH threads owns NF
// interleaved FFTs of length N (element n of FFT f sits at slot
// spad(n*NF + f)); each thread keeps E = N*NF/NTH elements in registers and
// applies radix-8 stages (plus one radix-2 or radix-4 stage when log2 N is
// not a multiple of 3).  Stage s reads x[t + r N/R], multiplies by the
// twiddles w_{Ls R}^{r (t mod Ls)}, does a radix-R DFT in registers and
// writes y[(t/Ls) Ls R + t mod Ls + r Ls] (autosorting Stockham, natural
// order in and out).  Twiddles come from a table of exp(-2 pi i k / 2048)
// computed on the host in FP64 and rounded once; a radix-8 butterfly loads
// only w^j and w^4j and forms w^2j, w^3j, w^5j, w^6j, w^7j by at most two
// complex products (a few ulp), since table loads stalled the stages.
#pragma once
#include "common.cuh"

namespace cip {



// Synchronisation of one team: the CTA-wide barrier (cta: every thread of the
// CTA runs the FFT, idle ones with active = false), a named barrier for teams
// wider than a warp, or a masked __syncwarp for teams inside one warp.
// Named barriers are a per-SM resource: a CTA that uses ids 0..k limits how
// many CTAs share an SM, so kernels with several teams per CTA use the
// CTA-wide form.
struct TeamSync {
  int bar_id;
  int nthreads;
  unsigned mask;
  bool cta;
  __device__ __forceinline__ void sync() const {
    if (cta) {
      __syncthreads();
    } else if (nthreads > 32) {
      asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
    } else {
      __syncwarp(mask);
    }
  }
};

// Team of `team_threads` threads, team index `team` within the CTA (team 0
// starts at thread 0).  Barrier ids 1..15 are used for multi-warp teams.
__device__ __forceinline__ TeamSync make_team_sync(int team, int team_threads) {
  TeamSync s;
  s.cta = false;
  s.nthreads = team_threads;
  s.bar_id = 1 + team;
  if (team_threads >= 32) {
    s.mask = 0xffffffffu;
  } else {
    int lane0 = (team * team_threads) & 31;
    s.mask = ((team_threads == 32) ? 0xffffffffu : ((1u << team_threads) - 1u)) << lane0;
  }
  return s;
}

// As make_team_sync, but teams wider than a warp synchronise on the CTA-wide
// barrier; then every thread of the CTA must call fft_team (idle threads with
// active = false).  Teams inside one warp keep their masked __syncwarp and
// their idle threads skip the call.
__device__ __forceinline__ TeamSync make_block_team_sync(int team, int team_threads) {
  TeamSync s = make_team_sync(team, team_threads);
  s.cta = team_threads > 32;
  return s;
}

// ---- radix-R DFTs in registers, SIGN = -1 forward, +1 inverse (unnormalised)
template <int SIGN, typename C> __device__ __forceinline__ C mul_si(C a) {
  // a * (SIGN * i)
  C r;
  if (SIGN < 0) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
  return r;
}

template <int SIGN, typename C> __device__ __forceinline__ void dft2(C* a) {
  C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_si<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C* a) { dft4<SIGN>(a[0], a[1], a[2], a[3]); }

template <int SIGN, typename C> __device__ __forceinline__ void dft8(C* a) {
  using R = decltype(a[0].x);
  const R h = R(0.70710678118654752440);  // 1/sqrt(2)
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  // w^k = exp(SIGN i pi k / 4): w^1 = (1 + SIGN i)/sqrt2, w^3 = (-1 + SIGN i)/sqrt2
  C w1o, w2o, w3o;
  if constexpr (SIGN < 0) {
    w1o.x = h * (o1.x + o1.y);
    w1o.y = h * (o1.y - o1.x);
    w3o.x = h * (o3.y - o3.x);
    w3o.y = -(h * (o3.y + o3.x));
  } else {
    w1o.x = h * (o1.x - o1.y);
    w1o.y = h * (o1.y + o1.x);
    w3o.x = -(h * (o3.x + o3.y));
    w3o.y = h * (o3.x - o3.y);
  }
  w2o = mul_si<SIGN>(o2);
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, w1o); a[5] = csub(e1, w1o);
  a[2] = cadd(e2, w2o); a[6] = csub(e2, w2o);
  a[3] = cadd(e3, w3o); a[7] = csub(e3, w3o);
}

template <int R, int SIGN, typename C> __device__ __forceinline__ void dft_r(C* a) {
  if constexpr (R == 2) dft2<SIGN>(a);
  else if constexpr (R == 4) dft4<SIGN>(a);
  else dft8<SIGN>(a);
}

template <typename C, int LOGN, int NF, int E, int SIGN, int R, int LS>
__device__ __forceinline__ void stockham_stage(C* buf, int f, int tt, const C* __restrict__ tw, const TeamSync& ts,
                                               bool active) {
  constexpr int N = 1 << LOGN;
  constexpr int B = E / R;
  constexpr int TT = N / E;
  static_assert(E % R == 0, "E must be a multiple of the radix");
  C a[E];
  // twiddles first: they do not depend on the data, so their load latency
  // overlaps the shared-memory reads and the team barrier
  C w[LS > 1 ? B * (R - 1) : 1];
  if (LS > 1 && active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = (tt + TT * b) & (LS - 1);
#pragma unroll
      if constexpr (R == 8) {
        const C w1 = ldg_tw(&tw[j * (kTwN / (LS * R))]), w4 = ldg_tw(&tw[4 * j * (kTwN / (LS * R))]);
        const C w2 = cmul(w1, w1), w3 = cmul(w1, w2);
        C* ww = &w[b * (R - 1)];
        ww[0] = w1; ww[1] = w2; ww[2] = w3; ww[3] = w4; ww[4] = cmul(w4, w1); ww[5] = cmul(w4, w2); ww[6] = cmul(w4, w3);
      } else {
        for (int r = 1; r < R; ++r) w[b * (R - 1) + r - 1] = ldg_tw(&tw[r * j * (kTwN / (LS * R))]);
      }
    }
  }
  // Padded addresses as base + constant: with q = (N/R)*NF, the unpadded
  // read index is i0 + r*q with i0 = t*NF + f, and (i0 & 15) + r*q never
  // crosses a multiple of 16 beyond r*q itself (q >= 16, or i0 < q <= 16
  // with q | 16), so spad(i0 + r*q) = spad(i0) + r*q + (r*q)/16; likewise
  // for the writes with u = LS*NF.
  constexpr int Q = (N / R) * NF;
  constexpr int U = LS * NF;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int t = tt + TT * b;
      const int p0 = spad(t * NF + f);
#pragma unroll
      for (int r = 0; r < R; ++r) a[b * R + r] = buf[p0 + r * Q + (r * Q) / 16];
    }
  }
  ts.sync();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int t = tt + TT * b;
      const int j = t & (LS - 1);
      if constexpr (LS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C wr = w[b * (R - 1) + r - 1];
          if (SIGN > 0) wr.y = -wr.y;
          a[b * R + r] = cmul(a[b * R + r], wr);
        }
      }
      dft_r<R, SIGN>(&a[b * R]);
      const int base = (t / LS) * LS * R + j;
      const int p0 = spad(base * NF + f);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[p0 + r * U + (r * U) / 16] = a[b * R + r];
    }
  }
  ts.sync();
}

// NF interleaved length-2^LOGN FFTs executed by the team's NTH = N*NF/E threads;
// `tid` is the thread's index inside the team.
// With a CTA-wide TeamSync, threads outside every team call this with
// active = false: they take part in the barriers only.
template <typename C, int LOGN, int NF, int E, int SIGN>
__device__ __forceinline__ void fft_team(C* buf, int tid, const C* __restrict__ tw, const TeamSync& ts,
                                         bool active = true) {
  constexpr int S8 = LOGN / 3;
  constexpr int REM = LOGN % 3;
  const int f = tid % NF;
  const int tt = tid / NF;
  if constexpr (S8 >= 1) stockham_stage<C, LOGN, NF, E, SIGN, 8, 1>(buf, f, tt, tw, ts, active);
  if constexpr (S8 >= 2) stockham_stage<C, LOGN, NF, E, SIGN, 8, 8>(buf, f, tt, tw, ts, active);
  if constexpr (S8 >= 3) stockham_stage<C, LOGN, NF, E, SIGN, 8, 64>(buf, f, tt, tw, ts, active);
  if constexpr (REM == 1) stockham_stage<C, LOGN, NF, E, SIGN, 2, (1 << (3 * S8))>(buf, f, tt, tw, ts, active);
  if constexpr (REM == 2) stockham_stage<C, LOGN, NF, E, SIGN, 4, (1 << (3 * S8))>(buf, f, tt, tw, ts, active);
}

// ---- stages with separate input and output accessors ------------------------
// The same radix-R Stockham stage as stockham_stage, for one FFT per team of
// TT = N/E threads, but the stage reads its inputs through `in(i0, off)` and
// writes its outputs through `out(i0, off, v)` (element i0 + off, where off is
// a compile-time multiple of N/R or of LS).  A first stage can then read data
// exactly as a bulk copy left it (unpadded, or straight from global memory) and
// a last stage can write its natural-order results straight to global memory;
// stages in between address the padded layout spad().  `mid()` runs between
// the reads and the writes (a team barrier when in and out alias).
//   reads:  x[t + r N/R]                                 (i0 = t, off = r N/R)
//   writes: y[(t/LS) LS R + (t mod LS) + r LS]           (i0 = base, off = r LS)
// For every stage of a radix-8 (+ one radix-2/4) decomposition of N >= 64,
// (i0 mod 16) + (off mod 16) < 16, so spad(i0 + off) = spad(i0) + off + off/16.
template <typename C, int LOGN, int E, int SIGN, int R, int LS, class In, class Mid, class Out>
__device__ __forceinline__ void fft_stage_io(int tt, const C* __restrict__ tw, In&& in, Mid&& mid, Out&& out) {
  constexpr int N = 1 << LOGN;
  constexpr int B = E / R;
  constexpr int TT = N / E;
  static_assert(E % R == 0, "E must be a multiple of the radix");
  constexpr bool HOIST = LS > 1 && B <= 2;  // twiddles ahead of the barrier when registers allow
  C a[E];
  C w[HOIST ? B * (R - 1) : 1];
  if constexpr (HOIST) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = (tt + TT * b) & (LS - 1);
#pragma unroll
      if constexpr (R == 8) {
        const C w1 = ldg_tw(&tw[j * (kTwN / (LS * R))]), w4 = ldg_tw(&tw[4 * j * (kTwN / (LS * R))]);
        const C w2 = cmul(w1, w1), w3 = cmul(w1, w2);
        C* ww = &w[b * (R - 1)];
        ww[0] = w1; ww[1] = w2; ww[2] = w3; ww[3] = w4; ww[4] = cmul(w4, w1); ww[5] = cmul(w4, w2); ww[6] = cmul(w4, w3);
      } else {
        for (int r = 1; r < R; ++r) w[b * (R - 1) + r - 1] = ldg_tw(&tw[r * j * (kTwN / (LS * R))]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int t = tt + TT * b;
#pragma unroll
    for (int r = 0; r < R; ++r) a[b * R + r] = in(t, r * (N / R));
  }
  mid();
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int t = tt + TT * b;
    const int j = t & (LS - 1);
    if constexpr (LS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C wr = HOIST ? w[b * (R - 1) + r - 1] : ldg_tw(&tw[r * j * (kTwN / (LS * R))]);
        if (SIGN > 0) wr.y = -wr.y;
        a[b * R + r] = cmul(a[b * R + r], wr);
      }
    }
    dft_r<R, SIGN>(&a[b * R]);
    const int base = (t / LS) * LS * R + j;
#pragma unroll
    for (int r = 0; r < R; ++r) out(base, r * LS, a[b * R + r]);
  }
}

// Whole FFT of length 2^LOGN by one team: the first stage reads through `in0`,
// the last writes through `outL`, stages in between use the padded buffer
// `buf` (spad layout, at least spad(N) elements).  `sync()` is the team
// barrier.  When in0 reads `buf` itself (unpadded), the first stage's reads
// complete before any write; when outL writes to `buf`, the last stage's
// writes follow a barrier after its reads.  outL_alias says whether outL
// writes memory that the last stage reads (then a barrier separates them).
template <typename C, int LOGN, int E, int SIGN, bool OUTL_ALIAS, class In0, class OutL, class Sync>
__device__ __forceinline__ void fft_team_io(C* buf, int tt, const C* __restrict__ tw, const Sync& sync, In0&& in0,
                                            OutL&& outL) {
  constexpr int S8 = LOGN / 3;
  constexpr int REM = LOGN % 3;
  constexpr int NST = S8 + (REM ? 1 : 0);
  static_assert(NST >= 2, "at least two stages");
  auto pin = [&](int i0, int off) { return buf[spad(i0) + off + (off >> 4)]; };
  auto pout = [&](int i0, int off, C v) { buf[spad(i0) + off + (off >> 4)] = v; };
  auto bar = [&]() { sync(); };
  auto none = [&]() {};
  // stage 0 (LS = 1, radix 8): in0 -> padded
  fft_stage_io<C, LOGN, E, SIGN, 8, 1>(tt, tw, in0, bar, pout);
  sync();
  // middle radix-8 stages
  if constexpr (NST >= 3) {
    fft_stage_io<C, LOGN, E, SIGN, 8, 8>(tt, tw, pin, bar, pout);
    sync();
  }
  if constexpr (NST >= 4) {
    fft_stage_io<C, LOGN, E, SIGN, 8, 64>(tt, tw, pin, bar, pout);
    sync();
  }
  // last stage: radix 8 at LS = 8^(S8-1) when REM == 0, else radix 2/4 at LS = 8^S8
  constexpr int RL = REM == 0 ? 8 : (REM == 1 ? 2 : 4);
  constexpr int LSL = REM == 0 ? (1 << (3 * (S8 - 1))) : (1 << (3 * S8));
  if constexpr (OUTL_ALIAS) fft_stage_io<C, LOGN, E, SIGN, RL, LSL>(tt, tw, pin, bar, outL);
  else fft_stage_io<C, LOGN, E, SIGN, RL, LSL>(tt, tw, pin, none, outL);
}

// ---- two real rows through one complex FFT ---------------------------------
// Inverse: from the half spectra Xa[k], Xb[k] (k = 0..N/2) of two real rows,
// build Z[k] = Xa[k] + i Xb[k] over the full length using Hermitian symmetry;
// DC and Nyquist keep only their real parts (c2r semantics).
template <typename C>
__device__ __forceinline__ void pair_spectrum_put(C* z, int N, int k, C xa, C xb) {
  if (k == 0 || k == N / 2) {
    z[spad(k)] = cpack<C>(xa.x, xb.x);
  } else {
    z[spad(k)] = cpack<C>(xa.x - xb.y, xa.y + xb.x);
    z[spad(N - k)] = cpack<C>(xa.x + xb.y, xb.x - xa.y);
  }
}

// Forward: Z = FFT(za + i zb) -> Qa[k] = (Z[k] + conj Z[N-k]) * s,
// Qb[k] = -i (Z[k] - conj Z[N-k]) * s, with s = 1/2 folded by the caller.
template <typename C>
__device__ __forceinline__ void pair_spectrum_get(const C* z, int N, int k, C& qa, C& qb) {
  C a = z[spad(k)];
  C b = cconj(z[spad((N - k) & (N - 1))]);
  qa = cadd(a, b);
  C d = csub(a, b);
  qb.x = d.y;
  qb.y = -d.x;
}

}  // namespace cip
