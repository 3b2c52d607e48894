// Internal launch interface between the C ABI (abi.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "df64.cuh"

namespace cip {

enum PriorKind { PRIOR_TV = 0, PRIOR_DCT8 = 1, PRIOR_L1 = 2, PRIOR_CONVDICT = 3, PRIOR_TV_ISO = 4, PRIOR_WDCT = 5 };
// row transforms of the prior-pass kernel without a prior: x rows out of the column-layout
// spectra (ROWS_OUT: read-back, wavelet chain), or q-hat from real rows (ROWS_IN)
enum RowKind { ROWS_OUT = 100, ROWS_IN = 101 };
// the two TV priors share T = [D_h; D_v] (two components, one halo row each side)
constexpr bool prior_is_tv(int p) { return p == PRIOR_TV || p == PRIOR_TV_ISO; }

// flags of the prior pass
enum { PA_STORE_T = 1, PA_RESID = 2, PA_IMPORT = 4 };
constexpr int kNPart = 5;  // sum (w-t)^2, sum w^2, sum t^2, sum u^2, sum (t - t_prev)^2
constexpr int kLowK = 2;   // half-spectrum columns k2 < kLowK get the low-column correction (TV)

inline int prior_ncomp(int prior) { return prior_is_tv(prior) ? 2 : 1; }

// Prior pass (one ADMM t/u update + the adjoint for the next x-update):
//   x = row-IDFT(xh)  ->  w = T x  ->  t = soft(w + u, tau)  ->  u' = u + w - t
//   -> q = qscale * T^T (t - u')  ->  qh = row-DFT(q) (half spectrum, pair-extracted)
// In IMPORT mode x is not used: t comes from t_imp and u' = u_in.
// The row spectra xh and qh use the column layout [N/2+1][maps][col_pitch(N)]: for each
// half-spectrum column k2 the N row values of every map are contiguous.
// ROWS_OUT: x = row-IDFT(xh) is written to u_out ([maps][N][N]) and nothing else happens.
// ROWS_IN: qh = row-DFT(2 qscale u_in) from real rows u_in ([maps][N][N]).
template <typename T> struct PassAArgs {
  using C = typename CT<T>::type;
  const C* xh;      // [N/2+1][M][CP] (column layout)
  C* qh;            // [N/2+1][M][CP] (column layout)
  const T* u_in;    // [M][ncomp][N][N]
  T* u_out;         // [M][ncomp][N][N]
  T* tprev;         // [M][ncomp][N][N] (STORE_T writes t, RESID reads t_prev)
  const T* t_imp;   // [M][ncomp][N][N] (IMPORT)
  double* partials; // [gridDim.y * gridDim.x][kNPart] (RESID)
  int* err;         // set to 1 when a bounded wait on an asynchronous copy gives up
  const C* tw;      // twiddle table, kTwN entries
  int M;
  T tau;            // lambda / rho
  T qscale;         // rho / 2 (the 1/2 of the pair extraction is folded here)
  int flags;
  int test_fault;   // 1: the staged u copy is replaced by a barrier that never completes (test of
                    // the bounded wait: no copy is issued, the wait gives up after 64 polls)
  int variant;      // 1: the kernel variant with the other FFT width (complex64, N = 256 .. 1024)
  C* lowbuf;        // TV: [2][kLowK][M][CP] row DFTs of the components of t - u' at k2 < kLowK
                    // for the low-column correction of the split column pass; NULL: not formed
  T dct[64];        // orthonormal DCT-II, dct[k*8+n]
};

// Column pass with the per-frequency solve (Eq. solx_Trans_DFT), the data
// term precomputed:  Q = col-DFT(qh);  X(w) = xb(w) + Pinv(w) Q(w);  xh = col-IDFT(X)
template <typename T> struct PassBArgs {
  using C = typename CT<T>::type;
  const C* qh;      // [N/2+1][M][CP] (column layout)
  C* xh;            // [N/2+1][M][CP] (column layout)
  const C* pinv;    // [N/2+1][M(M+1)/2][N] packed upper triangle per bin, scaled by 1/N^2
  const C* bhat;    // [N/2+1][M][N]: xb = Psi^{-1} beta Lambda^H F y / N^2 (FP64-formed)
  const C* tw;
  int N;
  int M;
  int plain;        // 1: plain FP32 method, bhat holds b = beta Lambda^H F y and X = Pinv (b + Q)
};

// plain FP32 method: factor formed and inverted in FP32, b = beta Lambda^H F y in FP32
cudaError_t launch_factor_fp32(const cdf* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                               double beta, float2* pinv, int* pinv_list, int list_cap, cudaStream_t s);
cudaError_t launch_rhs_fp32(const cdf* lam, const cdf* yhat, int K, int M, int N, double beta, float2* b,
                            cudaStream_t s);

// Convolutional-dictionary column solve (Eqs. solx_synt_DFT, solz_DFT, solz_DFT_SM), one
// thread per (frequency, channel).  Column layout [k2][plane][col_pitch(N)].
template <typename T> struct CDArgs {
  using C = typename CT<T>::type;
  C* colbuf;       // [H][M*L]: in G = col-DFT of rho (t - u) / N^2, out v (channel-major, m*L + l)
  const C* theta;  // [H][th_planes]: DFT of the embedded filters in the first L planes of each bin
  const C* p_in;   // [H][M]: p = sum_l theta_l v_l of the previous iteration (scaled 1/N^2)
  C* p_out;        // [H][M]
  const C* xb;     // [H][M]: Psi^{-1} beta Lambda^H F y / N^2
  const C* pinv;   // [H][M(M+1)/2]: packed (I + beta Lambda^H Lambda)^{-1} / N^2
  C* xcol;         // [H][M]: x-hat / N^2 (for read-back)
  const double* gs;  // [N] 4 sin^2(pi k / N): per-axis eigenvalues of the circular difference
  int N, M, L;
  int th_planes;   // planes per bin in theta's buffer (L, or 2L while the dictionary is learnt)
  T rho;
  T mu;            // gradient (Tikhonov) weight on the codes; z-update diagonal rho + mu (gs[k1] + gs[k2])
  T n2;            // N^2
};
template <typename T> cudaError_t launch_cd_solve(const CDArgs<T>& a, cudaStream_t s);

// 3D dictionary (Section IV-B, 3D case; csrc/convdict3d.cu): the same column layout for the
// channel-domain spectra; theta holds Theta_l(kappa, w) at plane kappa*L + l of [H][M*L][CP].
template <typename T> struct CD3Args {
  using C = typename CT<T>::type;
  C* colbuf;       // [H][M*L]: in G = col-DFT of rho (t - u) / N^2, out V (channel-major, m*L + l)
  const C* theta;  // [H][M*L]: 3D DFT of the embedded filters, plane kappa*L + l
  const C* p_in;   // [H][M]
  C* p_out;        // [H][M]
  const C* xb;     // [H][M]
  const C* pinv;   // [H][M(M+1)/2]
  C* xcol;         // [H][M]
  int N, M, L;
  T rho, n2;
  C w[16];         // exp(-2 pi i j / M), j < M
};
template <typename T> cudaError_t launch_cd3_solve(const CD3Args<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_p3_from_z(const typename CT<T>::type* zcol, const typename CT<T>::type* th3,
                             typename CT<T>::type* p, const CD3Args<T>& a, double scale, cudaStream_t s);
template <typename Tin>
cudaError_t launch_embed_filters3d(const Tin* d, double* out, int L, int Q, int P, int M, int N, cudaStream_t s);
template <typename T>
cudaError_t launch_theta3_store(const SetupC<T>* th64, typename CT<T>::type* th, const double2* w, int L, int M, int N,
                                cudaStream_t s);
template <typename T> bool cd3_fits(int M, int L);
template <typename T>
cudaError_t launch_p_from_z(const typename CT<T>::type* zcol, const typename CT<T>::type* th,
                            typename CT<T>::type* p, int N, int M, int L, cudaStream_t s,
                            double scale = 0.0, int th_planes = 0);
// Online dictionary update (Section IV-B, Eqs. d_admm, g_admm, h_admm): one filter-ADMM step in
// three launches.  The scaled dual e is kept as its spectrum (e-hat = theta - F(g - e)); the filters
// g live on the P x P support, so the spatial values the projection needs (d + e on the support) are
// partial inverse DFTs at the P x P support points, and the new theta = F g is a partial DFT from
// the support.  Spectra are unnormalised DFTs; zcol and xcol carry the column solve's 1/N^2.
constexpr int kDLBlock = 64;  // bins per CTA of the per-frequency launches (one column segment)
constexpr int kDLMaxP = 32;   // largest filter side the update supports
template <typename T> struct DLArgs {
  using C = typename CT<T>::type;
  const C* zcol;   // [H][M][L]: code spectra / N^2 (channel-major, m*L + l)
  const C* xcol;   // [H][M]: image spectra / N^2
  C* spec;         // [H][2L]: theta = F g in planes 0..L-1, F(g - e) in planes L..2L-1
  C* wcol;         // [H][L]: w = F(d + e) of this step
  C* ypart;        // [H][N/kDLBlock][L][P]: per-CTA sums over k1 of w(k1, k2) exp(2 pi i k1 a / N)
  C* yfull;        // [L][P][H]: the same summed over the whole column
  int* cnt;        // [H]: CTAs of a column that have written their sums (zero between launches)
  C* gfac;         // [H][L][P]: sum_b g(a, b) exp(-2 pi i k2 b / N)
  T* gs;           // [L][P][P]: the filters g on the support (centre P/2)
  double* rpart;   // [H][N/kDLBlock]: sums of |F(d - g)|^2 (weighted for the half spectrum)
  double* spart;   // [L]: ||g - g_prev||^2 per filter
  C* p_out;        // [H][M]: p = sum_l theta_l z_l / N^2 for the next x-update
  const C* tw;     // exp(-2 pi i j / kTwN)
  int N, M, L, P;
  int check;       // 1: form the residual sums (an adaptation check follows this step)
  T sigma;
};
template <typename T> cudaError_t launch_dl_solve(const DLArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_dl_filter(const DLArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_dl_spec(const DLArgs<T>& a, cudaStream_t s);
// F(g - e) <- theta - (theta - F(g - e)) f: the scaled dual times f = sigma_old / sigma_new
template <typename T>
cudaError_t launch_dl_rescale(typename CT<T>::type* spec, int L, int N, T f, cudaStream_t s);
template <typename Tin> cudaError_t launch_embed_filters(const Tin* d, double* out, int L, int P, int N, cudaStream_t s);
template <typename T>
cudaError_t launch_theta_store(const SetupC<T>* th64, typename CT<T>::type* th, int L, int N, cudaStream_t s);

template <typename T> int passA_rows(int N, int prior);
template <typename T> size_t passA_smem(int N, int prior);
template <typename T> cudaError_t launch_passA(const PassAArgs<T>& a, int N, int prior, cudaStream_t s);

// Fused column pass (csrc/colpass.cu): one CTA per half-spectrum column, factor and data term
// streamed through a ring of TMA bulk copies.  fits: the tile and at least two ring stages fit in
// shared memory.  `err` is set when a bounded wait gives up.
template <typename T> bool colpass_fused_fits(int N, int M);
template <typename T> size_t colpass_fused_smem(int N, int M);
template <typename T> cudaError_t launch_colpass_fused(const PassBArgs<T>& b, int S, int* err, cudaStream_t s);
// column DFTs of every (k2, map) column of the column layout, src -> dst (may alias);
// sign < 0 forward, > 0 inverse (unnormalised)
template <typename T>
cudaError_t launch_cols_fft(const typename CT<T>::type* src, typename CT<T>::type* dst,
                            const typename CT<T>::type* tw, int N, int maps, int sign, cudaStream_t s,
                            const typename CT<T>::type* src2 = nullptr, typename CT<T>::type* dst2 = nullptr,
                            int ncols2 = 0);
// split form: column FFT of qh into colbuf (same layout), per-bin solve in place, inverse column FFT
// into xh.  With lowbuf (TV, low-column correction), the same forward launch also transforms the
// 2 kLowK M low-frequency columns of lowbuf into lowcol, and the solve takes, for the columns
// k2 < kLowK, Q = rho (conj(dh(k2)) F A_h + conj(dv(k1)) F A_v) in place of the column DFT of q:
// near DC the FP32 transforms of q = D^T (t - u) carry a uniform rounding error that Psi^{-1}
// amplifies by ~1/g, the transforms of the components of t - u do not.
template <typename T>
cudaError_t launch_passB_split(const PassBArgs<T>& a, typename CT<T>::type* colbuf, int N, cudaStream_t s,
                               int* launches, const typename CT<T>::type* lowbuf = nullptr,
                               typename CT<T>::type* lowcol = nullptr, T rho = T(0));

// Setup / read-back FFTs (not fused).
// rows: nrows real rows of length N -> half spectra with pitch P (unnormalised forward DFT)
template <typename Tc, typename Tin>
cudaError_t launch_row_r2c(const Tin* in, typename CT<Tc>::type* out, int N, int nrows, Tc scale,
                           const typename CT<Tc>::type* tw, cudaStream_t s);
// in-place column DFT of nmaps [N][P] half-spectrum maps
template <typename Tc>
cudaError_t launch_col_c2c(typename CT<Tc>::type* data, int N, int nmaps, int sign,
                           const typename CT<Tc>::type* tw, cudaStream_t s);

// Factor formation in the setup precision (double-float for complex64 plans, FP64 for
// complex128 plans): Psi = rho g I + beta Lam^H Lam per bin; writes
// Psi^{-1} / N^2 packed into `pinv`.  Bins needing a pseudo-inverse are
// appended to `pinv_list` (count in pinv_list[0]).
// The setup-precision copy `pinv64` (same layout) is written too when non-null.
template <typename Tout>
cudaError_t launch_factor(const SetupC<Tout>* lam, const double* gs, int use_g, int K, int M, int N, double rho,
                          double beta, typename CT<Tout>::type* pinv, SetupC<Tout>* pinv64, int* pinv_list,
                          int list_cap,
                          cudaStream_t s);
template <typename Tout>
cudaError_t launch_factor_pinv(const SetupC<Tout>* lam, const double* gs, int use_g, int K, int M, int N,
                               double rho, double beta, typename CT<Tout>::type* pinv, SetupC<Tout>* pinv64,
                               const int* pinv_list, int list_cap, cudaStream_t s);
// xb = Pinv64 (beta Lam^H yhat) in the setup precision, rounded once to the plan precision
template <typename Tout>
cudaError_t launch_rhs(const SetupC<Tout>* lam, const SetupC<Tout>* yhat, const SetupC<Tout>* pinv64, int K, int M,
                       int N,
                       double beta, typename CT<Tout>::type* xb, cudaStream_t s);
// a[i] *= f for i < n (the scaled dual at a change of the penalty)
template <typename T> cudaError_t launch_scale(T* a, size_t n, T f, cudaStream_t s);

// deterministic reduction of pass-A partials: out[0..kNPart) sums, out[5]=r_rel, out[6]=s_rel,
// conv[0] set to 1 when both relative residuals < tol (tol > 0)
cudaError_t launch_reduce_partials(const double* partials, int nblocks, double rho, double tol, double* out,
                                   int* conv, cudaStream_t s);

// Kronecker prior T = Symmlet-8 wavelet (x) channel DCT (Section V; csrc/wavelet.cu)
template <typename T> struct WaveFilt {
  T h[16];  // lowpass
  T g[16];  // highpass g_k = (-1)^k h_{15-k}
};
// the orthonormal DCT-II along the channels, row k = frequency ([M][M], M <= 16), passed by value
// so that the per-pixel kernel reads it from the constant bank (every thread uses the same entry)
template <typename T> struct ChanDCT {
  T c[256];
};
// Symmlet lowpass with p vanishing moments (2p taps) from the spectral factorisation; false if p
// is outside [1, 8]
bool symlet_lowpass(int p, double* h);
// one level of the periodic 2D DWT (rows then columns) on the n x n band of each of M planes
// (n a power of two, 32 <= n <= N).  Forward: band from `in` (pitch, plane stride) -> the three
// detail subbands into det ([M][N][N], Mallat positions) and LL into `ll`.  Inverse: LL from `ll`
// and the details from det -> the n x n band into `out`.
template <typename T>
cudaError_t launch_dwt2_fwd(const T* in, int in_pitch, size_t in_plane, T* det, int N, T* ll, int ll_pitch,
                            size_t ll_plane, int n, int M, const WaveFilt<T>& f, cudaStream_t s);
template <typename T>
cudaError_t launch_dwt2_inv(const T* ll, int ll_pitch, size_t ll_plane, const T* det, int N, T* out, int out_pitch,
                            size_t out_plane, int n, int M, const WaveFilt<T>& f, cudaStream_t s);
// Bands of side n <= wave_fuse_n run all their remaining levels in one kernel, one CTA per
// channel, in shared memory (2 n0 (n0 + 1) values forward, 2 n0 (n0 / 2 + 1) inverse).  wave_fuse_band(N): the side
// of the first such band of an N x N image.  Forward: band n0 from `in` -> details and the final
// 16 x 16 LL into A ([M][N][N], Mallat positions).  Inverse: from A -> the band n0 into `out`.
template <typename T> constexpr int wave_fuse_n() { return 64; }
template <typename T> int wave_fuse_band(int N);
template <typename T>
cudaError_t launch_dwt2_fwd_fused(const T* in, int in_pitch, size_t in_plane, T* A, int N, int n0, int M,
                                  const WaveFilt<T>& f, cudaStream_t s);
template <typename T>
cudaError_t launch_dwt2_inv_fused(const T* A, int N, T* out, int out_pitch, size_t out_plane, int n0, int M,
                                  const WaveFilt<T>& f, cudaStream_t s);
// per pixel: channel DCT (cmat [M][M], row k = frequency), shrinkage / dual update / residual
// partials as the other prior passes (flags PA_*), q = t - u', coefficients <- C^T q in place
template <typename T>
cudaError_t launch_wdct_shrink(T* coef, const ChanDCT<T>& cmat, const T* u_in, T* u_out, T* tprev, const T* t_imp,
                               double* partials, int blocks, int N, int M, T tau, int flags, cudaStream_t s);

}  // namespace cip
