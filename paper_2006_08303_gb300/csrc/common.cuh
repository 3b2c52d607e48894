// Common device/host helpers for the cip library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

namespace cip {

constexpr int kTwN = 2048;  // twiddle table length (max FFT length)

// complex type per real type: float -> float2 (complex64), double -> double2 (complex128)
template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
  C c; c.x = (decltype(c.x))re; c.y = (decltype(c.y))im; return c;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// complex value from computed parts of the complex type's own real type
template <typename C, typename R> __device__ __forceinline__ C cpack(R re, R im) {
  C c;
  c.x = re;
  c.y = im;
  return c;
}
// read-only cached load of a table entry (twiddles)
__device__ __forceinline__ float2 ldg_tw(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_tw(const double2* p) { return __ldg(p); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { a.x *= s; a.y *= s; return a; }

// Shared-memory padding: one complex slot per 16 keeps every Stockham read
// and write pattern of the FFT free of bank conflicts.
__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }

// Half-spectrum row pitch (complex elements): N/2+1 columns rounded up so
// that every row starts on a 32-byte boundary.
__host__ __device__ __forceinline__ constexpr int half_pitch(int N) { return N / 2 + 4; }

// Column-contiguous per-bin planes ([k2][plane][k1], used by the factor, the
// data term and the split column buffer): N bins plus 32 elements of padding
// so that consecutive planes are not a power-of-two stride apart.
__host__ __device__ __forceinline__ constexpr int col_pitch(int N) { return N + 32; }

// Per-bin planes of the factor Psi^{-1} and of the data term, blocked by 32 bins of a column:
// [k2][k1 / 32][plane][32].  The planes of 32 consecutive bins of one column form one
// contiguous run, which the fused column pass fetches with a single bulk copy per ring stage,
// and a warp reading one plane of 32 consecutive bins reads one contiguous segment.
constexpr int kBinBlock = 32;
__host__ __device__ __forceinline__ size_t binp(int k2, int plane, int k1, int nplanes, int N) {
  return (((size_t)k2 * (N / kBinBlock) + (k1 >> 5)) * nplanes + plane) * kBinBlock + (k1 & (kBinBlock - 1));
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA unit, no shared memory, no
// completion to wait for).  The range is widened to 16-byte boundaries; the
// caller guarantees that the widened range lies inside one allocation.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
  const uintptr_t a1 = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~uintptr_t(15);
  if (a1 > a0) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
  }
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier --------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the asynchronous (TMA) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive once on the barrier and announce `bytes` of transactions for the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// plain arrival (no transactions): a consumer releasing a buffer
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// contiguous global -> shared copy by the TMA unit; both addresses 16-byte aligned, bytes a
// multiple of 16; completion is counted on `bar`
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar`: gives up after one second of the
// GPU's global timer (or 2^22 polls, whichever comes first), records the
// failure in *err and returns false, so that a lost copy ends the kernel with an
// error status instead of a hung GPU.  A legitimate wait lasts microseconds.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int* err,
                                                  int max_polls = 1 << 22) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < max_polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() - t0 > 1000000000ull) break;
  }
  if (err) atomicExch(err, 1);
  return false;
}

// The same wait by every lane of a converged warp (each lane's own successful wait orders its
// later reads after the asynchronous writes), with one decision for the whole warp: it goes on
// only if every lane saw the phase complete.
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long* bar, unsigned parity, int* err) {
  const bool mine = mbar_wait_bounded(bar, parity, err);
  return __all_sync(0xffffffffu, mine) != 0;
}

// Kernel attributes (shared-memory size, carveout, cluster size) are per function and per
// device: PerDeviceOnce runs the setting once for each device a call site meets.
struct PerDeviceOnce {
  std::atomic<unsigned long long> done{0};
  template <typename F> cudaError_t operator()(F&& set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = set();
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
  }
};

// Programmatic dependent launch.  The iteration's kernels are launched with
// programmatic stream serialisation: a kernel may start while its predecessor
// drains, runs only independent work (L2 prefetches of constant operands)
// before grid_dep_wait(), which returns once the predecessor grid has
// completed and its writes are visible, and then lets its own successor be
// scheduled (grid_dep_launch()).  Without the launch attribute both are no-ops.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kern` with programmatic stream serialisation (plus a cluster of
// cluster_x CTAs along x when cluster_x > 0).  The kernel must call grid_dep_wait() before it touches any
// memory that an earlier kernel of the stream writes or reads.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              unsigned cluster_x, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  unsigned n = 0;
  attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[n].val.programmaticStreamSerializationAllowed = 1;
  ++n;
  if (cluster_x > 0) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = cluster_x;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Plain launch through cudaLaunchKernelEx: the returned status is this launch's own, so a caller
// neither mistakes an earlier pending error for it nor has to clear that error to see it.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// soft(w, tau) = sign(w) max(|w| - tau, 0) with sign(0) = -1 (Eq. solt_trans);
// the result is identical to the sign convention's for w = 0 (both give 0).
template <typename T> __device__ __forceinline__ T soft(T w, T tau) {
  T a = fabs(w) - tau;
  a = a > T(0) ? a : T(0);
  return w > T(0) ? a : -a;
}

}  // namespace cip
