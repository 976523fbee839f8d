// fused.cu — one-launch FFT of a batch of equal-size signals, N <= 2^14:
// every pass of a transform runs on chip, so each signal is read from HBM
// once and written once (stage structure in fused.cuh).
#include "fused.cuh"

namespace dsfft {

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
__global__ void __launch_bounds__(Fused<PREC, LOG2N, LOG2R, SCALED>::TPB, Fused<PREC, LOG2N, LOG2R, SCALED>::MINB)
    fused_fft_kernel(const typename Elem<PREC>::T *in, typename Elem<PREC>::T *out, int64_t batch,
                     const uint4 *__restrict__ tw, const __grid_constant__ Stage0Twiddles tw0) {
  using K = Fused<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t first = (int64_t)blockIdx.x * K::TPC;
  const int64_t left = batch - first;
  const int count = left < K::TPC ? (int)left : K::TPC;
  const ContigIO<E> io{in + first * K::N, out + first * K::N, K::N};
  K::run_tile(io, count, tw, [&](int i) { return tw0.e[i]; }, reinterpret_cast<E *>(smem_raw));
}

// ---------------------------------------------------------------------------
// dispatch

template <int PREC, int LOG2N, bool NARROW, bool SCALED>
static cudaError_t launch_one(const void *in, void *out, int64_t batch, const uint4 *tw, const Stage0Twiddles &tw0,
                              cudaStream_t stream) {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, NARROW);
  using K = Fused<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  auto kern = fused_fft_kernel<PREC, LOG2N, LOG2R, SCALED>;
  const int64_t blocks = (batch + K::TPC - 1) / K::TPC;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(static_cast<const E *>(in), static_cast<E *>(out), batch, tw, tw0);
  return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of both scalings on the current
// device (needed above 48 KB); called once per plan creation.
template <int PREC, int LOG2N, bool NARROW>
static cudaError_t prepare_one() {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, NARROW);
  using K = Fused<PREC, LOG2N, LOG2R, false>;
  // Shared-memory carveout: enough for the blocks the register budget lets
  // reside (MINB, at least one), the rest stays L1 for the twiddle table.
  const int carve = carveout_for(K::SMEM, K::MINB);
  for (auto kern : {fused_fft_kernel<PREC, LOG2N, LOG2R, false>, fused_fft_kernel<PREC, LOG2N, LOG2R, true>}) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    if (e != cudaSuccess) return e;
    if (K::SMEM > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <int PREC, int LOG2N, bool NARROW>
static FusedShape shape_one() {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, NARROW);
  using K = Fused<PREC, LOG2N, LOG2R, false>;
  return FusedShape{LOG2R, K::T, K::TPC, K::TPB, K::SMEM};
}

using LaunchFn = cudaError_t (*)(const void *, void *, int64_t, const uint4 *, const Stage0Twiddles &,
                                 cudaStream_t);
using ShapeFn = FusedShape (*)();
using PrepareFn = cudaError_t (*)();

template <int PREC, bool NARROW, int... L>
struct Table {
  static constexpr LaunchFn plain[] = {launch_one<PREC, L, NARROW, false>...};
  static constexpr LaunchFn scaled[] = {launch_one<PREC, L, NARROW, true>...};
  static constexpr ShapeFn shape[] = {shape_one<PREC, L, NARROW>...};
  static constexpr PrepareFn prepare[] = {prepare_one<PREC, L, NARROW>...};
};

#define DSFFT_LOG2N_LIST 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14
template <bool NARROW>
struct Tables {
  using T32 = Table<kFP32, NARROW, DSFFT_LOG2N_LIST>;
  using T16 = Table<kFP16, NARROW, DSFFT_LOG2N_LIST>;
  using TB16 = Table<kBF16, NARROW, DSFFT_LOG2N_LIST>;
  static FusedShape shape(int prec, int i) {
    return prec == kFP32 ? T32::shape[i]() : prec == kFP16 ? T16::shape[i]() : TB16::shape[i]();
  }
  static cudaError_t prepare(int prec, int i) {
    return prec == kFP32 ? T32::prepare[i]() : prec == kFP16 ? T16::prepare[i]() : TB16::prepare[i]();
  }
  static LaunchFn launch(int prec, int i, bool scaled) {
    if (prec == kFP32) return scaled ? T32::scaled[i] : T32::plain[i];
    if (prec == kFP16) return scaled ? T16::scaled[i] : T16::plain[i];
    return scaled ? TB16::scaled[i] : TB16::plain[i];
  }
};

FusedShape fused_shape(int prec, int log2n, bool narrow) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return FusedShape{0, 0, 0, 0, 0};
  return narrow ? Tables<true>::shape(prec, log2n - 1) : Tables<false>::shape(prec, log2n - 1);
}

bool fused_has_narrow(int prec, int log2n) {
  return log2n >= 1 && log2n <= kFusedMaxLog2N && fused_log2r(prec, log2n, true) != fused_log2r(prec, log2n, false);
}

cudaError_t prepare_fused(int prec, int log2n, bool narrow) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  return narrow ? Tables<true>::prepare(prec, log2n - 1) : Tables<false>::prepare(prec, log2n - 1);
}

cudaError_t launch_fused(int prec, int log2n, bool narrow, bool scaled, const void *in, void *out, int64_t batch,
                         const uint4 *table, const Stage0Twiddles &tw0, cudaStream_t stream) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  LaunchFn f = narrow ? Tables<true>::launch(prec, log2n - 1, scaled) : Tables<false>::launch(prec, log2n - 1, scaled);
  return f(in, out, batch, table, tw0, stream);
}

}  // namespace dsfft
