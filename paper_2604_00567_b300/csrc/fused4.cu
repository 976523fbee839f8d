// fused4.cu — one-launch radix-4 FFT of a batch of equal-size signals,
// N <= 2^14 (stage structure in fused4.cuh).
#include "fused4.cuh"

namespace dsfft {

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
__global__ void __launch_bounds__(Fused4<PREC, LOG2N, LOG2R, SCALED>::TPB, Fused4<PREC, LOG2N, LOG2R, SCALED>::MINB)
    fused4_fft_kernel(const typename Elem<PREC>::T *in, typename Elem<PREC>::T *out, int64_t batch,
                      const uint4 *__restrict__ tw, const __grid_constant__ Stage0R4 tw0, int inverse) {
  using K = Fused4<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t first = (int64_t)blockIdx.x * K::TPC;
  const int64_t left = batch - first;
  const int count = left < K::TPC ? (int)left : K::TPC;
  const ContigIO<E> io{in + first * K::N, out + first * K::N, K::N};
  // sign operand of the +-i d3 terms: (s, -s) with s = -1 forward, +1 inverse
  typename K::S sgn;
  if constexpr (PREC == kFP32) sgn = inverse ? 1.0f : -1.0f;
  else if constexpr (PREC == kFP16) sgn = inverse ? 0xBC003C00u : 0x3C00BC00u;
  else sgn = inverse ? 0xBF803F80u : 0x3F80BF80u;
  K::run_tile(io, count, tw, tw0, sgn, reinterpret_cast<E *>(smem_raw));
}

template <int PREC, int LOG2N, bool SCALED>
static cudaError_t launch4_one(const void *in, void *out, int64_t batch, const uint4 *tw, const Stage0R4 &tw0,
                               int inverse, cudaStream_t stream) {
  constexpr int LOG2R = r4_log2r(LOG2N);
  using K = Fused4<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  const int64_t blocks = (batch + K::TPC - 1) / K::TPC;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  fused4_fft_kernel<PREC, LOG2N, LOG2R, SCALED><<<(unsigned)blocks, K::TPB, K::SMEM, stream>>>(
      static_cast<const E *>(in), static_cast<E *>(out), batch, tw, tw0, inverse);
  return cudaGetLastError();
}

template <int PREC, int LOG2N>
static cudaError_t prepare4_one() {
  constexpr int LOG2R = r4_log2r(LOG2N);
  using K = Fused4<PREC, LOG2N, LOG2R, false>;
  const int carve = carveout_for(K::SMEM, K::MINB);
  for (auto kern : {fused4_fft_kernel<PREC, LOG2N, LOG2R, false>, fused4_fft_kernel<PREC, LOG2N, LOG2R, true>}) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    if (e != cudaSuccess) return e;
    if (K::SMEM > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <int PREC, int LOG2N>
static FusedShape shape4_one() {
  constexpr int LOG2R = r4_log2r(LOG2N);
  using K = Fused4<PREC, LOG2N, LOG2R, false>;
  return FusedShape{LOG2R, K::T, K::TPC, K::TPB, K::SMEM};
}

using Launch4Fn = cudaError_t (*)(const void *, void *, int64_t, const uint4 *, const Stage0R4 &, int, cudaStream_t);
using Prepare4Fn = cudaError_t (*)();
using Shape4Fn = FusedShape (*)();

template <int PREC, int... L>
struct Table4 {
  static constexpr Launch4Fn plain[] = {launch4_one<PREC, L, false>...};
  static constexpr Launch4Fn scaled[] = {launch4_one<PREC, L, true>...};
  static constexpr Prepare4Fn prepare[] = {prepare4_one<PREC, L>...};
  static constexpr Shape4Fn shape[] = {shape4_one<PREC, L>...};
};

#define DSFFT_LOG2N_LIST4 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14
using T4_32 = Table4<kFP32, DSFFT_LOG2N_LIST4>;
using T4_16 = Table4<kFP16, DSFFT_LOG2N_LIST4>;
using T4_B16 = Table4<kBF16, DSFFT_LOG2N_LIST4>;

FusedShape fused4_shape(int prec, int log2n) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return FusedShape{0, 0, 0, 0, 0};
  const int i = log2n - 1;
  return prec == kFP32 ? T4_32::shape[i]() : prec == kFP16 ? T4_16::shape[i]() : T4_B16::shape[i]();
}

cudaError_t prepare_fused4(int prec, int log2n) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  const int i = log2n - 1;
  return prec == kFP32 ? T4_32::prepare[i]() : prec == kFP16 ? T4_16::prepare[i]() : T4_B16::prepare[i]();
}

cudaError_t launch_fused4(int prec, int log2n, bool scaled, int inverse, const void *in, void *out, int64_t batch,
                          const uint4 *twp4, const Stage0R4 &tw0, cudaStream_t stream) {
  if (log2n < 1 || log2n > kFusedMaxLog2N) return cudaErrorInvalidValue;
  const int i = log2n - 1;
  Launch4Fn f;
  if (prec == kFP32) f = scaled ? T4_32::scaled[i] : T4_32::plain[i];
  else if (prec == kFP16) f = scaled ? T4_16::scaled[i] : T4_16::plain[i];
  else f = scaled ? T4_B16::scaled[i] : T4_B16::plain[i];
  return f(in, out, batch, twp4, tw0, inverse, stream);
}

}  // namespace dsfft
