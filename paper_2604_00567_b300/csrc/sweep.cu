// sweep.cu — host dispatch of the two-sweep FFT for N > 2^14 (the kernels
// are in sweep.cuh, instantiated per precision by sweep_fp32.cu,
// sweep_fp16.cu and sweep_bf16.cu).
#include <atomic>

#include "internal.h"

namespace dsfft {

using SweepFn = cudaError_t (*)(const void *, void *, const BatchItem *, int64_t, int, int, const uint4 *,
                                const uint4 &, uint32_t, cudaStream_t);
template <int PREC>
SweepFn sweep_lookup(bool r4, bool scaled, bool last, int ls);
template <int PREC>
cudaError_t sweep_prepare_ls(bool r4, int ls);
extern template SweepFn sweep_lookup<kFP32>(bool, bool, bool, int);
extern template SweepFn sweep_lookup<kFP16>(bool, bool, bool, int);
extern template SweepFn sweep_lookup<kBF16>(bool, bool, bool, int);
extern template cudaError_t sweep_prepare_ls<kFP32>(bool, int);
extern template cudaError_t sweep_prepare_ls<kFP16>(bool, int);
extern template cudaError_t sweep_prepare_ls<kBF16>(bool, int);

int sweep_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cached) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

void sweep_split(int log2n, int *ls1, int *ls2) {
  *ls1 = (log2n + 1) / 2;
  *ls2 = log2n / 2;
}

// Radix-4 plans: both sweeps hold whole radix-4 passes (sweep 1 also the
// radix-2 pass of an odd log2 N), as balanced as LS in [7, 12] allows.
void sweep_split4(int log2n, int *ls1, int *ls2) {
  const int par = log2n & 1;
  const int n4 = (log2n - par) / 2;
  int a = (n4 + 1) / 2;
  while (a > 0 && (par + 2 * a > 12 || 2 * (n4 - a) < 7)) --a;
  while (par + 2 * a < 7 && 2 * (n4 - a) > 12) ++a;
  *ls1 = par + 2 * a;
  *ls2 = 2 * (n4 - a);
}

bool sweep_ls1_valid(int log2n, int ls1) { return ls1 >= 7 && ls1 <= 12 && log2n - ls1 >= 7 && log2n - ls1 <= 12; }

template <bool R4>
static cudaError_t prepare_sweeps_impl(int prec, int log2n, int ls1_req = 0) {
  int ls1, ls2;
  if (R4) sweep_split4(log2n, &ls1, &ls2);
  else sweep_split(log2n, &ls1, &ls2);
  if (!R4 && ls1_req > 0) {
    ls1 = ls1_req;
    ls2 = log2n - ls1_req;
  }
  if (ls1 < 7 || ls1 > 12 || ls2 < 7 || ls2 > 12) return cudaErrorInvalidValue;
  for (int ls : {ls1, ls2}) {
    cudaError_t e = prec == kFP32 ? sweep_prepare_ls<kFP32>(R4, ls)
                    : prec == kFP16 ? sweep_prepare_ls<kFP16>(R4, ls) : sweep_prepare_ls<kBF16>(R4, ls);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool R4>
static cudaError_t launch_sweeps_impl(int prec, int log2n, bool scaled, const void *in, void *out,
                                      const BatchItem *items, int64_t batch, const uint4 *twp, const uint4 &r2e,
                                      uint32_t sgn, cudaStream_t stream, int ls1_req = 0) {
  int ls1, ls2;
  if (R4) sweep_split4(log2n, &ls1, &ls2);
  else sweep_split(log2n, &ls1, &ls2);
  if (!R4 && ls1_req > 0) {
    ls1 = ls1_req;
    ls2 = log2n - ls1_req;
  }
  if (ls1 < 7 || ls1 > 12 || ls2 < 7 || ls2 > 12) return cudaErrorInvalidValue;
  auto get = [&](bool last, int ls) {
    return prec == kFP32 ? sweep_lookup<kFP32>(R4, scaled, last, ls)
           : prec == kFP16 ? sweep_lookup<kFP16>(R4, scaled, last, ls) : sweep_lookup<kBF16>(R4, scaled, last, ls);
  };
  cudaError_t e = get(false, ls1)(in, out, items, batch, log2n, 0, twp, r2e, sgn, stream);
  if (e != cudaSuccess) return e;
  return get(true, ls2)(out, out, items, batch, log2n, ls1, twp, r2e, sgn, stream);
}

cudaError_t prepare_sweeps(int prec, int log2n, int ls1) { return prepare_sweeps_impl<false>(prec, log2n, ls1); }

cudaError_t launch_sweeps(int prec, int log2n, bool scaled, const void *in, void *out, const BatchItem *items,
                          int64_t batch, const uint4 *twp, cudaStream_t stream, int ls1) {
  return launch_sweeps_impl<false>(prec, log2n, scaled, in, out, items, batch, twp, uint4{}, 0u, stream, ls1);
}

cudaError_t prepare_sweeps4(int prec, int log2n) { return prepare_sweeps_impl<true>(prec, log2n); }

cudaError_t launch_sweeps4(int prec, int log2n, bool scaled, int inverse, const void *in, void *out,
                           const BatchItem *items, int64_t batch, const uint4 *twp4, const uint4 &r2e,
                           cudaStream_t stream) {
  // sign operand of the +-i d3 terms: (s, -s), s = -1 forward, +1 inverse
  const uint32_t sgn = prec == kFP32 ? (inverse ? 0x3F800000u : 0xBF800000u)
                       : prec == kFP16 ? (inverse ? 0xBC003C00u : 0x3C00BC00u)
                                       : (inverse ? 0xBF803F80u : 0x3F80BF80u);
  return launch_sweeps_impl<true>(prec, log2n, scaled, in, out, items, batch, twp4, r2e, sgn, stream);
}

}  // namespace dsfft
