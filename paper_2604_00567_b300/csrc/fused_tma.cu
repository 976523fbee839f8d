// fused_tma.cu — persistent form of the fused on-chip transform (N <= 2^14)
// whose input arrives by bulk asynchronous copies (cp.async.bulk, the TMA
// engine) instead of per-thread loads.
//
// Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (a tile
// is the TPC transforms of the fused kernel's block).  Two shared-memory
// buffers alternate: while the CTA transforms the tile in one, the copy
// engine fills the other with the next tile, so HBM reads overlap the
// arithmetic without holding loads in flight in registers.  Each transform
// of a tile is one bulk copy of N contiguous elements into its padded
// region (stride PADN, the exchange layout of fused.cuh); the first register
// stage reads Z_0[tid + p T] from there (conflict-free), and the later
// exchanges reuse the same region.  The passes, twiddles and stores are
// those of the fused kernel, so the result is bit-identical to it.
//
// Synchronisation per buffer: one mbarrier, armed by the issuing thread with
// the tile's byte count (arrive.expect_tx) and completed by the copies
// (complete_tx).  A buffer is refilled only after a block barrier that every
// thread reaches once it has finished the previous tile, and each thread
// orders its generic-proxy accesses to the buffer before that refill with
// fence.proxy.async.
//
// Every wait is bounded (about one second of %globaltimer): a CTA whose copy
// does not complete sets bit 0 of `status`, waits (bounded again) for the
// copies it still has in flight, and returns; the block agrees on the
// outcome with __syncthreads_or, so no thread is left at a barrier.
#include "fused.cuh"

namespace dsfft {

namespace {

constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the mbarrier to complete; false after about
// kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

}  // namespace

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
struct FusedTma {
  using K = Fused<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename K::E;
  static constexpr int N = K::N;
  static constexpr int TPC = K::TPC;
  static constexpr int TPB = K::TPB;
  static constexpr int REGION_BYTES = K::PADN * (int)sizeof(E);
  static constexpr int BUF_BYTES = TPC * REGION_BYTES;
  static constexpr int SMEM = 16 + 2 * BUF_BYTES;   // two mbarriers, two buffers
  // Blocks per SM the shared memory allows (at most 2048 threads); the
  // register allocation is sized for that many.
  static constexpr int BY_SMEM = (227 * 1024) / (SMEM + 1024);
  static constexpr int BY_THREADS = 2048 / TPB;
  static constexpr int MINB = BY_SMEM < 1 ? 1 : BY_SMEM < BY_THREADS ? BY_SMEM : BY_THREADS;
  static_assert(K::NSTAGES > 1, "the bulk-copied input shares the exchange buffer");
  static_assert(REGION_BYTES % 16 == 0 && (N * sizeof(E)) % 16 == 0, "bulk copies move 16-byte multiples");
};

template <int PREC, int LOG2N, int LOG2R, bool SCALED>
__global__ void __launch_bounds__(FusedTma<PREC, LOG2N, LOG2R, SCALED>::TPB,
                                  FusedTma<PREC, LOG2N, LOG2R, SCALED>::MINB)
    fused_tma_fft_kernel(const typename Elem<PREC>::T *in, typename Elem<PREC>::T *out, int64_t batch,
                         const uint4 *__restrict__ tw, const __grid_constant__ Stage0Twiddles tw0, int *status,
                         uint32_t tx_extra) {
  using M = FusedTma<PREC, LOG2N, LOG2R, SCALED>;
  using K = typename M::K;
  using E = typename M::E;
  constexpr int N = M::N, TPC = M::TPC, T = K::T, R = K::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t bar0 = smem_addr(smem_raw);
  E *const buf0 = reinterpret_cast<E *>(smem_raw + 16);
  const int64_t tiles = (batch + TPC - 1) / TPC;

  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Thread 0: fill buffer b with tile `tile` (one copy per transform).
  // tx_extra (zero except under fault injection) raises the armed byte
  // count above what the copies deliver, so the wait runs out.
  auto issue = [&](int64_t tile, int b) {
    const int64_t first = tile * TPC;
    const int count = batch - first < TPC ? (int)(batch - first) : TPC;
    const uint32_t bar = bar0 + 8 * b;
    mbar_arrive_expect_tx(bar, (uint32_t)(count * N * sizeof(E)) + tx_extra);
    for (int t = 0; t < count; ++t)
      bulk_copy_g2s(smem_addr(reinterpret_cast<unsigned char *>(buf0) + b * M::BUF_BYTES + t * M::REGION_BYTES),
                    in + (first + t) * N, (uint32_t)(N * sizeof(E)), bar);
  };

  int64_t tile = blockIdx.x;
  if (threadIdx.x == 0) {
    if (tile < tiles) issue(tile, 0);
    if (tile + gridDim.x < tiles) issue(tile + gridDim.x, 1);
  }

  const int lt = threadIdx.x / T;
  const int tid = threadIdx.x % T;
  int k = 0;
  bool failed = false;
  for (; tile < tiles; ++k, tile += gridDim.x) {
    const int b = k & 1;
    const bool ok = mbar_wait(bar0 + 8 * b, (k >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // Every thread is done with tile k - 1: its buffer takes tile k + 1.
    if (k > 0 && threadIdx.x == 0 && tile + gridDim.x < tiles) issue(tile + gridDim.x, b ^ 1);

    const int64_t first = tile * TPC;
    const bool active = first + lt < batch;
    E *sm = reinterpret_cast<E *>(reinterpret_cast<unsigned char *>(buf0) + b * M::BUF_BYTES) + lt * K::PADN;
    E v[R];
    static_for<0, R>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      v[p] = sm[tid + p * T];
    });
    const auto tw0f = [&](int i) { return tw0.e[i]; };
    K::template stages<0, decltype(tw0f), true>(v, sm, tid, lt, tw, tw0f, active ? out + (first + lt) * N : nullptr,
                                                active);
    // This thread's reads and exchange writes of the buffer come before the
    // copy engine's next write into it.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (failed && threadIdx.x == 0) {
    atomicOr(status, 1);
    // Copies still in flight: the one that timed out (tile k), and tile
    // k + 1 when the prologue issued it (k = 0); later refills were not
    // issued.
    mbar_wait(bar0 + 8 * (k & 1), (k >> 1) & 1);
    if (k == 0 && tile + gridDim.x < tiles) mbar_wait(bar0 + 8, 0);
  }
}

}  // namespace dsfft

// ---------------------------------------------------------------------------
// dispatch (2^8 <= N <= 2^14, FP32 <= 2^13; the wide register block of
// fused.cuh)

namespace dsfft {

template <int PREC, int LOG2N, bool SCALED>
static cudaError_t launch_tma_one(const void *in, void *out, int64_t batch, const uint4 *tw, const Stage0Twiddles &tw0,
                                  int grid, int *status, uint32_t tx_extra, cudaStream_t stream) {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, false);
  using M = FusedTma<PREC, LOG2N, LOG2R, SCALED>;
  using E = typename M::E;
  const int64_t tiles = (batch + M::TPC - 1) / M::TPC;
  const unsigned g = (unsigned)(tiles < grid ? tiles : grid);
  fused_tma_fft_kernel<PREC, LOG2N, LOG2R, SCALED><<<g, M::TPB, M::SMEM, stream>>>(
      static_cast<const E *>(in), static_cast<E *>(out), batch, tw, tw0, status, tx_extra);
  return cudaGetLastError();
}

// Shared-memory limit of both scalings, and the resident blocks per SM.
template <int PREC, int LOG2N>
static cudaError_t prepare_tma_one(int *blocks_per_sm) {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, false);
  using M = FusedTma<PREC, LOG2N, LOG2R, false>;
  for (auto kern : {fused_tma_fft_kernel<PREC, LOG2N, LOG2R, false>, fused_tma_fft_kernel<PREC, LOG2N, LOG2R, true>}) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, M::SMEM);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, fused_tma_fft_kernel<PREC, LOG2N, LOG2R, true>, M::TPB, M::SMEM);
  if (e != cudaSuccess) return e;
  // carveout: the shared memory of the resident blocks, the rest stays L1
  const int carve = carveout_for(M::SMEM, *blocks_per_sm);
  for (auto kern : {fused_tma_fft_kernel<PREC, LOG2N, LOG2R, false>, fused_tma_fft_kernel<PREC, LOG2N, LOG2R, true>})
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <int PREC, int LOG2N>
static FusedShape shape_tma_one() {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N, false);
  using M = FusedTma<PREC, LOG2N, LOG2R, false>;
  return FusedShape{LOG2R, M::K::T, M::TPC, M::TPB, M::SMEM};
}

using TmaLaunchFn = cudaError_t (*)(const void *, void *, int64_t, const uint4 *, const Stage0Twiddles &, int, int *,
                                    uint32_t, cudaStream_t);
using TmaPrepareFn = cudaError_t (*)(int *);
using TmaShapeFn = FusedShape (*)();

template <int PREC, int... L>
struct TmaTable {
  static constexpr TmaLaunchFn plain[] = {launch_tma_one<PREC, L, false>...};
  static constexpr TmaLaunchFn scaled[] = {launch_tma_one<PREC, L, true>...};
  static constexpr TmaPrepareFn prepare[] = {prepare_tma_one<PREC, L>...};
  static constexpr TmaShapeFn shape[] = {shape_tma_one<PREC, L>...};
};

#define DSFFT_TMA_LOG2N_LIST 8, 9, 10, 11, 12, 13, 14
using Tma32 = TmaTable<kFP32, 8, 9, 10, 11, 12, 13>;
using Tma16 = TmaTable<kFP16, DSFFT_TMA_LOG2N_LIST>;
using TmaB16 = TmaTable<kBF16, DSFFT_TMA_LOG2N_LIST>;

// FP32 2^14 would need two 132 KB buffers: above the 227 KB of a block.
bool fused_tma_valid(int prec, int log2n) {
  return prec >= kFP32 && prec <= kBF16 && log2n >= kFusedTmaMinLog2N &&
         log2n <= (prec == kFP32 ? kFusedMaxLog2N - 1 : kFusedMaxLog2N);
}

FusedShape fused_tma_shape(int prec, int log2n) {
  if (!fused_tma_valid(prec, log2n)) return FusedShape{0, 0, 0, 0, 0};
  const int i = log2n - kFusedTmaMinLog2N;
  return prec == kFP32 ? Tma32::shape[i]() : prec == kFP16 ? Tma16::shape[i]() : TmaB16::shape[i]();
}

cudaError_t prepare_fused_tma(int prec, int log2n, int *grid) {
  if (!fused_tma_valid(prec, log2n) || !grid) return cudaErrorInvalidValue;
  const int i = log2n - kFusedTmaMinLog2N;
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = prec == kFP32 ? Tma32::prepare[i](&per_sm) : prec == kFP16 ? Tma16::prepare[i](&per_sm)
                                                                              : TmaB16::prepare[i](&per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_fused_tma(int prec, int log2n, bool scaled, const void *in, void *out, int64_t batch,
                             const uint4 *twp, const Stage0Twiddles &tw0, int grid, int *status, uint32_t tx_extra,
                             cudaStream_t stream) {
  if (!fused_tma_valid(prec, log2n) || grid < 1 || !status) return cudaErrorInvalidValue;
  if (batch <= 0) return cudaSuccess;
  const int i = log2n - kFusedTmaMinLog2N;
  const TmaLaunchFn f = prec == kFP32 ? (scaled ? Tma32::scaled[i] : Tma32::plain[i])
                        : prec == kFP16 ? (scaled ? Tma16::scaled[i] : Tma16::plain[i])
                                        : (scaled ? TmaB16::scaled[i] : TmaB16::plain[i]);
  return f(in, out, batch, twp, tw0, grid, status, tx_extra, stream);
}

}  // namespace dsfft
