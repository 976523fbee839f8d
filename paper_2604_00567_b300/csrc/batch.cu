// batch.cu — one persistent launch for a batch of transforms of mixed sizes
// (N <= 2^14) and precisions.
//
// The host groups the batch's transforms by (size, precision, direction
// table) into tiles of at most 1024/T transforms (T = threads per transform)
// and orders the tiles largest first.  Each resident block repeatedly takes
// the next tile from a device counter and runs it with the same register-stage
// code as the one-size kernel (fused.cuh), reading each transform through its
// own in/out pointers.  Every butterfly is the one the one-size launch runs,
// so each transform's result is bit-identical to transforming it alone.
#include "fused.cuh"

namespace dsfft {

constexpr int kBatchThreads = 1024;
// shared memory of the largest tile: 1024 threads x 16 eight-byte points
// (FP32) with one pad element per 16; FP16/BF16 tiles (32 four-byte points,
// one pad per 32) need less
constexpr int kBatchSmem = kBatchThreads * 16 * 8 * 17 / 16;
static_assert(kBatchSmem >= kBatchThreads * 32 * 4 * 33 / 32, "FP16 tiles fit");

template <int PREC, int LOG2N, bool SCALED>
__device__ __forceinline__ void batch_tile(const BatchTile &t, const BatchItem *items, unsigned char *smem) {
  constexpr int LOG2R = fused_log2r(PREC, LOG2N);
  using K = Fused<PREC, LOG2N, LOG2R, SCALED, kBatchThreads>;
  static_assert(K::NSTAGES == 1 || K::TPC * K::PADN * (int)sizeof(typename K::E) <= kBatchSmem, "tile fits");
  using E = typename K::E;
  const uint4 *tw = t.twp;
  K::run_tile(GatherIO<E>{items + t.first}, (int)t.count, tw, [tw](int i) { return tw_load<PREC>(tw, i); },
              reinterpret_cast<E *>(smem));
}

__global__ void __launch_bounds__(kBatchThreads, 1)
    batch_fft_kernel(const BatchTile *__restrict__ tiles, int ntiles, const BatchItem *__restrict__ items,
                     unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const BatchTile tile = tiles[t];
    switch (tile.path) {
#define DSFFT_BT(P, L)                                              \
  case batch_path_code(P, L, false):                               \
    batch_tile<P, L, false>(tile, items, smem);                    \
    break;                                                         \
  case batch_path_code(P, L, true):                                \
    batch_tile<P, L, true>(tile, items, smem);                     \
    break;
#define DSFFT_BT_ALL(P)                                                                                   \
  DSFFT_BT(P, 1) DSFFT_BT(P, 2) DSFFT_BT(P, 3) DSFFT_BT(P, 4) DSFFT_BT(P, 5) DSFFT_BT(P, 6) DSFFT_BT(P, 7) \
  DSFFT_BT(P, 8) DSFFT_BT(P, 9) DSFFT_BT(P, 10) DSFFT_BT(P, 11) DSFFT_BT(P, 12) DSFFT_BT(P, 13)          \
  DSFFT_BT(P, 14)
      DSFFT_BT_ALL(kFP32)
      DSFFT_BT_ALL(kFP16)
      DSFFT_BT_ALL(kBF16)
#undef DSFFT_BT_ALL
#undef DSFFT_BT
      default:
        break;
    }
    __syncthreads();   // the tile is done: shared memory and s_tile are free
  }
}

int batch_tile_capacity(int prec, int log2n) {
  const int r = fused_log2r(prec, log2n);
  const int t = 1 << (log2n - r);
  return kBatchThreads / t;
}

cudaError_t prepare_batch_kernel(int *grid) {
  cudaError_t e = cudaFuncSetAttribute(batch_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
  if (e != cudaSuccess) return e;
  // one block per SM: the rest of the L1/shared array stays L1
  e = cudaFuncSetAttribute(batch_fft_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           carveout_for(kBatchSmem, 1));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fft_kernel, kBatchThreads, kBatchSmem)) !=
      cudaSuccess)
    return e;
  *grid = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

cudaError_t launch_batch_kernel(const BatchTile *tiles, int ntiles, const BatchItem *items, unsigned *counter,
                                int grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  const int blocks = grid < ntiles ? grid : ntiles;
  batch_fft_kernel<<<blocks, kBatchThreads, kBatchSmem, stream>>>(tiles, ntiles, items, counter);
  return cudaGetLastError();
}

}  // namespace dsfft
