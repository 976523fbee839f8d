// noalloc.cu — fft_exec_batch_noalloc: run a mixed batch without allocating
// any device memory.
//
// Who needs this: callers that cannot call cudaMalloc on the path where they
// transform — a host program that owns all device memory through its own
// fixed pool and gives libraries no allocator, or a latency-bound loop where
// cudaMalloc/cudaFree would stall on their implicit device synchronisation.
// fft_batch_create allocates the work descriptors and the work counter of a
// batch; this entry point instead keeps them in one file-scope device array
// of fixed size, g_noalloc_scratch, that exists in every GPU that loads the
// library until the process exits.  The caller passes plans (created
// beforehand) and the input/output buffers; nothing else is allocated.
//
// The scratch array is shared by every call: its contents are those of the
// last call (the work counter is cleared at the start of each call), and
// calls whose work overlaps on the GPU (e.g. on two streams) race on it.
// Host code reaches the array only through the address returned by
// cudaGetSymbolAddress, looked up once per device with that device current,
// on the first call made on that device.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/dsfft.h"
#include "internal.h"

namespace dsfft {
namespace {

constexpr int kMaxItems = FFT_NOALLOC_MAX_ITEMS;
constexpr size_t kCounterBytes = 256;                                  // work counter, padded
constexpr size_t kTilesOffset = kCounterBytes;
constexpr size_t kItemsOffset = kTilesOffset + sizeof(BatchTile) * kMaxItems;
constexpr size_t kScratchBytes = kItemsOffset + sizeof(BatchItem) * kMaxItems;
constexpr int kMaxDevices = 64;

}  // namespace

// The batch's device-side scratch: [counter | tiles | items].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;                          // guards everything below
unsigned char *g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch per device
int g_grid[kMaxDevices];                  // persistent grid per device

// host staging (static: no heap allocation on this path)
BatchTile g_tiles[kMaxItems];
BatchItem g_items[kMaxItems];
struct Key {
  PlanView view;
  const void *plan;
  int dir;
  int index;
};
Key g_keys[kMaxItems];

bool key_less(const Key &a, const Key &b) {
  const bool la = a.view.kernel != 0, lb = b.view.kernel != 0;
  if (la != lb) return la < lb;                               // persistent-kernel sizes first
  if (a.view.log2n != b.view.log2n) return a.view.log2n > b.view.log2n;
  if (a.plan != b.plan) return a.plan < b.plan;
  if (a.dir != b.dir) return a.dir < b.dir;
  return a.index < b.index;
}

fft_status fail(fft_status s, const char *msg) {
  set_last_error(msg);
  return s;
}

fft_status cuda_fail(cudaError_t e, const char *where) {
  char buf[200];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  set_last_error(buf);
  return FFT_ERR_CUDA;
}

}  // namespace
}  // namespace dsfft

using namespace dsfft;

extern "C" fft_status fft_exec_batch_noalloc(const fft_noalloc_item *items, int64_t count, void *stream) {
  if (count < 0 || (count > 0 && !items)) return FFT_ERR_INVALID_ARG;
  if (count > kMaxItems)
    return fail(FFT_ERR_INVALID_SIZE, "fft_exec_batch_noalloc: more than FFT_NOALLOC_MAX_ITEMS (4096) items");
  if (count == 0) return FFT_OK;
  TraceRange trace("dsfft exec_batch_noalloc");
  int device = -1;
  for (int64_t i = 0; i < count; ++i) {
    const fft_noalloc_item &it = items[i];
    PlanView v;
    if (!plan_view(it.plan, &v)) return FFT_ERR_INVALID_ARG;
    if (it.direction != FFT_FORWARD && it.direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if (it.reserved != 0 || !it.in || !it.out) return FFT_ERR_INVALID_ARG;
    if (v.radix != 2) return fail(FFT_ERR_UNSUPPORTED, "fft_exec_batch_noalloc: radix-4 plans are not batched");
    const uintptr_t eb = v.prec == kFP32 ? 8 : 4;
    if (((uintptr_t)it.in % eb) != 0 || ((uintptr_t)it.out % eb) != 0) return FFT_ERR_INVALID_ARG;
    if (v.kernel == 1 && it.in == it.out)
      return fail(FFT_ERR_UNSUPPORTED, "fft_exec_batch_noalloc: in-place transform on the HBM-sweep path");
    if (device < 0) device = v.device;
    if (v.device != device) return fail(FFT_ERR_INVALID_ARG, "fft_exec_batch_noalloc: plans on different devices");
  }
  if (device >= kMaxDevices) return fail(FFT_ERR_UNSUPPORTED, "fft_exec_batch_noalloc: device ordinal too large");

  std::lock_guard<std::mutex> lock(g_mu);
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  struct Restore {
    int prev, device;
    ~Restore() {
      if (prev != device) cudaSetDevice(prev);
    }
  } restore{prev, device};

  // one-time set-up on this device: the device address of the scratch array
  // (the array's name is only a host-side stand-in) and the launch grid
  if (!g_scratch_dev[device]) {
    void *p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    int grid = 0;
    if ((e = prepare_batch_kernel(&grid)) != cudaSuccess) return cuda_fail(e, "batch kernel attributes");
    g_grid[device] = grid;
    g_scratch_dev[device] = static_cast<unsigned char *>(p);
  }
  unsigned char *base = g_scratch_dev[device];
  unsigned *d_counter = reinterpret_cast<unsigned *>(base);
  BatchTile *d_tiles = reinterpret_cast<BatchTile *>(base + kTilesOffset);
  BatchItem *d_items = reinterpret_cast<BatchItem *>(base + kItemsOffset);

  // group the items: persistent-kernel sizes (largest first), then the rest
  for (int64_t i = 0; i < count; ++i) {
    plan_view(items[i].plan, &g_keys[i].view);
    g_keys[i].plan = items[i].plan;
    g_keys[i].dir = items[i].direction == FFT_FORWARD ? 0 : 1;
    g_keys[i].index = (int)i;
  }
  std::sort(g_keys, g_keys + count, key_less);
  int ntiles = 0;
  for (int64_t i = 0; i < count; ++i)
    g_items[i] = BatchItem{items[g_keys[i].index].in, items[g_keys[i].index].out};
  for (int64_t i = 0; i < count;) {
    const Key &k = g_keys[i];
    int64_t j = i;
    while (j < count && g_keys[j].plan == k.plan && g_keys[j].dir == k.dir) ++j;
    if (k.view.kernel == 0) {
      const int cap = batch_tile_capacity(k.view.prec, k.view.log2n);
      for (int64_t t = i; t < j; t += cap) {
        BatchTile tile;
        memset(&tile, 0, sizeof tile);
        tile.path = batch_path_code(k.view.prec, k.view.log2n, k.view.scale[k.dir] != 0);
        tile.count = (uint32_t)std::min<int64_t>(cap, j - t);
        tile.first = (uint32_t)t;
        tile.twp = k.view.twp[k.dir];
        g_tiles[ntiles++] = tile;
      }
    }
    i = j;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // pageable sources: each copy has read the host array when it returns
  if ((e = cudaMemcpyAsync(d_items, g_items, sizeof(BatchItem) * (size_t)count, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_fail(e, "copy items");
  if (ntiles > 0) {
    if ((e = cudaMemcpyAsync(d_tiles, g_tiles, sizeof(BatchTile) * (size_t)ntiles, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return cuda_fail(e, "copy tiles");
    // clears the work counter, then launches the persistent kernel
    if ((e = launch_batch_kernel(d_tiles, ntiles, d_items, d_counter, g_grid[device], st)) != cudaSuccess)
      return cuda_fail(e, "batch kernel launch");
  }
  for (int64_t i = 0; i < count;) {
    const Key &k = g_keys[i];
    int64_t j = i;
    while (j < count && g_keys[j].plan == k.plan && g_keys[j].dir == k.dir) ++j;
    if (k.view.kernel != 0) {
      const bool scaled = k.view.scale[k.dir] != 0;
      e = k.view.kernel == 2 ? launch_cluster(k.view.prec, k.view.log2n, scaled, nullptr, nullptr, d_items + i,
                                              j - i, k.view.twp[k.dir], *k.view.tw0[k.dir], k.view.status,
                                              k.view.fault_tx, st)
                             : launch_sweeps(k.view.prec, k.view.log2n, scaled, nullptr, nullptr, d_items + i, j - i,
                                             k.view.twp[k.dir], st, k.view.sweep_ls1);
      if (e != cudaSuccess) return cuda_fail(e, "large-size launch");
    }
    i = j;
  }
  return FFT_OK;
}
