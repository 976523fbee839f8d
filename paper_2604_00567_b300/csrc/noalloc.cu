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
// The descriptors reach the array as the parameters of small copy kernels
// (the launch copies its parameters when it is issued), not by copies from
// host memory: the call neither waits for the stream's earlier work (as a
// copy from pageable memory would) nor leaves a copy that reads host memory
// later, when the host array may already hold the next call's descriptors.
//
// The scratch array is shared by every call: its contents are those of the
// last call (the work counter is cleared at the start of each call), and
// calls whose work overlaps on the GPU (e.g. on two streams) race on it.
// Host code reaches the array only through the address returned by
// cudaGetSymbolAddress, looked up with the device current on the first call
// made on that device (and again if that device's context was replaced, e.g.
// after cudaDeviceReset); device code in this file names it directly.
#include <cuda.h>
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
static_assert(kTilesOffset % 16 == 0 && kItemsOffset % 16 == 0, "16-byte words");
static_assert(sizeof(BatchTile) % 16 == 0 && sizeof(BatchItem) % 16 == 0, "16-byte words");

// One copy launch: up to two runs of 16-byte words carried in the kernel's
// parameters (32 KB parameter space, sm_70 and later with CUDA 12.1+).
constexpr int kChunkWords = 2032;
struct UploadChunk {
  uint32_t offset[2];   // byte offsets of the two runs in the scratch array
  uint32_t words[2];    // 16-byte words of each run (run 1 follows run 0 in data)
  uint4 data[kChunkWords];
};
static_assert(sizeof(UploadChunk) <= 32764, "kernel parameter limit");

}  // namespace

// The batch's device-side scratch: [counter | tiles | items].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void __launch_bounds__(256) noalloc_upload_kernel(const __grid_constant__ UploadChunk c) {
  const uint32_t n0 = c.words[0], n = n0 + c.words[1];
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t off = i < n0 ? c.offset[0] + 16u * i : c.offset[1] + 16u * (i - n0);
    *reinterpret_cast<uint4 *>(g_noalloc_scratch + off) = c.data[i];
  }
}

namespace {

std::mutex g_mu;                            // guards everything below
unsigned char *g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch per device
unsigned long long g_ctx_id[kMaxDevices];   // context the address belongs to
int g_grid[kMaxDevices];                    // persistent grid per device

// host staging (static: no heap allocation on this path); the copy kernels
// take their contents by value
BatchTile g_tiles[kMaxItems];
BatchItem g_items[kMaxItems];
UploadChunk g_chunk;
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

// Unique id of the current context (the driver's cuCtxGetId, reached through
// the runtime's entry-point query, so the library needs no link to libcuda).
cudaError_t current_context_id(unsigned long long *id) {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  cudaError_t e;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1)) != cudaSuccess)
      return e;
    if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2)) != cudaSuccess)
      return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<GetCurrent>(f1);
    get_id = reinterpret_cast<GetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Copies the runs (scratch offset, host source, bytes; multiples of 16) into
// the scratch array by copy-kernel launches on `st`, packing consecutive runs
// into each launch's parameters.
struct Run {
  size_t offset;
  const void *src;
  size_t bytes;
};
cudaError_t upload(const Run *runs, int nruns, cudaStream_t st) {
  int seg = 0;
  uint32_t used = 0;
  auto flush = [&]() -> cudaError_t {
    if (used == 0) return cudaSuccess;
    if (seg < 2) g_chunk.words[1] = 0;
    noalloc_upload_kernel<<<1, 256, 0, st>>>(g_chunk);
    seg = 0;
    used = 0;
    return cudaGetLastError();
  };
  for (int r = 0; r < nruns; ++r) {
    size_t done = 0;
    const size_t words = runs[r].bytes / 16;
    while (done < words) {
      if (seg == 2 || used == (uint32_t)kChunkWords) {
        const cudaError_t e = flush();
        if (e != cudaSuccess) return e;
      }
      const size_t take = std::min<size_t>(words - done, (size_t)kChunkWords - used);
      g_chunk.offset[seg] = (uint32_t)(runs[r].offset + 16 * done);
      g_chunk.words[seg] = (uint32_t)take;
      memcpy(&g_chunk.data[used], static_cast<const unsigned char *>(runs[r].src) + 16 * done, 16 * take);
      used += (uint32_t)take;
      done += take;
      ++seg;
    }
  }
  return flush();
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

  // one-time set-up on this device (again if its context was replaced):
  // the device address of the scratch array (the array's name is only a
  // host-side stand-in) and the launch grid
  unsigned long long ctx_id = 0;
  if ((e = current_context_id(&ctx_id)) != cudaSuccess) return cuda_fail(e, "current context");
  if (!g_scratch_dev[device] || g_ctx_id[device] != ctx_id) {
    void *p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    int grid = 0;
    if ((e = prepare_batch_kernel(&grid)) != cudaSuccess) return cuda_fail(e, "batch kernel attributes");
    g_grid[device] = grid;
    g_scratch_dev[device] = static_cast<unsigned char *>(p);
    g_ctx_id[device] = ctx_id;
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
  // descriptors into the scratch array by value (kernel parameters)
  const Run runs[2] = {{kItemsOffset, g_items, sizeof(BatchItem) * (size_t)count},
                       {kTilesOffset, g_tiles, sizeof(BatchTile) * (size_t)ntiles}};
  if ((e = upload(runs, ntiles > 0 ? 2 : 1, st)) != cudaSuccess) return cuda_fail(e, "descriptor upload");
  if (ntiles > 0) {
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
                                              j - i, k.view.twp[k.dir], *k.view.tw0[k.dir], k.view.tw1[k.dir],
                                              k.view.status, k.view.fault_tx, st)
                             : launch_sweeps(k.view.prec, k.view.log2n, scaled, nullptr, nullptr, d_items + i, j - i,
                                             k.view.twp[k.dir], st, k.view.sweep_ls1);
      if (e != cudaSuccess) return cuda_fail(e, "large-size launch");
    }
    i = j;
  }
  return FFT_OK;
}
