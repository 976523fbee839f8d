// internal.h — host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

struct fft_plan;   // the C ABI's opaque plan (defined in api.cu)

namespace dsfft {

enum Prec : int { kFP32 = 0, kFP16 = 1, kBF16 = 2 };

// Shared-memory carveout (percent of the SM's 228 KB maximum) that holds
// `blocks` resident blocks of `smem` dynamic bytes (plus the 1 KB the runtime
// reserves per block).  The runtime picks the smallest shared-memory
// configuration of the SM (0, 8, 16, 32, 64, 100, 132, 164, 196 or 228 KB on
// this architecture) at or above the percentage, so the percentage is that of
// the smallest configuration that fits, rounded down.  What the blocks do not
// need stays L1 (measured faster than the maximum carveout for the cluster,
// sweep and batch kernels: the cluster kernel's MIO-throttle and barrier
// stalls drop while its L1 hit rate hardly changes).
inline int carveout_for(int smem, int blocks) {
  static const int kConfigKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
  const long long need = (long long)(smem + 1024) * (blocks > 0 ? blocks : 1);
  int kb = 228;
  for (int c : kConfigKB)
    if (1024LL * c >= need) {
      kb = c;
      break;
    }
  const int carve = (int)(100LL * kb / 228);
  return carve < 1 ? 1 : carve;
}

// One transform of a mixed batch: device pointers to its input and output.
struct BatchItem {
  const void *in;
  void *out;
};

// One unit of work of the persistent batch kernel: `count` transforms of
// one size/precision/direction, items [first, first + count).
struct BatchTile {
  uint32_t path;      // batch_path_code(prec, log2n, scaled)
  uint32_t count;
  uint32_t first;
  uint32_t reserved;
  const uint4 *twp;   // per-pass twiddle table of the direction
  uint64_t reserved2;
};

__host__ __device__ constexpr uint32_t batch_path_code(int prec, int log2n, bool scaled) {
  return (uint32_t)((((prec * 32) + log2n) << 1) | (scaled ? 1 : 0));
}

constexpr int kMaxLog2N = 24;
constexpr int kFusedMaxLog2N = 14;   // whole transform staged on chip

// Packed table entries for k in [0, count), multiplier times mscale (1, 1/2
// or 1/4).
cudaError_t launch_build_table(int log2n, int64_t count, int fac, double eps, int prec, int inverse, double mscale,
                               uint4 *out, int *counts, cudaStream_t stream);
// Per-pass table entries [0, count) of the N - 1 in form `form` (table.cu
// put_entry): 0 the 16-byte packed entry, 1 the compact 8-byte FP16/BF16
// entry, 2 the compact 8-byte FP32 entry (the kernels read forms 1 and 2,
// common.cuh TwEntry).
cudaError_t launch_per_pass_table(int log2n, const uint4 *table, void *twp, int64_t count, int form,
                                  cudaStream_t stream);

// Radix-4 passes (at levels par, par + 2, ..., par = log2 N mod 2; one
// radix-2 pass at level 0 first when log2 N is odd): offset of level l in
// the per-pass radix-4 table, which holds N - 1 - par entries in all.
__host__ __device__ constexpr int64_t r4_offset(int l, int par) { return (int64_t(1) << l) - 1 - par; }
cudaError_t launch_per_pass_table4(int log2n, const uint4 *table4, void *twp4, int64_t count, int form,
                                   cudaStream_t stream);
cudaError_t launch_fp64_table(int log2n, int fac, double eps, double *t, double *m, int *path,
                              cudaStream_t stream);

// Shape of the fused kernel for (prec, log2n).
struct FusedShape {
  int log2r;                 // points per thread = 2^log2r
  int threads_per_transform;
  int transforms_per_block;
  int threads_per_block;
  int smem_bytes;
};
// `narrow`: the half-width register block (see fused_log2r); it exists for a
// size when fused_has_narrow, otherwise the wide kernel runs.
FusedShape fused_shape(int prec, int log2n, bool narrow = false);
bool fused_has_narrow(int prec, int log2n);
cudaError_t prepare_fused(int prec, int log2n, bool narrow = false);

// Persistent fused kernel fed by bulk copies (fused_tma.cu), 2^8 <= N <=
// 2^14 (FP32: 2^13).  `grid`: the resident blocks of the device (prepare_fused_tma);
// `status`: device word whose bit 0 a block sets when a bounded wait for its
// copies gives up; `tx_extra` (fault injection, normally 0) is added to the
// byte count each copy barrier expects.  `in` must be 16-byte aligned.
constexpr int kFusedTmaMinLog2N = 8;
bool fused_tma_valid(int prec, int log2n);
FusedShape fused_tma_shape(int prec, int log2n);
cudaError_t prepare_fused_tma(int prec, int log2n, int *grid);

// Twiddles of the first register stage (passes 0 .. log2(R)-1, whose j is 0
// for every thread): the first 2^r - 1 per-pass entries, passed by value so
// the kernel reads them from the constant bank.
struct Stage0Twiddles {
  uint4 e[31];
};

// Twiddles of every phase-1 pass of the FP32 cluster kernel (passes 0 .. 7
// of N = 2^15 and 2^16: the first 255 per-pass entries, the same for every
// CTA), passed by value like Stage0Twiddles.  The FP16/BF16 cluster kernels
// read their later phase-1 twiddles from the per-pass table instead (measured
// faster there).
struct Phase1Twiddles {
  uint4 e[255];
};

// Fused on-chip transform of `batch` signals of length 2^log2n.  `twp` is
// the device per-pass table, `tw0` its first entries.
cudaError_t launch_fused(int prec, int log2n, bool narrow, bool scaled, const void *in, void *out, int64_t batch,
                         const uint4 *twp, const Stage0Twiddles &tw0, cudaStream_t stream);

cudaError_t launch_fused_tma(int prec, int log2n, bool scaled, const void *in, void *out, int64_t batch,
                             const uint4 *twp, const Stage0Twiddles &tw0, int grid, int *status, uint32_t tx_extra,
                             cudaStream_t stream);

// N > 2^14: two sweeps over HBM (passes [0, ls1) then the rest; ls1 = 0
// picks ceil(m/2)).  Both sweeps hold 7..12 passes (sweep_ls1_valid).
// `in` and `out` must differ; sweep 2 runs in place on `out`.
void sweep_split(int log2n, int *ls1, int *ls2);
bool sweep_ls1_valid(int log2n, int ls1);
// SMs of the current device (cached per device; 0 when unknown): the sweeps
// switch to their narrow-group kernels at or below one block per two SMs.
int sweep_sm_count();
cudaError_t prepare_sweeps(int prec, int log2n, int ls1 = 0);
// `items` (device array, one per transform) replaces in/out when non-null.
cudaError_t launch_sweeps(int prec, int log2n, bool scaled, const void *in, void *out, const BatchItem *items,
                          int64_t batch, const uint4 *twp, cudaStream_t stream, int ls1 = 0);

// Radix-4 plans, N > 2^14: two sweeps of whole radix-4 passes (sweep 1 also
// holds the radix-2 pass of an odd log2 N); `twp4` the per-pass radix-4
// table, `r2e` the radix-2 entry k = 0.
void sweep_split4(int log2n, int *ls1, int *ls2);
cudaError_t prepare_sweeps4(int prec, int log2n);
cudaError_t launch_sweeps4(int prec, int log2n, bool scaled, int inverse, const void *in, void *out,
                           const BatchItem *items, int64_t batch, const uint4 *twp4, const uint4 &r2e,
                           cudaStream_t stream);

// 2^15 <= N <= 2^17 (FP16/BF16) or <= 2^16 (FP32): one launch on a cluster
// of 2^cluster_log2k CTAs whose distributed shared memory holds the
// transform between the two halves of the passes.  -1 = not handled.
int cluster_log2k(int prec, int log2n);
cudaError_t prepare_cluster(int prec, int log2n);
// `tw0`: the first per-pass entries (the fused kernel's stage-0 twiddles);
// `tw1`: every phase-1 entry (FP32 only, required there).
// `status`: device word whose bit 1 a CTA sets when its bounded wait for
// the phase-1 data gives up (the FP16/BF16 kernels); `tx_extra`
// (fault injection, normally 0) is added to the bytes that wait expects.
cudaError_t launch_cluster(int prec, int log2n, bool scaled, const void *in, void *out, const BatchItem *items,
                           int64_t batch, const uint4 *twp, const Stage0Twiddles &tw0, const Phase1Twiddles *tw1,
                           int *status, uint32_t tx_extra, cudaStream_t stream);

// Read-only view of a plan's launch parameters (for entry points outside
// api.cu); false for a null plan.
struct PlanView {
  int device, kernel, prec, log2n;
  int scale[2];
  const uint4 *twp[2];
  const Stage0Twiddles *tw0[2];   // host copies of the first per-pass entries
  const Phase1Twiddles *tw1[2];   // FP32 cluster plans: every phase-1 entry (else null)
  int radix;                      // 2 or 4
  int sweep_ls1;                  // passes in sweep 1 (0: ceil(m/2))
  int *status;                    // device error word of the bounded waits
  uint32_t fault_tx;              // fault injection: extra bytes each bounded copy wait expects (normally 0)
};

// Host-side trace range around a library call (NVTX: visible in Nsight
// timelines and usable as an ncu --nvtx filter; no cost without a tool).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

bool plan_view(const ::fft_plan *p, PlanView *v);
void set_last_error(const char *msg);

// cudaMalloc for every buffer the library owns.  Fault injection for tests:
// with the environment variable DSFFT_FAULT_ALLOC=k set, the k-th call after
// the variable took its current value fails with cudaErrorMemoryAllocation
// (nothing is allocated); unset, it is plain cudaMalloc.
cudaError_t device_alloc(void **ptr, size_t bytes);
template <class T>
cudaError_t device_alloc(T **ptr, size_t bytes) {
  return device_alloc(reinterpret_cast<void **>(ptr), bytes);
}

// Radix-4 fused kernel (N <= 2^14): per-pass radix-4 table and first-stage
// twiddles (fused4.cuh); `inverse` selects the +i of the inverse butterflies.
struct Stage0R4;
FusedShape fused4_shape(int prec, int log2n);
cudaError_t prepare_fused4(int prec, int log2n);
cudaError_t launch_fused4(int prec, int log2n, bool scaled, int inverse, const void *in, void *out, int64_t batch,
                          const uint4 *twp4, const Stage0R4 &tw0, cudaStream_t stream);

// Persistent mixed-size batch kernel (N <= 2^14, any precision).
int batch_tile_capacity(int prec, int log2n);
cudaError_t prepare_batch_kernel(int *grid);
cudaError_t launch_batch_kernel(const BatchTile *tiles, int ntiles, const BatchItem *items, unsigned *counter,
                                int grid, cudaStream_t stream);

}  // namespace dsfft
