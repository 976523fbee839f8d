// api.cu — the C ABI of libdsfft (declared in include/dsfft.h): plan
// creation (FP64 table build on the GPU, rounding once, resident packed
// tables for both directions), execution dispatch and error reporting.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dsfft.h"
#include "fused4.cuh"
#include "internal.h"

using namespace dsfft;

struct fft_plan {
  int64_t n;
  int log2n;
  int prec;
  int fac;
  double eps;
  int scale[2];         // [0] forward, [1] inverse
  int device;
  uint4 *table[2];      // packed tables (N/2 entries), [0] forward, [1] inverse
  uint4 *twp[2];        // per-pass copies (N - 1 entries) read by the kernels
  Stage0Twiddles tw0[2];  // host copy of the first min(N, 32) - 1 per-pass entries
  Phase1Twiddles tw1[2];  // FP32 N = 2^15, 2^16: host copy of the first 255 per-pass entries
  bool has_tw1;           // tw1 filled (FP32 plans of the cluster sizes)
  int kernel;           // 0 fused, 1 sweeps, 2 cluster
  bool narrow;          // fused: half-width register block
  int variant;          // fft_variant
  int autotuned;        // 0 built-in, 1 timed, 2 cache
  FusedShape shape;
  int cos_count, sin_count;
  int radix;            // 2, or 4 (radix-4 passes, fused kernel only)
  uint4 *table4[2];     // radix-4: packed table, k in [0, 3N/4)
  uint4 *twp4[2];       // radix-4: per-pass table (N - 1 - log2 N mod 2 entries)
  Stage0R4 s0r4[2];     // radix-4: first-stage twiddles (host copy)
  int sweep_ls1;        // sweeps: passes in sweep 1 (0: ceil(m/2))
  int tma_grid;         // fused_tma: resident blocks of the device
  uint32_t fault_tx;     // fault injection (DSFFT_FAULT_WAIT): extra bytes each bounded copy wait expects, else 0
  int *status;          // device error word of the bounded waits
};

namespace {

thread_local char g_last_error[256] = "";

fft_status cuda_fail(cudaError_t e, const char *where) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return FFT_ERR_OOM;
  return FFT_ERR_CUDA;
}

// Make `device` current for the lifetime of the guard (device < 0 keeps the
// caller's current device), restoring the caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int device) {
    if (device < 0) return;
    err = cudaGetDevice(&prev);
    if (err != cudaSuccess) return;
    if (prev != device) {
      err = cudaSetDevice(device);
      switched = err == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

bool variant_valid(int prec, int log2n, int v) {
  switch (v) {
    case FFT_VARIANT_FUSED_WIDE: return log2n <= kFusedMaxLog2N;
    case FFT_VARIANT_FUSED_NARROW: return log2n <= kFusedMaxLog2N && fused_has_narrow(prec, log2n);
    case FFT_VARIANT_CLUSTER: return log2n > kFusedMaxLog2N && cluster_log2k(prec, log2n) >= 0;
    case FFT_VARIANT_SWEEPS: return log2n > kFusedMaxLog2N;
    case FFT_VARIANT_FUSED_TMA: return fused_tma_valid(prec, log2n);
  }
  return false;
}

// Built-in choice: the variant the autotuner measured fastest on a B300 for
// each size (128 MiB batches; opts.autotune re-measures on the running GPU).
int default_variant(int prec, int log2n) {
  if (log2n <= kFusedMaxLog2N) {
    const bool narrow = prec == kFP32 ? (log2n >= 5 && log2n <= 7)
                                      : (log2n >= 5 && log2n <= 8);
    return narrow && fused_has_narrow(prec, log2n) ? FFT_VARIANT_FUSED_NARROW : FFT_VARIANT_FUSED_WIDE;
  }
  if (cluster_log2k(prec, log2n) >= 0) return FFT_VARIANT_CLUSTER;   // 2^15..2^17 (FP32 2^16)
  return FFT_VARIANT_SWEEPS;
}

// Built-in passes in sweep 1 for the sweeps variant (0: ceil(m/2)): the
// split measured fastest on a B300 (256 MiB batches; FP32 2^18: 10 + 8
// passes 30.3 % of HBM against 28.6 % for 8 + 10 and 24.8 % for 9 + 9;
// FP16 2^20: 11 + 9 21.9 % against 20.9 % for 10 + 10).
int default_sweep_ls1(int prec, int log2n) {
  switch (log2n) {
    case 17: return prec == kFP32 ? 10 : 8;
    case 18: return prec == kFP32 ? 10 : 9;
    case 19: return prec == kFP32 ? 11 : 9;
    case 20: return prec == kFP32 ? 12 : 11;
    case 21: return prec == kFP32 ? 10 : 12;
    case 22: return prec == kFP32 ? 11 : 12;
  }
  return 0;
}

// Make the plan run variant v (valid for its size): kernel choice and the
// kernels' attributes on the current device.
cudaError_t apply_variant(fft_plan *p, int v) {
  p->variant = v;
  p->narrow = v == FFT_VARIANT_FUSED_NARROW;
  p->kernel = v == FFT_VARIANT_FUSED_WIDE || v == FFT_VARIANT_FUSED_NARROW || v == FFT_VARIANT_FUSED_TMA ? 0
              : v == FFT_VARIANT_CLUSTER                                                                  ? 2
                                                                                                          : 1;
  p->shape = fused_shape(p->prec, p->log2n < kFusedMaxLog2N ? p->log2n : kFusedMaxLog2N, p->narrow);
  if (v == FFT_VARIANT_FUSED_TMA) {
    p->shape = fused_tma_shape(p->prec, p->log2n);
    // the wide kernel also runs, for inputs that are not 16-byte aligned
    const cudaError_t e = prepare_fused(p->prec, p->log2n, false);
    return e != cudaSuccess ? e : prepare_fused_tma(p->prec, p->log2n, &p->tma_grid);
  }
  if (p->kernel == 0) return prepare_fused(p->prec, p->log2n, p->narrow);
  if (p->kernel == 2) return prepare_cluster(p->prec, p->log2n);
  return prepare_sweeps(p->prec, p->log2n, p->sweep_ls1);
}

// Queue one transform batch of plan p on `stream` (d: 0 forward, 1 inverse).
cudaError_t plan_launch(const fft_plan *p, const void *in, void *out, int64_t batch, int d, cudaStream_t stream) {
  const bool scaled = p->scale[d] != 0;
  if (p->radix == 4) {
    if (p->kernel == 1)
      return launch_sweeps4(p->prec, p->log2n, scaled, d, in, out, nullptr, batch, p->twp4[d], p->s0r4[d].r2, stream);
    return launch_fused4(p->prec, p->log2n, scaled, d, in, out, batch, p->twp4[d], p->s0r4[d], stream);
  }
  if (p->variant == FFT_VARIANT_FUSED_TMA && ((uintptr_t)in & 15) == 0)
    return launch_fused_tma(p->prec, p->log2n, scaled, in, out, batch, p->twp[d], p->tw0[d], p->tma_grid, p->status,
                            p->fault_tx, stream);
  if (p->kernel == 0)
    return launch_fused(p->prec, p->log2n, p->narrow, scaled, in, out, batch, p->twp[d], p->tw0[d], stream);
  if (p->kernel == 2)
    return launch_cluster(p->prec, p->log2n, scaled, in, out, nullptr, batch, p->twp[d], p->tw0[d],
                          p->has_tw1 ? &p->tw1[d] : nullptr,
                          p->status, p->fault_tx, stream);
  return launch_sweeps(p->prec, p->log2n, scaled, in, out, nullptr, batch, p->twp[d], stream, p->sweep_ls1);
}

// ---- autotune cache: a JSON object {"<gpu>|<prec>|<log2n>|<fac>": variant, ...}
std::mutex g_cache_mu;

std::map<std::string, int> cache_read(const char *path) {
  std::map<std::string, int> m;
  FILE *f = fopen(path, "rb");
  if (!f) return m;
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  fclose(f);
  size_t i = 0;
  while ((i = text.find('"', i)) != std::string::npos) {
    const size_t j = text.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = text.substr(i + 1, j - i - 1);
    size_t c = text.find_first_not_of(" \t\r\n", j + 1);
    if (c != std::string::npos && text[c] == ':') {
      c = text.find_first_not_of(" \t\r\n", c + 1);
      if (c != std::string::npos && (isdigit((unsigned char)text[c]) || text[c] == '-')) m[key] = atoi(text.c_str() + c);
    }
    i = j + 1;
  }
  return m;
}

void cache_write(const char *path, const std::map<std::string, int> &m) {
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  fprintf(f, "{\n  \"format\": 1");
  for (const auto &kv : m)
    if (kv.first != "format") fprintf(f, ",\n  \"%s\": %d", kv.first.c_str(), kv.second);
  fprintf(f, "\n}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

// Time every valid variant of plan p on a 128 MiB batch and keep the
// fastest (forward direction).
// Candidate (variant, passes in sweep 1) of the autotuner: every variant
// the size has, the sweeps with each valid split within two passes of the
// balanced one (the measured best splits of a B300 lie there, e.g. FP32
// 2^20: 12 + 8).  Cached as variant * 100 + passes (0: the default split).
struct Candidate {
  int variant, ls1;
};

cudaError_t apply_candidate(fft_plan *p, const Candidate &c) {
  p->sweep_ls1 = c.variant == FFT_VARIANT_SWEEPS ? c.ls1 : 0;
  return apply_variant(p, c.variant);
}

cudaError_t autotune_plan(fft_plan *p) {
  Candidate cands[16];
  int nc = 0;
  for (int v = FFT_VARIANT_FUSED_WIDE; v <= FFT_VARIANT_FUSED_TMA; ++v) {
    if (!variant_valid(p->prec, p->log2n, v)) continue;
    if (v != FFT_VARIANT_SWEEPS) {
      cands[nc++] = Candidate{v, 0};
      continue;
    }
    const int mid = (p->log2n + 1) / 2;
    for (int l = mid - 2; l <= mid + 2; ++l)
      if (sweep_ls1_valid(p->log2n, l)) cands[nc++] = Candidate{v, l};
  }
  if (nc < 2) return cudaSuccess;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
  if (e != cudaSuccess) return e;
  char key[384];
  snprintf(key, sizeof key, "%s|%d|%d|%d", prop.name, p->prec, p->log2n, p->fac);
  const char *path = getenv("DSFFT_AUTOTUNE_CACHE");
  if (path && *path) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto m = cache_read(path);
    auto it = m.find(key);
    if (it != m.end()) {
      const int val = it->second;
      const Candidate c{val >= 100 ? val / 100 : val, val >= 100 ? val % 100 : 0};
      if (variant_valid(p->prec, p->log2n, c.variant) &&
          (c.ls1 == 0 || (c.variant == FFT_VARIANT_SWEEPS && sweep_ls1_valid(p->log2n, c.ls1)))) {
        p->autotuned = 2;
        return apply_candidate(p, c);
      }
    }
  }
  const size_t eb = p->prec == kFP32 ? 8 : 4;
  const size_t tbytes = (size_t)p->n * eb;
  const int64_t batch = std::max<int64_t>(1, (int64_t)((128u << 20) / tbytes));
  void *in = nullptr, *out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int best = -1;
  float best_ms = 0.f;
  do {
    if ((e = device_alloc(&in, tbytes * batch)) != cudaSuccess) break;
    if ((e = device_alloc(&out, tbytes * batch)) != cudaSuccess) break;
    if ((e = cudaMemset(in, 0x11, tbytes * batch)) != cudaSuccess) break;   // finite, normal values
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) break;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
      if ((e = apply_candidate(p, cands[c])) != cudaSuccess) break;
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = plan_launch(p, in, out, batch, 0, st);
      if (e != cudaSuccess) break;
      if ((e = cudaEventRecord(a, st)) != cudaSuccess) break;
      for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = plan_launch(p, in, out, batch, 0, st);
      if (e != cudaSuccess) break;
      if ((e = cudaEventRecord(b, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) break;
      if (best < 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
  } while (0);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return e;
  p->autotuned = 1;
  if (path && *path) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto m = cache_read(path);
    m[key] = cands[best].ls1 ? cands[best].variant * 100 + cands[best].ls1 : cands[best].variant;
    cache_write(path, m);
  }
  return apply_candidate(p, cands[best]);
}

int ilog2_exact(int64_t n) {
  if (n < 2 || (n & (n - 1)) != 0) return -1;
  int l = 0;
  while ((1LL << l) < n) ++l;
  return l;
}

size_t elem_bytes(int prec) { return prec == kFP32 ? 8 : 4; }

}  // namespace

bool dsfft::plan_view(const fft_plan *p, PlanView *v) {
  if (!p || !v) return false;
  v->device = p->device;
  v->kernel = p->kernel;
  v->prec = p->prec;
  v->log2n = p->log2n;
  v->scale[0] = p->scale[0];
  v->scale[1] = p->scale[1];
  v->twp[0] = p->twp[0];
  v->twp[1] = p->twp[1];
  v->tw0[0] = &p->tw0[0];
  v->tw0[1] = &p->tw0[1];
  v->tw1[0] = p->has_tw1 ? &p->tw1[0] : nullptr;
  v->tw1[1] = p->has_tw1 ? &p->tw1[1] : nullptr;
  v->radix = p->radix;
  v->sweep_ls1 = p->sweep_ls1;
  v->status = p->status;
  v->fault_tx = p->fault_tx;
  return true;
}

void dsfft::set_last_error(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

cudaError_t dsfft::device_alloc(void **ptr, size_t bytes) {
  static std::mutex mu;
  static std::string seen;
  static long count = 0;
  const char *v = getenv("DSFFT_FAULT_ALLOC");
  if (v && *v) {
    std::lock_guard<std::mutex> lk(mu);
    if (seen != v) {
      seen = v;
      count = 0;
    }
    if (++count == atol(v)) {
      *ptr = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(ptr, bytes);
}

extern "C" {

struct fft_batch {
  int device = 0;
  std::vector<fft_plan *> plans;
  int64_t count = 0;
  BatchItem *d_items = nullptr;     // items reordered by group
  BatchTile *d_tiles = nullptr;
  unsigned *d_counter = nullptr;
  int ntiles = 0;
  int grid = 0;
  struct Large {
    const fft_plan *plan;
    int dir;                        // 0 forward, 1 inverse
    int64_t first, count;           // slice of d_items
  };
  std::vector<Large> large;
  // internal streams for the large groups (forked from the caller's stream
  // by `fork`, joined back by `join`), so that they overlap one another and
  // the persistent kernel's tail; in a captured graph they are parallel
  // branches
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t device_bytes = 0;
};

namespace {

// Queue every launch of the batch: the large groups round-robin on the
// internal streams, forked from and joined back to `stream`, then the
// persistent kernel on `stream` (work after the call on `stream` waits for
// all of it).  The large groups go first: the persistent kernel takes its
// tiles dynamically, so it fills the SMs their tails leave idle (measured:
// mixed batch of 4096 transforms 0.258 ms against 0.267 ms the other way).
cudaError_t batch_enqueue(const fft_batch *b, cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  const size_t nside = b->side.size();
  if (nside > 0) {
    if ((e = cudaEventRecord(b->fork, stream)) != cudaSuccess) return e;
    for (cudaStream_t s : b->side)
      if ((e = cudaStreamWaitEvent(s, b->fork, 0)) != cudaSuccess) return e;
  }
  for (size_t k = 0; k < b->large.size(); ++k) {
    const auto &g = b->large[k];
    const fft_plan *p = g.plan;
    const bool scaled = p->scale[g.dir] != 0;
    cudaStream_t st = nside > 0 ? b->side[k % nside] : stream;
    if (p->kernel == 2)
      e = launch_cluster(p->prec, p->log2n, scaled, nullptr, nullptr, b->d_items + g.first, g.count, p->twp[g.dir],
                         p->tw0[g.dir], p->has_tw1 ? &p->tw1[g.dir] : nullptr, p->status, p->fault_tx, st);
    else
      e = launch_sweeps(p->prec, p->log2n, scaled, nullptr, nullptr, b->d_items + g.first, g.count, p->twp[g.dir],
                        st, p->sweep_ls1);
    if (e != cudaSuccess) return e;
  }
  if (b->ntiles > 0) {
    e = launch_batch_kernel(b->d_tiles, b->ntiles, b->d_items, b->d_counter, b->grid, stream);
    if (e != cudaSuccess) return e;
  }
  for (size_t i = 0; i < nside; ++i) {
    if ((e = cudaEventRecord(b->join[i], b->side[i])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(stream, b->join[i], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void batch_release(fft_batch *b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_counter) cudaFree(b->d_counter);
  for (fft_plan *p : b->plans) fft_plan_destroy(p);
  delete b;
}

}  // namespace


const char *fft_status_string(fft_status s) {
  switch (s) {
    case FFT_OK: return "ok";
    case FFT_ERR_INVALID_ARG: return "invalid argument";
    case FFT_ERR_INVALID_SIZE: return "invalid size (N must be a power of two in [2, 2^24])";
    case FFT_ERR_UNSUPPORTED: return "unsupported request";
    case FFT_ERR_OOM: return "device out of memory";
    case FFT_ERR_CUDA: return "CUDA error";
    case FFT_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

const char *fft_last_error_string(void) { return g_last_error; }

fft_status fft_plan_opts_init(fft_precision prec, fft_plan_opts *opts) {
  if (!opts) return FFT_ERR_INVALID_ARG;
  if (prec != FFT_PREC_FP32 && prec != FFT_PREC_FP16 && prec != FFT_PREC_BF16) return FFT_ERR_INVALID_ARG;
  memset(opts, 0, sizeof *opts);
  opts->lf_eps = 1e-7;
  opts->scale_forward = prec == FFT_PREC_FP32 ? FFT_SCALE_NONE : FFT_SCALE_HALF_PER_PASS;
  opts->scale_inverse = FFT_SCALE_NONE;
  opts->device = -1;
  return FFT_OK;
}

fft_status fft_plan_create(fft_plan **plan, int64_t n, fft_precision prec, fft_factorization fac,
                           const fft_plan_opts *opts_in) {
  TraceRange trace("dsfft plan_create");
  if (!plan) return FFT_ERR_INVALID_ARG;
  *plan = nullptr;
  if (prec != FFT_PREC_FP32 && prec != FFT_PREC_FP16 && prec != FFT_PREC_BF16) return FFT_ERR_INVALID_ARG;
  if (fac != FFT_FAC_LINZER_FEIG_CLAMPED && fac != FFT_FAC_COSINE && fac != FFT_FAC_DUAL_SELECT)
    return FFT_ERR_INVALID_ARG;
  fft_plan_opts opts;
  fft_plan_opts_init(prec, &opts);
  if (opts_in) {
    opts = *opts_in;
    for (int r : opts.reserved)
      if (r != 0) return FFT_ERR_INVALID_ARG;
  }
  if (opts.autotune != 0 && opts.autotune != 1) return FFT_ERR_INVALID_ARG;
  if (opts.radix != 0 && opts.radix != 2 && opts.radix != 4) return FFT_ERR_INVALID_ARG;
  if (opts.sweep_passes != 0 && (opts.sweep_passes < 7 || opts.sweep_passes > 12)) return FFT_ERR_INVALID_ARG;
  if (opts.variant < FFT_VARIANT_AUTO || opts.variant > FFT_VARIANT_FUSED_TMA) return FFT_ERR_INVALID_ARG;
  if (!(opts.lf_eps > 0.0) || !(opts.lf_eps < 1.0)) return FFT_ERR_INVALID_ARG;
  for (int s : {opts.scale_forward, opts.scale_inverse})
    if (s != FFT_SCALE_NONE && s != FFT_SCALE_HALF_PER_PASS) return FFT_ERR_INVALID_ARG;
  const int log2n = ilog2_exact(n);
  if (log2n < 1 || log2n > kMaxLog2N) return FFT_ERR_INVALID_SIZE;
  const int radix = opts.radix == 4 ? 4 : 2;
  const int r4_variant = log2n <= kFusedMaxLog2N ? FFT_VARIANT_FUSED_WIDE : FFT_VARIANT_SWEEPS;
  if (radix == 4 && opts.variant != FFT_VARIANT_AUTO && opts.variant != r4_variant) {
    snprintf(g_last_error, sizeof g_last_error, "radix-4 plans run the fused radix-4 kernel (N <= 2^%d) or "
             "radix-4 sweeps", kFusedMaxLog2N);
    return FFT_ERR_UNSUPPORTED;
  }
  if (opts.sweep_passes != 0 &&
      (radix == 4 || (opts.variant != FFT_VARIANT_AUTO && opts.variant != FFT_VARIANT_SWEEPS) ||
       !sweep_ls1_valid(log2n, opts.sweep_passes) || log2n <= kFusedMaxLog2N)) {
    snprintf(g_last_error, sizeof g_last_error, "sweep_passes %d does not exist for this plan", opts.sweep_passes);
    return FFT_ERR_UNSUPPORTED;
  }
  if (opts.variant != FFT_VARIANT_AUTO && !variant_valid(prec, log2n, opts.variant)) {
    snprintf(g_last_error, sizeof g_last_error, "variant %d does not exist for N = 2^%d", opts.variant, log2n);
    return FFT_ERR_UNSUPPORTED;
  }

  DeviceGuard guard(opts.device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "select device");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

  fft_plan *p = new fft_plan();
  p->n = n;
  p->log2n = log2n;
  p->prec = prec;
  p->fac = fac;
  p->eps = opts.lf_eps;
  p->scale[0] = opts.scale_forward;
  p->scale[1] = opts.scale_inverse;
  p->device = device;
  p->radix = radix;
  if (const char *f = getenv("DSFFT_FAULT_WAIT")) p->fault_tx = atoi(f) > 0 ? 16u : 0u;

  const size_t entries = (size_t)(n / 2);
  // per-pass tables hold compact 8-byte entries (form 1 FP16/BF16, form 2
  // FP32); the first-stage copies are 16-byte entries (form 0)
  const int compact = (int)prec == kFP32 ? 2 : 1;
  const size_t tw_bytes = sizeof(uint2);
  int *counts = nullptr;
  uint4 *head = nullptr;      // 16-byte forms of the first-stage entries: [dir][radix 2/4][31]
  uint4 *head1 = nullptr;     // FP32 cluster sizes: 16-byte forms of the phase-1 entries: [dir][255]
  cudaStream_t st = nullptr;
  fft_status status = FFT_OK;
  int host_counts[2] = {0, 0};
  do {
    if ((e = device_alloc(&p->table[0], entries * sizeof(uint4))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc table"); break; }
    if ((e = device_alloc(&p->table[1], entries * sizeof(uint4))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc table"); break; }
    if ((e = device_alloc(&p->twp[0], (size_t)(n - 1) * tw_bytes)) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc table"); break; }
    if ((e = device_alloc(&p->twp[1], (size_t)(n - 1) * tw_bytes)) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc table"); break; }
    if ((e = device_alloc(&counts, 2 * sizeof(int))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc counts"); break; }
    if ((e = device_alloc(&head, 4 * 31 * sizeof(uint4))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc"); break; }
    if ((e = device_alloc(&p->status, 16)) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc status"); break; }
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { status = cuda_fail(e, "stream"); break; }
    if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(int), st)) != cudaSuccess) { status = cuda_fail(e, "memset"); break; }
    if ((e = cudaMemsetAsync(p->status, 0, 16, st)) != cudaSuccess) { status = cuda_fail(e, "memset"); break; }
    if ((e = launch_build_table(log2n, n / 2, fac, opts.lf_eps, prec, 0, p->scale[0] ? 0.5 : 1.0, p->table[0], counts, st)) != cudaSuccess) { status = cuda_fail(e, "table build"); break; }
    if ((e = launch_build_table(log2n, n / 2, fac, opts.lf_eps, prec, 1, p->scale[1] ? 0.5 : 1.0, p->table[1], nullptr, st)) != cudaSuccess) { status = cuda_fail(e, "table build"); break; }
    const int64_t cnt0 = (n < 32 ? n : 32) - 1;
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
      if ((e = launch_per_pass_table(log2n, p->table[d], p->twp[d], n - 1, compact, st)) != cudaSuccess) break;
      if ((e = launch_per_pass_table(log2n, p->table[d], head + d * 62, cnt0, 0, st)) != cudaSuccess) break;
      e = cudaMemcpyAsync(p->tw0[d].e, head + d * 62, (size_t)cnt0 * sizeof(uint4), cudaMemcpyDeviceToHost, st);
    }
    if (e != cudaSuccess) { status = cuda_fail(e, "per-pass table"); break; }
    p->has_tw1 = prec == kFP32 && cluster_log2k(prec, log2n) >= 0;
    if (p->has_tw1) {
      if ((e = device_alloc(&head1, 2 * 255 * sizeof(uint4))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc"); break; }
      for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        if ((e = launch_per_pass_table(log2n, p->table[d], head1 + d * 255, 255, 0, st)) != cudaSuccess) break;
        e = cudaMemcpyAsync(p->tw1[d].e, head1 + d * 255, 255 * sizeof(uint4), cudaMemcpyDeviceToHost, st);
      }
      if (e != cudaSuccess) { status = cuda_fail(e, "phase-1 twiddles"); break; }
    }
    if ((e = cudaMemcpyAsync(host_counts, counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) { status = cuda_fail(e, "copy counts"); break; }
    if (radix == 4) {
      const int64_t c4 = 3 * n / 4, p4 = n - 1 - (log2n & 1);
      for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        if ((e = device_alloc(&p->table4[d], (size_t)(c4 > 0 ? c4 : 1) * sizeof(uint4))) != cudaSuccess) break;
        if ((e = device_alloc(&p->twp4[d], (size_t)(p4 > 0 ? p4 : 1) * tw_bytes)) != cudaSuccess) break;
        if ((e = launch_build_table(log2n, c4, fac, opts.lf_eps, prec, d, p->scale[d] ? 0.25 : 1.0, p->table4[d],
                                    nullptr, st)) != cudaSuccess)
          break;
        if ((e = launch_per_pass_table4(log2n, p->table4[d], p->twp4[d], p4, compact, st)) != cudaSuccess) break;
        const int64_t cnt = p4 < 31 ? p4 : 31;
        if ((e = launch_per_pass_table4(log2n, p->table4[d], head + d * 62 + 31, cnt, 0, st)) != cudaSuccess) break;
        memset(&p->s0r4[d], 0, sizeof(Stage0R4));
        if (cnt > 0 && (e = cudaMemcpyAsync(p->s0r4[d].e, head + d * 62 + 31, (size_t)cnt * sizeof(uint4),
                                            cudaMemcpyDeviceToHost, st)) != cudaSuccess)
          break;
      }
      if (e != cudaSuccess) { status = cuda_fail(e, "radix-4 tables"); break; }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { status = cuda_fail(e, "table build sync"); break; }
    for (int d = 0; d < 2; ++d) p->s0r4[d].r2 = p->tw0[d].e[0];
    if (radix == 4) {
      p->variant = r4_variant;
      if (log2n <= kFusedMaxLog2N) {
        p->kernel = 0;
        p->shape = fused4_shape(prec, log2n);
        e = prepare_fused4(prec, log2n);
      } else {
        p->kernel = 1;
        p->shape = fused_shape(prec, kFusedMaxLog2N, false);
        e = prepare_sweeps4(prec, log2n);
      }
      if (e != cudaSuccess) { status = cuda_fail(e, "kernel attributes"); break; }
      break;
    }
    p->sweep_ls1 = opts.sweep_passes ? opts.sweep_passes : default_sweep_ls1(prec, log2n);
    const int v = opts.sweep_passes ? FFT_VARIANT_SWEEPS
                  : opts.variant != FFT_VARIANT_AUTO ? opts.variant : default_variant(prec, log2n);
    if ((e = apply_variant(p, v)) != cudaSuccess) { status = cuda_fail(e, "kernel attributes"); break; }
    if (opts.autotune && opts.variant == FFT_VARIANT_AUTO && !opts.sweep_passes && (e = autotune_plan(p)) != cudaSuccess) { status = cuda_fail(e, "autotune"); break; }
  } while (0);
  if (st) cudaStreamDestroy(st);
  if (counts) cudaFree(counts);
  if (head) cudaFree(head);
  if (head1) cudaFree(head1);
  if (status != FFT_OK) {
    for (int d = 0; d < 2; ++d) {
      if (p->table[d]) cudaFree(p->table[d]);
      if (p->twp[d]) cudaFree(p->twp[d]);
      if (p->table4[d]) cudaFree(p->table4[d]);
      if (p->twp4[d]) cudaFree(p->twp4[d]);
    }
    if (p->status) cudaFree(p->status);
    delete p;
    return status;
  }
  p->cos_count = host_counts[0];
  p->sin_count = host_counts[1];
  *plan = p;
  return FFT_OK;
}

fft_status fft_plan_destroy(fft_plan *plan) {
  if (!plan) return FFT_OK;
  DeviceGuard guard(plan->device);
  for (int d = 0; d < 2; ++d) {
    if (plan->table[d]) cudaFree(plan->table[d]);
    if (plan->twp[d]) cudaFree(plan->twp[d]);
    if (plan->table4[d]) cudaFree(plan->table4[d]);
    if (plan->twp4[d]) cudaFree(plan->twp4[d]);
  }
  if (plan->status) cudaFree(plan->status);
  delete plan;
  return FFT_OK;
}

fft_status fft_exec(const fft_plan *plan, const void *in, void *out, int64_t batch, fft_direction dir,
                    void *stream) {
  if (!plan) return FFT_ERR_INVALID_ARG;
  if (dir != FFT_FORWARD && dir != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
  if (batch < 0) return FFT_ERR_INVALID_ARG;
  if (batch == 0) return FFT_OK;
  if (!in || !out) return FFT_ERR_INVALID_ARG;
  const size_t eb = elem_bytes(plan->prec);
  if (((uintptr_t)in % eb) != 0 || ((uintptr_t)out % eb) != 0) return FFT_ERR_INVALID_ARG;
  const int d = dir == FFT_FORWARD ? 0 : 1;
  if (plan->kernel == 1 && in == out) {
    snprintf(g_last_error, sizeof g_last_error, "in-place transforms are not supported by the HBM-sweep path");
    return FFT_ERR_UNSUPPORTED;
  }
  TraceRange trace("dsfft exec");
  DeviceGuard guard(plan->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "select device");
  cudaError_t e;
  e = plan_launch(plan, in, out, batch, d, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    static const char *what[3] = {"fused kernel launch", "sweep kernel launch", "cluster kernel launch"};
    return cuda_fail(e, what[plan->kernel]);
  }
  return FFT_OK;
}

fft_status fft_plan_device_status(const fft_plan *plan) {
  if (!plan) return FFT_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "select device");
  int word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, plan->status, sizeof word, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word != 0) e = cudaMemset(plan->status, 0, sizeof word);
  if (e != cudaSuccess) return cuda_fail(e, "read device status");
  if (word != 0) {
    snprintf(g_last_error, sizeof g_last_error, "a bounded wait for bulk copies gave up (status word 0x%x)", word);
    return FFT_ERR_TIMEOUT;
  }
  return FFT_OK;
}

fft_status fft_plan_get_table4(const fft_plan *plan, fft_direction dir, void *host_dst, size_t bytes) {
  if (!plan || !host_dst) return FFT_ERR_INVALID_ARG;
  if (dir != FFT_FORWARD && dir != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
  if (plan->radix != 4) return FFT_ERR_UNSUPPORTED;
  const size_t need = (size_t)(3 * plan->n / 4) * sizeof(uint4);
  if (bytes < need) return FFT_ERR_INVALID_ARG;
  if (need == 0) return FFT_OK;
  DeviceGuard guard(plan->device);
  cudaError_t e = cudaMemcpy(host_dst, plan->table4[dir == FFT_FORWARD ? 0 : 1], need, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "copy table");
  return FFT_OK;
}

fft_status fft_plan_get_table(const fft_plan *plan, fft_direction dir, void *host_dst, size_t bytes) {
  if (!plan || !host_dst) return FFT_ERR_INVALID_ARG;
  if (dir != FFT_FORWARD && dir != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
  const size_t need = (size_t)(plan->n / 2) * sizeof(uint4);
  if (bytes < need) return FFT_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  cudaError_t e = cudaMemcpy(host_dst, plan->table[dir == FFT_FORWARD ? 0 : 1], need, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "copy table");
  return FFT_OK;
}

fft_status fft_plan_get_info(const fft_plan *plan, fft_plan_info *info) {
  if (!plan || !info) return FFT_ERR_INVALID_ARG;
  memset(info, 0, sizeof *info);
  info->n = plan->n;
  info->log2n = plan->log2n;
  info->precision = plan->prec;
  info->factorization = plan->fac;
  info->kernel = plan->kernel;
  info->launches = plan->kernel == 1 ? 2 : 1;
  info->points_per_thread = 1 << plan->shape.log2r;
  info->threads_per_transform = plan->shape.threads_per_transform;
  info->transforms_per_block = plan->shape.transforms_per_block;
  const int64_t twb = (int64_t)sizeof(uint2);   // compact per-pass entries
  info->table_bytes = (int64_t)2 * (plan->n / 2 * (int64_t)sizeof(uint4) + (plan->n - 1) * twb);
  if (plan->radix == 4) info->table_bytes += (int64_t)2 * (3 * plan->n / 4 * (int64_t)sizeof(uint4) + plan->n * twb);
  info->element_bytes = (int64_t)elem_bytes(plan->prec);
  info->scale_forward = plan->scale[0];
  info->scale_inverse = plan->scale[1];
  info->cos_count = plan->cos_count;
  info->sin_count = plan->sin_count;
  info->variant = plan->variant;
  info->autotuned = plan->autotuned;
  info->radix = plan->radix;
  info->sweep_passes = 0;
  if (plan->kernel == 1) {
    int l1, l2;
    if (plan->radix == 4) sweep_split4(plan->log2n, &l1, &l2);
    else sweep_split(plan->log2n, &l1, &l2);
    info->sweep_passes = plan->sweep_ls1 ? plan->sweep_ls1 : l1;
  }
  return FFT_OK;
}

fft_status fft_twiddle_fp64(int64_t n, fft_factorization fac, double lf_eps, double *host_t, double *host_m,
                            int32_t *host_path) {
  if (!host_t || !host_m || !host_path) return FFT_ERR_INVALID_ARG;
  if (fac != FFT_FAC_LINZER_FEIG_CLAMPED && fac != FFT_FAC_COSINE && fac != FFT_FAC_DUAL_SELECT)
    return FFT_ERR_INVALID_ARG;
  if (!(lf_eps > 0.0) || !(lf_eps < 1.0)) return FFT_ERR_INVALID_ARG;
  const int log2n = ilog2_exact(n);
  if (log2n < 1 || log2n > kMaxLog2N) return FFT_ERR_INVALID_SIZE;
  const size_t h = (size_t)(n / 2);
  double *t = nullptr, *m = nullptr;
  int *path = nullptr;
  fft_status status = FFT_OK;
  cudaError_t e;
  do {
    if ((e = device_alloc(&t, h * sizeof(double))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc"); break; }
    if ((e = device_alloc(&m, h * sizeof(double))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc"); break; }
    if ((e = device_alloc(&path, h * sizeof(int))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc"); break; }
    if ((e = launch_fp64_table(log2n, fac, lf_eps, t, m, path, nullptr)) != cudaSuccess) { status = cuda_fail(e, "fp64 table"); break; }
    if ((e = cudaMemcpy(host_t, t, h * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) { status = cuda_fail(e, "copy"); break; }
    if ((e = cudaMemcpy(host_m, m, h * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) { status = cuda_fail(e, "copy"); break; }
    if ((e = cudaMemcpy(host_path, path, h * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) { status = cuda_fail(e, "copy"); break; }
  } while (0);
  if (t) cudaFree(t);
  if (m) cudaFree(m);
  if (path) cudaFree(path);
  return status;
}

fft_status fft_batch_create(fft_batch **batch, const fft_batch_item *items, int64_t count,
                            const fft_plan_opts *opts) {
  if (!batch) return FFT_ERR_INVALID_ARG;
  *batch = nullptr;
  if (count < 0 || (count > 0 && !items)) return FFT_ERR_INVALID_ARG;
  if (count > 0x7FFFFFFFLL) return FFT_ERR_INVALID_SIZE;
  // validate every item before touching the device
  for (int64_t i = 0; i < count; ++i) {
    const fft_batch_item &it = items[i];
    if (it.precision < FFT_PREC_FP32 || it.precision > FFT_PREC_BF16) return FFT_ERR_INVALID_ARG;
    if (it.factorization < FFT_FAC_LINZER_FEIG_CLAMPED || it.factorization > FFT_FAC_DUAL_SELECT)
      return FFT_ERR_INVALID_ARG;
    if (it.direction != FFT_FORWARD && it.direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if (it.reserved != 0 || !it.in || !it.out) return FFT_ERR_INVALID_ARG;
    const size_t eb = elem_bytes(it.precision);
    if (((uintptr_t)it.in % eb) != 0 || ((uintptr_t)it.out % eb) != 0) return FFT_ERR_INVALID_ARG;
    const int l = ilog2_exact(it.n);
    if (l < 1 || l > kMaxLog2N) return FFT_ERR_INVALID_SIZE;
  }
  fft_batch *b = new fft_batch();
  b->count = count;
  fft_status status = FFT_OK;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaGetDevice");
  }
  // one plan per (n, precision, factorization)
  std::map<std::tuple<int64_t, int, int>, fft_plan *> plan_of;
  struct Ref {
    fft_plan *plan;
    int dir;
    int64_t index;
  };
  std::vector<Ref> refs;
  refs.reserve((size_t)count);
  for (int64_t i = 0; i < count && status == FFT_OK; ++i) {
    const fft_batch_item &it = items[i];
    auto key = std::make_tuple(it.n, (int)it.precision, (int)it.factorization);
    auto f = plan_of.find(key);
    fft_plan *p = nullptr;
    if (f == plan_of.end()) {
      fft_plan_opts o;
      fft_plan_opts_init((fft_precision)it.precision, &o);
      if (opts) o = *opts;
      status = fft_plan_create(&p, it.n, (fft_precision)it.precision, (fft_factorization)it.factorization, &o);
      if (status != FFT_OK) break;
      plan_of[key] = p;
      b->plans.push_back(p);
    } else {
      p = f->second;
    }
    if (p->kernel == 1 && it.in == it.out) status = FFT_ERR_UNSUPPORTED;
    refs.push_back(Ref{p, it.direction == FFT_FORWARD ? 0 : 1, i});
  }
  if (status != FFT_OK) {
    batch_release(b);
    return status;
  }
  // order: persistent-kernel groups (largest N first), then the large groups
  std::stable_sort(refs.begin(), refs.end(), [](const Ref &a, const Ref &c) {
    const bool la = a.plan->kernel != 0, lc = c.plan->kernel != 0;
    if (la != lc) return la < lc;
    if (a.plan->log2n != c.plan->log2n) return a.plan->log2n > c.plan->log2n;
    if (a.plan != c.plan) return a.plan < c.plan;
    return a.dir < c.dir;
  });
  std::vector<BatchItem> h_items((size_t)count);
  std::vector<BatchTile> h_tiles;
  for (int64_t i = 0; i < count; ++i) h_items[(size_t)i] = BatchItem{items[refs[(size_t)i].index].in, items[refs[(size_t)i].index].out};
  for (int64_t i = 0; i < count;) {
    const Ref &r = refs[(size_t)i];
    int64_t j = i;
    while (j < count && refs[(size_t)j].plan == r.plan && refs[(size_t)j].dir == r.dir) ++j;
    if (r.plan->kernel == 0) {
      const int cap = batch_tile_capacity(r.plan->prec, r.plan->log2n);
      for (int64_t k = i; k < j; k += cap) {
        BatchTile t{};
        t.path = batch_path_code(r.plan->prec, r.plan->log2n, r.plan->scale[r.dir] != 0);
        t.count = (uint32_t)std::min<int64_t>(cap, j - k);
        t.first = (uint32_t)k;
        t.twp = r.plan->twp[r.dir];
        h_tiles.push_back(t);
      }
    } else {
      b->large.push_back(fft_batch::Large{r.plan, r.dir, i, j - i});
    }
    i = j;
  }
  b->ntiles = (int)h_tiles.size();
  do {
    if (count > 0) {
      if ((e = device_alloc(&b->d_items, sizeof(BatchItem) * (size_t)count)) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc items"); break; }
      if ((e = cudaMemcpy(b->d_items, h_items.data(), sizeof(BatchItem) * (size_t)count, cudaMemcpyHostToDevice)) != cudaSuccess) { status = cuda_fail(e, "copy items"); break; }
      b->device_bytes += (int64_t)(sizeof(BatchItem) * (size_t)count);
    }
    if (b->ntiles > 0) {
      if ((e = device_alloc(&b->d_tiles, sizeof(BatchTile) * h_tiles.size())) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc tiles"); break; }
      if ((e = cudaMemcpy(b->d_tiles, h_tiles.data(), sizeof(BatchTile) * h_tiles.size(), cudaMemcpyHostToDevice)) != cudaSuccess) { status = cuda_fail(e, "copy tiles"); break; }
      if ((e = device_alloc(&b->d_counter, sizeof(unsigned))) != cudaSuccess) { status = cuda_fail(e, "cudaMalloc counter"); break; }
      if ((e = prepare_batch_kernel(&b->grid)) != cudaSuccess) { status = cuda_fail(e, "batch kernel attributes"); break; }
      b->device_bytes += (int64_t)(sizeof(BatchTile) * h_tiles.size() + sizeof(unsigned));
    }
    // up to four internal streams for the large groups
    const size_t nside = std::min<size_t>(b->large.size(), 4);
    if (nside > 0) {
      if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) { status = cuda_fail(e, "event"); break; }
      for (size_t i = 0; i < nside && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) break;
        b->side.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
        b->join.push_back(ev);
      }
      if (e != cudaSuccess) { status = cuda_fail(e, "internal streams"); break; }
    }
  } while (0);
  if (status != FFT_OK) {
    batch_release(b);
    return status;
  }
  for (fft_plan *p : b->plans) b->device_bytes += (int64_t)2 * (p->n / 2 + p->n - 1) * (int64_t)sizeof(uint4);
  *batch = b;
  return FFT_OK;
}

fft_status fft_batch_exec(fft_batch *batch, void *stream) {
  TraceRange trace("dsfft batch_exec");
  if (!batch) return FFT_ERR_INVALID_ARG;
  DeviceGuard guard(batch->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "select device");
  cudaError_t e = batch_enqueue(batch, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return FFT_OK;
}

fft_status fft_batch_exec_graph(fft_batch *batch, void *stream) {
  TraceRange trace("dsfft batch_exec_graph");
  if (!batch) return FFT_ERR_INVALID_ARG;
  DeviceGuard guard(batch->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "select device");
  cudaError_t e;
  if (!batch->graph_exec) {
    if (!batch->capture_stream &&
        (e = cudaStreamCreateWithFlags(&batch->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "capture stream");
    if ((e = cudaStreamBeginCapture(batch->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "begin capture");
    cudaError_t le = batch_enqueue(batch, batch->capture_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(batch->capture_stream, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le, "batch launch during capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    if ((e = cudaGraphInstantiate(&batch->graph_exec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "graph instantiate");
    }
    batch->graph = g;
  }
  if ((e = cudaGraphLaunch(batch->graph_exec, (cudaStream_t)stream)) != cudaSuccess)
    return cuda_fail(e, "graph launch");
  return FFT_OK;
}

fft_status fft_batch_get_info(const fft_batch *batch, fft_batch_info *info) {
  if (!batch || !info) return FFT_ERR_INVALID_ARG;
  memset(info, 0, sizeof *info);
  info->items = batch->count;
  info->plans = (int32_t)batch->plans.size();
  info->tiles = batch->ntiles;
  info->persistent_blocks = batch->ntiles > 0 ? std::min(batch->grid, batch->ntiles) : 0;
  info->large_groups = (int32_t)batch->large.size();
  int launches = batch->ntiles > 0 ? 1 : 0;
  for (const auto &g : batch->large) launches += g.plan->kernel == 1 ? 2 : 1;
  info->launches = launches;
  info->graph_ready = batch->graph_exec != nullptr;
  info->device_bytes = batch->device_bytes;
  return FFT_OK;
}

fft_status fft_batch_destroy(fft_batch *batch) {
  batch_release(batch);
  return FFT_OK;
}

}  // extern "C"
