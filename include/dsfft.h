/*
 * dsfft.h — C ABI of the dual-select FMA radix-2 FFT library (libdsfft.so).
 *
 * The library computes batched complex DFTs (Eq. 1: A = a + W b, B = a - W b,
 * W = exp(-j 2 pi k/N)) with an m = log2 N pass radix-2 Stockham FFT
 * (Section IV) whose butterflies are 6-FMA forms driven by a precomputed
 * twiddle table (Sections II-III):
 *   - dual-select (Algorithm 1): per twiddle, the cosine-outer form
 *     (ratio tan theta, multiplier cos theta) when |cos| >= |sin|, else the
 *     sine-outer form (ratio cot theta, multiplier sin theta); |ratio| <= 1
 *     (Theorem 1), no clamp;
 *   - linzer_feig_clamped (Eqs. 4-6): sine-outer everywhere, sin clamped to
 *     -eps where |sin| < eps (the clamp practice of Section I);
 *   - cosine (Eqs. 7-9): cosine-outer everywhere.
 * Only the table differs between the three; the kernels are identical.
 * Tables are computed in FP64 on the GPU and rounded once to the plan's
 * precision.  All arithmetic of a transform runs in that precision (FP32
 * FFMA, or packed FP16/BF16 HFMA2 on the CUDA cores).
 *
 * Data layout (all precisions): a batch of `batch` transforms, transform b
 * at element offset b*N, each element an interleaved (re, im) pair:
 *   FFT_PREC_FP32: 8 bytes  (float re, float im)      — "complex64"
 *   FFT_PREC_FP16: 4 bytes  (half re,  half im)        — "complex-FP16"
 *   FFT_PREC_BF16: 4 bytes  (bf16 re,  bf16 im)
 * Output is in natural frequency order.  Pointers passed to fft_exec are
 * device pointers (cudaMalloc or equivalent) aligned to the element size.
 *
 * Ownership: a plan owns its device tables; the caller owns `in`, `out` and
 * the stream.  A plan is immutable after creation and may be used from
 * several host threads and streams concurrently.
 *
 * Errors: every call returns an fft_status.  Argument and plan errors are
 * returned synchronously and leave no work queued.  Launch failures return
 * FFT_ERR_CUDA (the CUDA error string is available from
 * fft_last_error_string on the calling thread).  Device-side bounded waits
 * that give up are reported through fft_plan_device_status.
 *
 * Fault injection for tests (environment, read when the call is made):
 *   DSFFT_FAULT_ALLOC=k   the k-th device allocation of the library fails
 *                         (FFT_ERR_OOM), counting from when the value is set;
 *   DSFFT_FAULT_WAIT=1    plans created while it is set arm their kernels'
 *                         bounded waits with 16 bytes that never arrive, so
 *                         each such wait runs out (about one second) and the
 *                         plan's device status word records it.
 */
#ifndef DSFFT_H
#define DSFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported entry points; everything else in the library is hidden. */
#if defined(__GNUC__)
#define DSFFT_API __attribute__((visibility("default")))
#else
#define DSFFT_API
#endif

typedef enum fft_status {
    FFT_OK = 0,
    FFT_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, negative batch */
    FFT_ERR_INVALID_SIZE = 2,  /* N not a power of two or outside [2, 2^24] */
    FFT_ERR_UNSUPPORTED = 3,   /* valid request the library does not implement */
    FFT_ERR_OOM = 4,           /* device allocation failed */
    FFT_ERR_CUDA = 5,          /* a CUDA runtime call or launch failed */
    FFT_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} fft_status;

typedef enum fft_precision {
    FFT_PREC_FP32 = 0,
    FFT_PREC_FP16 = 1,
    FFT_PREC_BF16 = 2
} fft_precision;

typedef enum fft_factorization {
    FFT_FAC_LINZER_FEIG_CLAMPED = 0,   /* Eqs. 4-6 with the eps clamp */
    FFT_FAC_COSINE = 1,                /* Eqs. 7-9 */
    FFT_FAC_DUAL_SELECT = 2            /* Algorithm 1 */
} fft_factorization;

typedef enum fft_direction {
    FFT_FORWARD = -1,   /* W = exp(-j 2 pi k/N) (Eq. 1) */
    FFT_INVERSE = 1     /* conjugate twiddles; unnormalised unless scaled */
} fft_direction;

typedef enum fft_scaling {
    FFT_SCALE_NONE = 0,
    /* exact x0.5 per pass: a' = RN(a/2), multiplier stored as RN(m/2), so the
     * output is DFT/N.  Keeps FP16 data in range. */
    FFT_SCALE_HALF_PER_PASS = 1
} fft_scaling;

/* Kernel variants a plan can run (all bit-identical; they differ in speed). */
typedef enum fft_variant {
    FFT_VARIANT_AUTO = 0,          /* built-in choice, or the autotuner's */
    FFT_VARIANT_FUSED_WIDE = 1,    /* N <= 2^14: 32 (FP16/BF16) / 16 (FP32) points per thread */
    FFT_VARIANT_FUSED_NARROW = 2,  /* N <= 2^14: half the points per thread (where
                                      that keeps a transform within 1024 threads) */
    FFT_VARIANT_CLUSTER = 3,       /* 2^15 <= N <= 2^17 (FP16/BF16), <= 2^16 (FP32):
                                      one launch on a thread-block cluster */
    FFT_VARIANT_SWEEPS = 4,        /* N >= 2^15: two HBM sweeps */
    FFT_VARIANT_FUSED_TMA = 5      /* 2^8 <= N <= 2^14 (FP32: 2^13): the wide fused kernel as a
                                      persistent grid whose input tiles arrive by
                                      double-buffered bulk asynchronous copies
                                      (TMA); inputs not 16-byte aligned run the
                                      wide kernel */
} fft_variant;

typedef struct fft_plan_opts {
    double lf_eps;          /* clamp for FFT_FAC_LINZER_FEIG_CLAMPED (default 1e-7) */
    int32_t scale_forward;  /* fft_scaling of forward transforms */
    int32_t scale_inverse;  /* fft_scaling of inverse transforms */
    int32_t device;         /* CUDA device ordinal; -1 = current device */
    /* 1: when `variant` is AUTO, time every candidate variant for this
     * (precision, N) — for the sweeps also the split of the passes between
     * the two sweeps, within one pass of the balanced split — on the plan's
     * GPU at creation (about 128 MiB of scratch buffers, freed before
     * returning) and keep the fastest; the choice is
     * cached per GPU model in the JSON file named by the environment variable
     * DSFFT_AUTOTUNE_CACHE, if set, and reused by later plans. 0: built-in
     * choice. */
    int32_t autotune;
    int32_t variant;        /* fft_variant; a variant the size does not have
                               gives FFT_ERR_UNSUPPORTED */
    /* 0 or 2: radix-2 passes (the paper's algorithm).  4: radix-4 passes
     * (the radix-4 extension the paper's Discussion proposes; the fused
     * kernel for N <= 2^14, two HBM sweeps of radix-4 passes above; other
     * variants give FFT_ERR_UNSUPPORTED): each radix-4 pass
     * (span L) maps Z[q N/4 + s L + j], q = 0..3, to
     * Y[4 s L + p L + j] = sum_q W_4L^(q j) Z[...] (-i)^(q p) (+i inverse);
     * each of its three twiddle products uses the 6-FMA form of its own
     * dual-select entry, then four sums; one radix-2 pass (span 1) first when
     * log2 N is odd.  Scaled directions divide by 4 per radix-4 pass.  The
     * results differ from the radix-2 algorithm's in rounding only. */
    int32_t radix;
    /* N > 2^14, radix 2: passes in the first of the two HBM sweeps (the
     * second runs the rest; both must hold 7..12 passes).  0 = the balanced
     * split ceil(log2 N / 2), or the autotuner's choice with autotune = 1.
     * Nonzero selects the sweeps variant (FFT_ERR_UNSUPPORTED with another
     * variant, radix 4 or N <= 2^14; FFT_ERR_INVALID_ARG outside 7..12). */
    int32_t sweep_passes;
    int32_t reserved[1];    /* must be zero */
} fft_plan_opts;

typedef struct fft_plan_info {
    int64_t n;                  /* transform length N */
    int32_t log2n;
    int32_t precision;          /* fft_precision */
    int32_t factorization;      /* fft_factorization */
    int32_t kernel;             /* 0 = fused on-chip transform (N <= 2^14),
                                   1 = two HBM sweeps, 2 = one launch on a
                                   thread-block cluster (DSMEM) */
    int32_t launches;           /* kernel launches per fft_exec */
    int32_t points_per_thread;  /* register block of the fused kernel */
    int32_t threads_per_transform;
    int32_t transforms_per_block;
    int64_t table_bytes;        /* device bytes of the tables (both directions) */
    int64_t element_bytes;      /* 8 (FP32) or 4 (FP16/BF16) */
    int32_t scale_forward;
    int32_t scale_inverse;
    int32_t cos_count;          /* table entries on the cosine path */
    int32_t sin_count;          /* table entries on the sine path */
    int32_t variant;            /* fft_variant the plan runs */
    int32_t autotuned;          /* 1 = chosen by timing, 2 = from the cache */
    int32_t radix;              /* 2 or 4 */
    int32_t sweep_passes;       /* passes in sweep 1 when the plan runs sweeps, else 0 */
} fft_plan_info;

typedef struct fft_plan fft_plan;

/* Fill `opts` with the defaults for `prec`: lf_eps = 1e-7, device = -1,
 * scale_forward = HALF_PER_PASS for FP16/BF16 and NONE for FP32,
 * scale_inverse = NONE. */
DSFFT_API fft_status fft_plan_opts_init(fft_precision prec, fft_plan_opts *opts);

/* Create a plan for length-N transforms (N = 2^m, 2 <= N <= 2^24).  Builds
 * the FP64 twiddle table of Algorithm 1 (or of Eqs. 4-6 / 7-9) on the GPU
 * for k in [0, N/2), rounds ratio and multiplier once to `prec`, and keeps
 * the packed tables for both directions resident on the device.  Blocks
 * until the tables are built.  `opts` may be NULL (defaults).
 * On success *plan owns the device memory; release with fft_plan_destroy. */
DSFFT_API fft_status fft_plan_create(fft_plan **plan, int64_t n, fft_precision prec,
                           fft_factorization fac, const fft_plan_opts *opts);

/* Release a plan (NULL is accepted).  Work already queued that uses the plan
 * must have completed. */
DSFFT_API fft_status fft_plan_destroy(fft_plan *plan);

/* Transform `batch` signals (layout above) from `in` to `out`, asynchronously
 * on `stream` (a cudaStream_t; NULL = legacy default stream).  `in` is never
 * modified unless in == out.  in == out (in-place) is supported except by
 * the HBM-sweep kernel (fft_plan_info.kernel == 1: FP16/BF16 N >= 2^18,
 * FP32 N >= 2^17), which returns FFT_ERR_UNSUPPORTED for it; partially
 * overlapping buffers are not allowed.  batch == 0 is a no-op.  Device
 * pointers, element-aligned. */
DSFFT_API fft_status fft_exec(const fft_plan *plan, const void *in, void *out, int64_t batch,
                    fft_direction dir, void *stream);

/* Copy the plan's packed device table for `dir` to host memory
 * (N/2 entries of 16 bytes; `bytes` must be at least 8*N).  Entry k:
 *   FP32 : word0 = ratio t (float), word1 = multiplier m (float),
 *          word2 = sigma*m (float), word3 = path (0 cosine, 1 sine)
 *   FP16/BF16: word0 = (lo: -t, hi: t), word1 = (lo: sigma*m, hi: m),
 *          word2 = byte-permute selector of the operand swap (0x1032 on
 *          the cosine path, 0x3210 on the sine path),
 *          word3 = (lo: -sigma*m, hi: -m)
 * where sigma = +1 on the cosine path and -1 on the sine path and m already
 * carries the x0.5 of a scaled direction.  Synchronous. */
DSFFT_API fft_status fft_plan_get_table(const fft_plan *plan, fft_direction dir, void *host_dst,
                              size_t bytes);

/* Radix-4 plans: copy the packed radix-4 table of `dir` (3N/4 entries of
 * 16 bytes, k in [0, 3N/4): W^k by the rules above, multipliers divided by 4
 * on a scaled direction; same entry layout as fft_plan_get_table) to host
 * memory.  FFT_ERR_UNSUPPORTED for a radix-2 plan. */
DSFFT_API fft_status fft_plan_get_table4(const fft_plan *plan, fft_direction dir, void *host_dst, size_t bytes);

/* Read and clear the plan's device error word.  Kernels whose waits are
 * bounded set it when such a wait gives up (about one second): the
 * FFT_VARIANT_FUSED_TMA kernel waiting for a bulk copy (bit 0), the
 * FP16/BF16 cluster kernel waiting for its phase-1 data (bit 1); the
 * affected blocks skip their remaining work, so the output is incomplete.
 * Returns FFT_ERR_TIMEOUT if it was set since the last call, else FFT_OK.
 * Synchronous: waits for all work queued on the plan's device first. */
DSFFT_API fft_status fft_plan_device_status(const fft_plan *plan);

/* Describe the plan (kernel choice, launch shape, table sizes). */
DSFFT_API fft_status fft_plan_get_info(const fft_plan *plan, fft_plan_info *info);

/* Run the FP64 stage of the table builder on the current device and return
 * the unrounded entries for k in [0, N/2): ratio t, multiplier m (forward
 * direction, no scaling) and path (0 cosine, 1 sine), into host arrays of
 * N/2 elements each.  Synchronous.  Used to check the GPU's FP64
 * trigonometry against a host evaluation. */
DSFFT_API fft_status fft_twiddle_fp64(int64_t n, fft_factorization fac, double lf_eps,
                            double *host_t, double *host_m, int32_t *host_path);

/* ------------------------------------------------------------------------ */
/* Mixed batches: transforms of different sizes, precisions, factorizations
 * and directions, each with its own input and output buffer, run as one
 * persistent kernel launch (every transform with N <= 2^14) plus one launch
 * per (size, precision, factorization, direction) group of larger transforms
 * (cluster or sweep kernels reading the same per-transform pointers).  The
 * persistent kernel takes tiles of equal-size transforms, largest first,
 * from a device work counter.  Each transform's result is bit-identical to
 * fft_exec of the same plan on that transform alone. */

typedef struct fft_batch_item {
    int64_t n;                /* transform length, as for fft_plan_create */
    int32_t precision;        /* fft_precision */
    int32_t factorization;    /* fft_factorization */
    int32_t direction;        /* fft_direction */
    int32_t reserved;         /* must be zero */
    const void *in;           /* device pointer, element-aligned */
    void *out;                /* device pointer; may equal `in` except for
                                 sizes that use HBM sweeps */
} fft_batch_item;

typedef struct fft_batch fft_batch;

typedef struct fft_batch_info {
    int64_t items;             /* transforms in the batch */
    int32_t plans;             /* distinct plans the batch created */
    int32_t tiles;             /* work tiles of the persistent kernel */
    int32_t persistent_blocks; /* blocks of the persistent launch */
    int32_t large_groups;      /* groups of N > 2^14 launched separately */
    int32_t launches;          /* kernel launches per fft_batch_exec */
    int32_t graph_ready;       /* 1 once fft_batch_exec_graph captured */
    int64_t device_bytes;      /* device memory the batch owns (tables,
                                  descriptors, work counter) */
} fft_batch_info;

/* Build a batch from `count` items (copied; the buffers they point to are
 * the caller's and must stay valid while the batch is used).  Plans are
 * created once per distinct (n, precision, factorization); `opts` applies to
 * every plan (NULL = the defaults of each item's precision).  Uploads the
 * work descriptors; blocks until done. */
DSFFT_API fft_status fft_batch_create(fft_batch **batch, const fft_batch_item *items, int64_t count,
                                      const fft_plan_opts *opts);

/* Run every transform of the batch asynchronously on `stream`.  The
 * persistent launch runs on `stream`; the groups of larger transforms run on
 * up to four streams the batch owns, forked from `stream` and joined back to
 * it by events (so they overlap one another and the persistent launch's
 * tail); work queued on `stream` after the call waits for all of them.  A
 * batch must not run concurrently with itself (its work counter and internal
 * streams are shared by its calls). */
DSFFT_API fft_status fft_batch_exec(fft_batch *batch, void *stream);

/* Same work as fft_batch_exec, through a CUDA graph: the first call captures
 * the launches (on a stream the batch owns) and instantiates the graph,
 * every call launches the graph on `stream`.  Not thread-safe with itself on
 * the same batch. */
DSFFT_API fft_status fft_batch_exec_graph(fft_batch *batch, void *stream);

DSFFT_API fft_status fft_batch_get_info(const fft_batch *batch, fft_batch_info *info);

/* Release the batch, its plans and its graph (NULL accepted); queued work
 * using it must have completed. */
DSFFT_API fft_status fft_batch_destroy(fft_batch *batch);

/* ------------------------------------------------------------------------ */
/* A mixed batch that allocates no device memory.  This entry point has no
 * counterpart in the paper; it exists for callers that cannot call cudaMalloc
 * where they transform — a host program that owns all device memory through
 * its own fixed pool, or a latency-bound loop where cudaMalloc/cudaFree would
 * stall on their implicit synchronisation.  It runs the same kernels as
 * fft_batch_exec, with the work descriptors and work counter in one fixed
 * device array of the library (about 192 KB, present in every GPU that loads
 * the library until exit) instead of memory the batch allocates.
 *   - `items`: `count` <= FFT_NOALLOC_MAX_ITEMS transforms, each with a plan
 *     created beforehand (fft_plan_create allocates; do that first), a
 *     direction (FFT_FORWARD / FFT_INVERSE), `reserved` = 0 and device
 *     input/output pointers aligned to the element size.  Refused: more
 *     items (FFT_ERR_INVALID_SIZE); a bad direction, a nonzero reserved
 *     field, a null or misaligned pointer, plans on different devices
 *     (FFT_ERR_INVALID_ARG); in == out for a plan on the HBM-sweep path and
 *     radix-4 plans (FFT_ERR_UNSUPPORTED).  A refused call launches nothing;
 *     count = 0 returns FFT_OK without launching.
 *   - Asynchronous on `stream`: the descriptors reach the device array as
 *     the parameters of small copy kernels, so the call does not wait for
 *     earlier work on `stream` and reads no host memory after it returns.
 *   - The first call on a device (and the first after that device's context
 *     is replaced, e.g. by cudaDeviceReset) also looks up the device address
 *     of the array and sets the kernel's attributes; make that first call
 *     before any stream capture.
 *   - Every call reuses the same array (the work counter is cleared at the
 *     start of each call); calls whose work overlaps on the GPU, e.g. on two
 *     streams, race on it — order them on one stream. */
#define FFT_NOALLOC_MAX_ITEMS 4096

typedef struct fft_noalloc_item {
    const fft_plan *plan;
    int32_t direction;        /* fft_direction */
    int32_t reserved;         /* must be zero */
    const void *in;
    void *out;
} fft_noalloc_item;

DSFFT_API fft_status fft_exec_batch_noalloc(const fft_noalloc_item *items, int64_t count, void *stream);

/* ---- Host-memory batches ------------------------------------------------------
 * Not in the paper: a transfer pipeline for batches that live in host
 * memory.  The batch is cut into chunks of `chunk_transforms` signals; chunk
 * c is copied host -> device, transformed by the plan and copied back on
 * internal stream c mod `depth`, so the two copy directions and the kernels
 * of different chunks overlap.  The pipeline owns depth x 2 device staging
 * buffers of one chunk each (allocated at creation) and references the plan,
 * which must outlive it.  Host buffers: batch * N elements in the plan's
 * layout; page-locked (cudaHostAlloc / cudaHostRegister) memory lets the
 * copies run asynchronously, pageable memory works but serialises.
 * host_in == host_out is allowed.  Calls on one pipeline must not overlap on
 * the GPU (they share the staging buffers): order them on one stream. */
typedef struct fft_pipeline fft_pipeline;

/* depth in [1, 8]; FFT_ERR_OOM when the staging buffers do not fit. */
DSFFT_API fft_status fft_pipeline_create(fft_pipeline **pipe, const fft_plan *plan, int64_t chunk_transforms,
                                         int32_t depth);
/* Asynchronous: the chunks start after work already queued on `stream`,
 * and later work on `stream` waits for the last copy back. */
DSFFT_API fft_status fft_pipeline_exec(fft_pipeline *pipe, const void *host_in, void *host_out, int64_t batch,
                                       fft_direction dir, void *stream);
/* Waits for the pipeline's streams, then frees it (NULL is accepted). */
DSFFT_API fft_status fft_pipeline_destroy(fft_pipeline *pipe);

/* ---- Serving loop with continuous batching --------------------------------
 * The paper has no serving layer: this is a front end that keeps requests of
 * mixed size, precision and direction flowing through the same kernels
 * (every transform is bit-identical to fft_exec of its request alone).
 *
 * A server owns one device arena of `memory_budget` bytes (allocated once at
 * create), its resident plans (created on first use of a size, or by
 * fft_server_prepare) and a scheduler thread.  Life of a request:
 *   submit  -> queued (FIFO);
 *   admitted when its output (count * n elements) fits in the arena: the
 *            output slot is taken; a later request never overtakes an
 *            earlier one that does not fit yet;
 *   launched in the next "tick": all admitted requests are launched together
 *            (one persistent launch for every N <= 2^14 transform of the
 *            tick, one launch per larger request) on one of the server's
 *            streams, as soon as one of `max_ticks_in_flight` slots is free,
 *            so arrivals join the GPU's queue while earlier ticks run;
 *   done     when the tick's event has completed (steady-clock timestamps of
 *            every step are kept);
 *   released by fft_server_release (or at completion with
 *            release_on_complete), which frees the arena slot.
 * Inputs stay in the caller's device memory and must remain valid and
 * unmodified until the request is done. */
typedef struct fft_server fft_server;

typedef struct fft_server_opts {
    int32_t device;               /* -1: the current device */
    int32_t max_ticks_in_flight;  /* 1..8 (default 2) */
    uint64_t memory_budget;       /* arena bytes (default 40e9) */
    int64_t max_tick_transforms;  /* N <= 2^14 transforms per tick (default 2^20) */
    int32_t autotune;             /* plans created with autotune (0/1) */
    int32_t release_on_complete;  /* free the output slot at completion: the
                                     output pointer is then not usable (0/1) */
    int64_t max_tick_bytes;       /* output bytes per tick at most (the first
                                     request of a tick is always taken); 0 =
                                     no limit (default).  Smaller ticks finish
                                     sooner, which shortens the wait of the
                                     requests that arrive while they run.
                                     When set, a tick takes the admitted
                                     backlog's share per tick slot, between
                                     an eighth of this limit and the limit:
                                     small ticks while the queue is short,
                                     full ones under a backlog. */
    int32_t reserved[2];          /* must be zero */
} fft_server_opts;

typedef struct fft_request {
    int64_t n;                    /* power of two in [2, 2^24] */
    int32_t precision;            /* fft_precision */
    int32_t factorization;        /* fft_factorization */
    int32_t direction;            /* fft_direction */
    int32_t reserved;             /* must be zero */
    int64_t count;                /* signals, >= 1 */
    const void *in;               /* device, count * n elements (fft_exec layout) */
    uint64_t tag;                 /* returned with the completion */
} fft_request;

typedef struct fft_completion {
    uint64_t ticket;
    uint64_t tag;
    int32_t status;               /* fft_status of the request */
    int32_t reserved;
    void *out;                    /* device, in the arena; valid until released */
    int64_t bytes;                /* count * n * element bytes */
    int64_t t_submit_ns;          /* steady clock (CLOCK_MONOTONIC), ns */
    int64_t t_admit_ns;
    int64_t t_launch_ns;
    int64_t t_done_ns;            /* when the scheduler saw the tick complete */
    int64_t tick;
} fft_completion;

typedef struct fft_server_stats {
    int64_t submitted, admitted, completed, released;
    int64_t queued;               /* waiting for admission */
    int64_t in_flight;            /* admitted, not yet done */
    int64_t ticks;
    int64_t transforms;           /* completed transforms */
    int64_t plans;                /* resident plans */
    uint64_t arena_bytes, arena_used, arena_peak;
    int64_t reserved[4];
} fft_server_stats;

/* Defaults (see the field comments). */
DSFFT_API fft_status fft_server_opts_init(fft_server_opts *opts);
/* Allocates the arena and per-slot descriptor buffers, starts the scheduler
 * thread.  FFT_ERR_OOM when the arena cannot be allocated. */
DSFFT_API fft_status fft_server_create(fft_server **server, const fft_server_opts *opts);
/* Creates (if needed) the resident plan of (n, precision, factorization). */
DSFFT_API fft_status fft_server_prepare(fft_server *server, int64_t n, fft_precision precision,
                                        fft_factorization factorization);
/* Queues a request (thread-safe; never waits for the GPU).  FFT_ERR_OOM when
 * its output alone exceeds the arena; FFT_ERR_INVALID_SIZE for a bad n or an
 * N <= 2^14 request of more than max_tick_transforms signals. */
DSFFT_API fft_status fft_server_submit(fft_server *server, const fft_request *req, uint64_t *ticket);
/* Submits reqs[i] at start + arrival_ns[i] (open-loop replay of an arrival
 * trace from the calling thread, which it blocks until the last submission);
 * tickets[i] receives the ticket (may be null). */
DSFFT_API fft_status fft_server_replay(fft_server *server, const fft_request *reqs, const int64_t *arrival_ns,
                                       int64_t count, uint64_t *tickets);
/* Copies up to `max` completions not yet returned (in completion order). */
DSFFT_API fft_status fft_server_poll(fft_server *server, fft_completion *out, int64_t max, int64_t *got);
/* Waits for one ticket; FFT_ERR_TIMEOUT after timeout_s seconds. */
DSFFT_API fft_status fft_server_wait(fft_server *server, uint64_t ticket, double timeout_s, fft_completion *out);
/* Copies a done, unreleased request's output to `dst` (device or host) on
 * `stream` (asynchronous). */
DSFFT_API fft_status fft_server_copy_out(fft_server *server, uint64_t ticket, void *dst, int64_t bytes, void *stream);
/* Frees a done request's arena slot (FFT_ERR_INVALID_ARG if not done). */
DSFFT_API fft_status fft_server_release(fft_server *server, uint64_t ticket);
/* Waits until every submitted request is done; FFT_ERR_TIMEOUT otherwise
 * (for example when unreleased outputs keep the queue from being admitted). */
DSFFT_API fft_status fft_server_drain(fft_server *server, double timeout_s);
DSFFT_API fft_status fft_server_get_stats(fft_server *server, fft_server_stats *stats);
/* Drains (up to 60 s), stops the thread and frees everything. */
DSFFT_API fft_status fft_server_destroy(fft_server *server);

/* Static description of a status code. */
DSFFT_API const char *fft_status_string(fft_status status);

/* Text of the last CUDA error seen by a library call on this host thread
 * ("" if none). */
DSFFT_API const char *fft_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* DSFFT_H */
