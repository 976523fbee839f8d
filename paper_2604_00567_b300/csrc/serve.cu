// serve.cu — the serving loop: continuous batching of FFT requests under a
// device-memory budget (fft_server_* in include/dsfft.h).
//
// Threads: callers submit/poll/wait/release under the server mutex; one
// scheduler thread owns every launch.  Its loop:
//   1. admission: pop the FIFO head while its output fits in the arena
//      (first-fit allocator over one cudaMalloc'd block);
//   2. launch: when a tick slot is free and requests are admitted, take them
//      (up to max_tick_transforms small transforms) as one tick: the N <= 2^14
//      transforms go to one persistent batch-kernel launch (descriptors
//      staged through the slot's pinned buffer), each larger request to its
//      plan's own launch, all on the slot's stream, then an event;
//   3. completion: ticks whose event has completed (checked in launch order)
//      mark their requests done and wake waiters;
//   4. sleep on the condition variable (a submission or release wakes it;
//      20 us while ticks are on the GPU).
// Every transform runs the butterflies of fft_exec on its own input and
// output, so its result does not depend on what it was batched with.
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/dsfft.h"
#include "internal.h"

using namespace dsfft;

namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

int ilog2_pow2(int64_t n) {
  if (n < 2 || (n & (n - 1)) != 0) return -1;
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

constexpr uint64_t kAlign = 256;

// First-fit allocator over [0, size): free blocks by offset, merged on free.
class Arena {
 public:
  void init(uint64_t size) {
    size_ = size;
    free_.clear();
    free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(uint64_t bytes, uint64_t *off) {
    const uint64_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      *off = it->first;
      const uint64_t rest = it->second - need;
      const uint64_t start = it->first + need;
      free_.erase(it);
      if (rest) free_[start] = rest;
      used_ += need;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    const uint64_t len = (bytes + kAlign - 1) / kAlign * kAlign;
    used_ -= len;
    auto next = free_.lower_bound(off);
    uint64_t start = off, end = off + len;
    if (next != free_.end() && next->first == end) {
      end += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        free_.erase(prev);
      }
    }
    free_[start] = end - start;
  }
  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }

 private:
  uint64_t size_ = 0, used_ = 0, peak_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

enum State { kQueued, kAdmitted, kLaunched, kDone, kReleased };

struct Request {
  fft_request req;
  const fft_plan *plan = nullptr;
  PlanView view;
  uint64_t ticket = 0;
  int64_t bytes = 0;
  uint64_t arena_off = 0;
  State state = kQueued;
  bool delivered = false;     // returned by poll or wait
  fft_completion c;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  BatchItem *d_items = nullptr, *h_items = nullptr;
  BatchTile *d_tiles = nullptr, *h_tiles = nullptr;
  unsigned *d_counter = nullptr;
  bool busy = false;
  int64_t tick = 0;
  std::vector<Request *> reqs;
};

}  // namespace

struct fft_server {
  fft_server_opts opts;
  int device = 0;
  int grid = 0;
  unsigned char *arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  std::deque<int> slot_order;       // busy slots in launch order

  std::mutex mu;                    // guards everything below
  std::condition_variable cv_sched;   // wakes the scheduler
  std::condition_variable cv_done;    // wakes waiters
  std::map<std::tuple<int64_t, int, int>, fft_plan *> plans;
  std::mutex plan_mu;               // plan creation (outside mu)
  std::unordered_map<uint64_t, Request *> by_ticket;
  std::deque<Request *> queued;     // FIFO awaiting admission
  std::deque<Request *> admitted;   // awaiting launch
  int64_t admitted_bytes = 0;       // output bytes of `admitted`
  std::deque<uint64_t> done_order;  // tickets done, in completion order (poll's queue)
  uint64_t next_ticket = 1;
  int64_t submitted = 0, n_admitted = 0, completed = 0, released = 0, ticks = 0, transforms = 0;
  int64_t in_flight = 0;
  bool stop = false;
  std::thread thread;
};

namespace {

fft_status fail(fft_status s, const char *msg) {
  set_last_error(msg);
  return s;
}

fft_status cuda_fail(cudaError_t e, const char *where) {
  char buf[200];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  set_last_error(buf);
  return e == cudaErrorMemoryAllocation ? FFT_ERR_OOM : FFT_ERR_CUDA;
}

// Resident plan of (n, prec, fac), created on first use.
fft_status get_plan(fft_server *s, int64_t n, int prec, int fac, const fft_plan **out) {
  std::lock_guard<std::mutex> g(s->plan_mu);
  const auto key = std::make_tuple(n, prec, fac);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) {
      *out = it->second;
      return FFT_OK;
    }
  }
  fft_plan_opts po;
  fft_plan_opts_init((fft_precision)prec, &po);
  po.device = s->device;
  po.autotune = s->opts.autotune;
  fft_plan *p = nullptr;
  fft_status st = fft_plan_create(&p, n, (fft_precision)prec, (fft_factorization)fac, &po);
  if (st != FFT_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  s->plans[key] = p;
  *out = p;
  return FFT_OK;
}

// Admission (caller holds mu): FIFO, the head must fit.
void admit(fft_server *s) {
  while (!s->queued.empty()) {
    Request *r = s->queued.front();
    uint64_t off = 0;
    if (!s->arena.alloc((uint64_t)r->bytes, &off)) break;
    r->arena_off = off;
    r->c.out = s->arena_base + off;
    r->c.t_admit_ns = now_ns();
    r->state = kAdmitted;
    s->queued.pop_front();
    s->admitted.push_back(r);
    s->admitted_bytes += r->bytes;
    ++s->n_admitted;
  }
}

void finish(fft_server *s, Request *r, fft_status st, int64_t t) {
  r->c.status = st;
  r->c.t_done_ns = t;
  r->state = kDone;
  s->done_order.push_back(r->ticket);
  ++s->completed;
  --s->in_flight;
  if (st == FFT_OK) s->transforms += r->req.count;
  if (s->opts.release_on_complete) {
    s->arena.release(r->arena_off, (uint64_t)r->bytes);
    r->state = kReleased;
    ++s->released;
  }
}

bool small_request(const Request *r) { return r->view.kernel == 0; }

// Queue one tick on slot `sl` (no lock held; the requests are owned by the
// tick).  Returns the first CUDA error.
cudaError_t launch_tick(fft_server *s, Slot &sl) {
  TraceRange trace("dsfft server tick");
  // small transforms, grouped by (plan, direction), larger sizes first
  std::vector<Request *> small;
  for (Request *r : sl.reqs)
    if (small_request(r)) small.push_back(r);
  std::stable_sort(small.begin(), small.end(), [](const Request *a, const Request *b) {
    if (a->view.log2n != b->view.log2n) return a->view.log2n > b->view.log2n;
    if (a->plan != b->plan) return a->plan < b->plan;
    return a->req.direction < b->req.direction;
  });
  int64_t nitems = 0;
  int ntiles = 0;
  for (size_t i = 0; i < small.size();) {
    size_t j = i;
    while (j < small.size() && small[j]->plan == small[i]->plan && small[j]->req.direction == small[i]->req.direction)
      ++j;
    const PlanView &v = small[i]->view;
    const int d = small[i]->req.direction == FFT_FORWARD ? 0 : 1;
    const int64_t first = nitems;
    const size_t eb = v.prec == kFP32 ? 8 : 4;
    const int64_t n = int64_t(1) << v.log2n;
    for (size_t k = i; k < j; ++k) {
      const Request *r = small[k];
      const unsigned char *in = static_cast<const unsigned char *>(r->req.in);
      unsigned char *out = static_cast<unsigned char *>(r->c.out);
      for (int64_t t = 0; t < r->req.count; ++t)
        sl.h_items[nitems++] = BatchItem{in + t * n * eb, out + t * n * eb};
    }
    const int cap = batch_tile_capacity(v.prec, v.log2n);
    for (int64_t t = first; t < nitems; t += cap) {
      BatchTile tile;
      memset(&tile, 0, sizeof tile);
      tile.path = batch_path_code(v.prec, v.log2n, v.scale[d] != 0);
      tile.count = (uint32_t)std::min<int64_t>(cap, nitems - t);
      tile.first = (uint32_t)t;
      tile.twp = v.twp[d];
      sl.h_tiles[ntiles++] = tile;
    }
    i = j;
  }
  cudaError_t e = cudaSuccess;
  if (ntiles > 0) {
    if ((e = cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(BatchItem) * (size_t)nitems, cudaMemcpyHostToDevice,
                             sl.stream)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(sl.d_tiles, sl.h_tiles, sizeof(BatchTile) * (size_t)ntiles, cudaMemcpyHostToDevice,
                             sl.stream)) != cudaSuccess)
      return e;
    if ((e = launch_batch_kernel(sl.d_tiles, ntiles, sl.d_items, sl.d_counter, s->grid, sl.stream)) != cudaSuccess)
      return e;
  }
  for (Request *r : sl.reqs) {
    if (small_request(r)) continue;
    const fft_status st = fft_exec(r->plan, r->req.in, r->c.out, r->req.count, (fft_direction)r->req.direction,
                                   sl.stream);
    if (st != FFT_OK) return cudaErrorLaunchFailure;
  }
  return cudaEventRecord(sl.event, sl.stream);
}

void scheduler(fft_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    admit(s);
    // launch a tick into a free slot
    int free_slot = -1;
    for (int i = 0; i < (int)s->slots.size(); ++i)
      if (!s->slots[i].busy) {
        free_slot = i;
        break;
      }
    if (free_slot >= 0 && !s->admitted.empty()) {
      Slot &sl = s->slots[free_slot];
      sl.reqs.clear();
      int64_t small_count = 0, tick_bytes = 0;
      // tick size: the admitted backlog spread over the tick slots, between
      // an eighth of max_tick_bytes and max_tick_bytes (when that limit is
      // set): a short queue gives small ticks that finish soon, a backlog
      // full-size ticks that amortise each tick's launches
      int64_t cap = s->opts.max_tick_bytes;
      if (cap > 0) {
        const int64_t share = s->admitted_bytes / (int64_t)s->slots.size();
        cap = std::min(cap, std::max(cap / 8, share));
      }
      while (!s->admitted.empty()) {
        Request *r = s->admitted.front();
        if (small_request(r) && small_count + r->req.count > s->opts.max_tick_transforms) break;
        if (cap > 0 && !sl.reqs.empty() && tick_bytes + r->bytes > cap) break;
        tick_bytes += r->bytes;
        if (small_request(r)) small_count += r->req.count;
        s->admitted.pop_front();
        s->admitted_bytes -= r->bytes;
        r->state = kLaunched;
        sl.reqs.push_back(r);
      }
      sl.busy = true;
      sl.tick = ++s->ticks;
      s->slot_order.push_back(free_slot);
      const int64_t t = now_ns();
      for (Request *r : sl.reqs) {
        r->c.t_launch_ns = t;
        r->c.tick = sl.tick;
      }
      lk.unlock();
      const cudaError_t e = launch_tick(s, sl);
      lk.lock();
      if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "server tick launch: %s", cudaGetErrorString(e));
        set_last_error(buf);
        cudaStreamSynchronize(sl.stream);
        const int64_t tn = now_ns();
        for (Request *r : sl.reqs) finish(s, r, FFT_ERR_CUDA, tn);
        sl.busy = false;
        s->slot_order.pop_back();
        s->cv_done.notify_all();
      }
      continue;   // admit / launch more before sleeping
    }
    // completions, in launch order
    bool progressed = false;
    while (!s->slot_order.empty()) {
      Slot &sl = s->slots[s->slot_order.front()];
      const cudaError_t q = cudaEventQuery(sl.event);
      if (q == cudaErrorNotReady) break;
      const fft_status st = q == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
      const int64_t t = now_ns();
      for (Request *r : sl.reqs) finish(s, r, st, t);
      sl.reqs.clear();
      sl.busy = false;
      s->slot_order.pop_front();
      progressed = true;
    }
    if (progressed) {
      s->cv_done.notify_all();
      continue;
    }
    if (s->stop && s->queued.empty() && s->admitted.empty() && s->slot_order.empty()) break;
    if (!s->slot_order.empty())
      s->cv_sched.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
  }
}

Request *find_ticket(fft_server *s, uint64_t ticket) {
  auto it = s->by_ticket.find(ticket);
  return it == s->by_ticket.end() ? nullptr : it->second;
}

// The completion has been handed to the caller (caller holds mu): a record
// that is both delivered and released is dropped.
void deliver(fft_server *s, Request *r) {
  r->delivered = true;
  if (r->state == kReleased) {
    s->by_ticket.erase(r->ticket);
    delete r;
  }
}

void free_slot_buffers(Slot &sl) {
  if (sl.event) cudaEventDestroy(sl.event);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  if (sl.d_items) cudaFree(sl.d_items);
  if (sl.d_tiles) cudaFree(sl.d_tiles);
  if (sl.d_counter) cudaFree(sl.d_counter);
  if (sl.h_items) cudaFreeHost(sl.h_items);
  if (sl.h_tiles) cudaFreeHost(sl.h_tiles);
  sl = Slot();
}

void free_server(fft_server *s) {
  for (Slot &sl : s->slots) free_slot_buffers(sl);
  for (auto &kv : s->plans) fft_plan_destroy(kv.second);
  for (auto &kv : s->by_ticket) delete kv.second;
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
}

}  // namespace

extern "C" {

fft_status fft_server_opts_init(fft_server_opts *opts) {
  if (!opts) return FFT_ERR_INVALID_ARG;
  memset(opts, 0, sizeof *opts);
  opts->device = -1;
  opts->max_ticks_in_flight = 2;
  opts->memory_budget = 40000000000ULL;
  opts->max_tick_transforms = int64_t(1) << 20;
  return FFT_OK;
}

fft_status fft_server_create(fft_server **server, const fft_server_opts *opts_in) {
  if (!server) return FFT_ERR_INVALID_ARG;
  *server = nullptr;
  fft_server_opts o;
  fft_server_opts_init(&o);
  if (opts_in) o = *opts_in;
  for (int r : o.reserved)
    if (r != 0) return FFT_ERR_INVALID_ARG;
  if (o.max_ticks_in_flight < 1 || o.max_ticks_in_flight > 8) return FFT_ERR_INVALID_ARG;
  if (o.memory_budget < kAlign || o.max_tick_transforms < 1 || o.max_tick_transforms > (int64_t(1) << 26))
    return FFT_ERR_INVALID_ARG;
  if ((o.autotune != 0 && o.autotune != 1) || (o.release_on_complete != 0 && o.release_on_complete != 1))
    return FFT_ERR_INVALID_ARG;
  if (o.max_tick_bytes < 0) return FFT_ERR_INVALID_ARG;

  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const int device = o.device >= 0 ? o.device : prev;
  if (device != prev && (e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  struct Restore {
    int prev, device;
    ~Restore() {
      if (prev != device) cudaSetDevice(prev);
    }
  } restore{prev, device};

  fft_server *s = new fft_server();
  s->opts = o;
  s->device = device;
  fft_status st = FFT_OK;
  do {
    if ((e = prepare_batch_kernel(&s->grid)) != cudaSuccess) { st = cuda_fail(e, "batch kernel attributes"); break; }
    if ((e = device_alloc(&s->arena_base, o.memory_budget)) != cudaSuccess) { st = cuda_fail(e, "arena"); break; }
    s->arena.init(o.memory_budget);
    s->slots.resize((size_t)o.max_ticks_in_flight);
    const size_t ni = (size_t)o.max_tick_transforms;
    for (Slot &sl : s->slots) {
      if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess) break;
      if ((e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming)) != cudaSuccess) break;
      if ((e = device_alloc(&sl.d_items, ni * sizeof(BatchItem))) != cudaSuccess) break;
      if ((e = device_alloc(&sl.d_tiles, ni * sizeof(BatchTile))) != cudaSuccess) break;
      if ((e = device_alloc(&sl.d_counter, sizeof(unsigned))) != cudaSuccess) break;
      if ((e = cudaHostAlloc(&sl.h_items, ni * sizeof(BatchItem), cudaHostAllocDefault)) != cudaSuccess) break;
      if ((e = cudaHostAlloc(&sl.h_tiles, ni * sizeof(BatchTile), cudaHostAllocDefault)) != cudaSuccess) break;
    }
    if (e != cudaSuccess) { st = cuda_fail(e, "tick slot buffers"); break; }
  } while (0);
  if (st != FFT_OK) {
    free_server(s);
    return st;
  }
  s->thread = std::thread(scheduler, s);
  *server = s;
  return FFT_OK;
}

fft_status fft_server_prepare(fft_server *server, int64_t n, fft_precision precision,
                              fft_factorization factorization) {
  if (!server) return FFT_ERR_INVALID_ARG;
  const fft_plan *p = nullptr;
  return get_plan(server, n, precision, factorization, &p);
}

fft_status fft_server_submit(fft_server *s, const fft_request *req, uint64_t *ticket) {
  if (!s || !req) return FFT_ERR_INVALID_ARG;
  if (req->reserved != 0 || req->count < 1 || !req->in) return FFT_ERR_INVALID_ARG;
  if (req->direction != FFT_FORWARD && req->direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
  if (req->precision != FFT_PREC_FP32 && req->precision != FFT_PREC_FP16 && req->precision != FFT_PREC_BF16)
    return FFT_ERR_INVALID_ARG;
  if (req->factorization != FFT_FAC_LINZER_FEIG_CLAMPED && req->factorization != FFT_FAC_COSINE &&
      req->factorization != FFT_FAC_DUAL_SELECT)
    return FFT_ERR_INVALID_ARG;
  const int log2n = ilog2_pow2(req->n);
  if (log2n < 1 || log2n > kMaxLog2N) return FFT_ERR_INVALID_SIZE;
  const int64_t eb = req->precision == FFT_PREC_FP32 ? 8 : 4;
  if ((uintptr_t)req->in % (uintptr_t)eb != 0) return FFT_ERR_INVALID_ARG;
  if (req->count > (int64_t(1) << 40) / req->n) return FFT_ERR_INVALID_SIZE;
  const int64_t bytes = req->count * req->n * eb;
  if ((uint64_t)bytes > s->arena.size()) return fail(FFT_ERR_OOM, "fft_server_submit: output larger than the arena");
  if (log2n <= kFusedMaxLog2N && req->count > s->opts.max_tick_transforms)
    return fail(FFT_ERR_INVALID_SIZE, "fft_server_submit: more signals than max_tick_transforms");

  const fft_plan *plan = nullptr;
  fft_status st = get_plan(s, req->n, req->precision, req->factorization, &plan);
  if (st != FFT_OK) return st;
  Request *r = new Request();
  r->req = *req;
  r->plan = plan;
  plan_view(plan, &r->view);
  r->bytes = bytes;
  memset(&r->c, 0, sizeof r->c);
  r->c.tag = req->tag;
  r->c.bytes = bytes;
  r->c.t_submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->c.ticket = r->ticket;
    s->by_ticket[r->ticket] = r;
    s->queued.push_back(r);
    ++s->submitted;
    ++s->in_flight;
  }
  s->cv_sched.notify_one();
  if (ticket) *ticket = r->ticket;
  return FFT_OK;
}

fft_status fft_server_replay(fft_server *s, const fft_request *reqs, const int64_t *arrival_ns, int64_t count,
                             uint64_t *tickets) {
  if (!s || count < 0 || (count > 0 && (!reqs || !arrival_ns))) return FFT_ERR_INVALID_ARG;
  const int64_t t0 = now_ns();
  for (int64_t i = 0; i < count; ++i) {
    const int64_t due = t0 + arrival_ns[i];
    int64_t t;
    while ((t = now_ns()) < due) {
      if (due - t > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(due - t - 100000));
    }
    uint64_t tk = 0;
    const fft_status st = fft_server_submit(s, &reqs[i], &tk);
    if (st != FFT_OK) return st;
    if (tickets) tickets[i] = tk;
  }
  return FFT_OK;
}

fft_status fft_server_poll(fft_server *s, fft_completion *out, int64_t max, int64_t *got) {
  if (!s || !got || max < 0 || (max > 0 && !out)) return FFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t k = 0;
  while (k < max && !s->done_order.empty()) {
    const uint64_t t = s->done_order.front();
    s->done_order.pop_front();
    Request *r = find_ticket(s, t);
    if (!r || r->delivered) continue;
    out[k++] = r->c;
    deliver(s, r);
  }
  *got = k;
  return FFT_OK;
}

fft_status fft_server_wait(fft_server *s, uint64_t ticket, double timeout_s, fft_completion *out) {
  if (!s || timeout_s < 0) return FFT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  Request *r = find_ticket(s, ticket);
  if (!r) return FFT_ERR_INVALID_ARG;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state != kDone && r->state != kReleased) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != kDone &&
        r->state != kReleased)
      return FFT_ERR_TIMEOUT;
  }
  if (out) *out = r->c;
  deliver(s, r);
  return FFT_OK;
}

fft_status fft_server_copy_out(fft_server *s, uint64_t ticket, void *dst, int64_t bytes, void *stream) {
  if (!s || !dst || bytes < 0) return FFT_ERR_INVALID_ARG;
  void *src = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Request *r = find_ticket(s, ticket);
    if (!r || r->state != kDone || bytes > r->bytes) return FFT_ERR_INVALID_ARG;
    src = r->c.out;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  const cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, (cudaStream_t)stream);
  if (prev != s->device) cudaSetDevice(prev);
  return e == cudaSuccess ? FFT_OK : cuda_fail(e, "fft_server_copy_out");
}

fft_status fft_server_release(fft_server *s, uint64_t ticket) {
  if (!s) return FFT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Request *r = find_ticket(s, ticket);
    if (!r || r->state != kDone) return FFT_ERR_INVALID_ARG;
    s->arena.release(r->arena_off, (uint64_t)r->bytes);
    r->state = kReleased;
    ++s->released;
    if (r->delivered) {
      s->by_ticket.erase(ticket);
      delete r;
    }
  }
  s->cv_sched.notify_one();
  return FFT_OK;
}

fft_status fft_server_drain(fft_server *s, double timeout_s) {
  if (!s || timeout_s < 0) return FFT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (s->in_flight > 0) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->in_flight > 0) return FFT_ERR_TIMEOUT;
  }
  return FFT_OK;
}

fft_status fft_server_get_stats(fft_server *s, fft_server_stats *st) {
  if (!s || !st) return FFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof *st);
  st->submitted = s->submitted;
  st->admitted = s->n_admitted;
  st->completed = s->completed;
  st->released = s->released;
  st->queued = (int64_t)s->queued.size();
  st->in_flight = s->in_flight;
  st->ticks = s->ticks;
  st->transforms = s->transforms;
  st->plans = (int64_t)s->plans.size();
  st->arena_bytes = s->arena.size();
  st->arena_used = s->arena.used();
  st->arena_peak = s->arena.peak();
  return FFT_OK;
}

fft_status fft_server_destroy(fft_server *s) {
  if (!s) return FFT_OK;
  fft_server_drain(s, 60.0);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests that never got admitted are dropped
    for (Request *r : s->queued) {
      --s->in_flight;
      r->state = kReleased;
    }
    s->queued.clear();
  }
  s->cv_sched.notify_all();
  if (s->thread.joinable()) s->thread.join();
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  for (Slot &sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  const int dev = s->device;
  free_server(s);
  if (prev != dev) cudaSetDevice(prev);
  return FFT_OK;
}

}  // extern "C"
