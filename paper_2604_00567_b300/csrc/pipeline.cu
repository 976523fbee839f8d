// pipeline.cu — transforms of host-memory batches (fft_pipeline_* in
// include/dsfft.h): the batch is cut into chunks of whole transforms; chunk
// c goes host -> device, through the plan's kernels and back on internal
// stream c mod depth, so the host-to-device copy of one chunk, the kernels of
// the next and the device-to-host copy of a third run at the same time (two
// copy directions and the SMs are separate engines).  The staging buffers
// are allocated once, at creation.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/dsfft.h"
#include "internal.h"

using namespace dsfft;

struct fft_pipeline {
  const fft_plan *plan = nullptr;
  PlanView view;
  int64_t chunk = 0;          // transforms per chunk
  size_t chunk_bytes = 0;
  size_t transform_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<void *> din, dout;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
};

namespace {

fft_status pipe_fail(cudaError_t e, const char *where) {
  char buf[200];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  set_last_error(buf);
  return e == cudaErrorMemoryAllocation ? FFT_ERR_OOM : FFT_ERR_CUDA;
}

struct DeviceScope {
  int prev = -1;
  bool switched = false;
  explicit DeviceScope(int device) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != device && cudaSetDevice(device) == cudaSuccess)
      switched = true;
  }
  ~DeviceScope() {
    if (switched) cudaSetDevice(prev);
  }
};

void release(fft_pipeline *p) {
  for (cudaStream_t s : p->streams)
    if (s) cudaStreamSynchronize(s);
  for (void *b : p->din)
    if (b) cudaFree(b);
  for (void *b : p->dout)
    if (b) cudaFree(b);
  for (cudaEvent_t ev : p->done)
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t s : p->streams)
    if (s) cudaStreamDestroy(s);
  if (p->start) cudaEventDestroy(p->start);
  delete p;
}

}  // namespace

extern "C" {

fft_status fft_pipeline_create(fft_pipeline **pipe, const fft_plan *plan, int64_t chunk_transforms, int32_t depth) {
  if (!pipe || !plan) return FFT_ERR_INVALID_ARG;
  *pipe = nullptr;
  if (chunk_transforms < 1 || depth < 1 || depth > 8) return FFT_ERR_INVALID_ARG;
  PlanView v;
  if (!plan_view(plan, &v)) return FFT_ERR_INVALID_ARG;
  const size_t eb = v.prec == kFP32 ? 8 : 4;
  const size_t tb = eb << v.log2n;
  if ((size_t)chunk_transforms > ((size_t)1 << 40) / tb) return FFT_ERR_INVALID_SIZE;
  DeviceScope scope(v.device);
  fft_pipeline *p = new fft_pipeline();
  p->plan = plan;
  p->view = v;
  p->chunk = chunk_transforms;
  p->transform_bytes = tb;
  p->chunk_bytes = tb * (size_t)chunk_transforms;
  p->streams.assign((size_t)depth, nullptr);
  p->din.assign((size_t)depth, nullptr);
  p->dout.assign((size_t)depth, nullptr);
  p->done.assign((size_t)depth, nullptr);
  cudaError_t e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  for (int i = 0; i < depth && e == cudaSuccess; ++i) {
    if ((e = cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming)) != cudaSuccess) break;
    if ((e = device_alloc(&p->din[i], p->chunk_bytes)) != cudaSuccess) break;
    e = device_alloc(&p->dout[i], p->chunk_bytes);
  }
  if (e != cudaSuccess) {
    release(p);
    return pipe_fail(e, "fft_pipeline_create");
  }
  *pipe = p;
  return FFT_OK;
}

fft_status fft_pipeline_exec(fft_pipeline *p, const void *host_in, void *host_out, int64_t batch,
                             fft_direction dir, void *stream) {
  if (!p || batch < 0) return FFT_ERR_INVALID_ARG;
  if (dir != FFT_FORWARD && dir != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
  if (batch == 0) return FFT_OK;
  if (!host_in || !host_out) return FFT_ERR_INVALID_ARG;
  TraceRange trace("dsfft pipeline_exec");
  DeviceScope scope(p->view.device);
  cudaStream_t user = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(p->start, user);
  if (e != cudaSuccess) return pipe_fail(e, "fft_pipeline_exec");
  const int depth = (int)p->streams.size();
  for (int i = 0; i < depth; ++i)
    if ((e = cudaStreamWaitEvent(p->streams[i], p->start, 0)) != cudaSuccess) return pipe_fail(e, "fft_pipeline_exec");
  const unsigned char *src = static_cast<const unsigned char *>(host_in);
  unsigned char *dst = static_cast<unsigned char *>(host_out);
  int64_t c = 0;
  for (int64_t first = 0; first < batch; first += p->chunk, ++c) {
    const int s = (int)(c % depth);
    const int64_t cnt = batch - first < p->chunk ? batch - first : p->chunk;
    const size_t off = (size_t)first * p->transform_bytes, bytes = (size_t)cnt * p->transform_bytes;
    if ((e = cudaMemcpyAsync(p->din[s], src + off, bytes, cudaMemcpyHostToDevice, p->streams[s])) != cudaSuccess)
      return pipe_fail(e, "host-to-device copy");
    const fft_status st = fft_exec(p->plan, p->din[s], p->dout[s], cnt, dir, p->streams[s]);
    if (st != FFT_OK) return st;
    if ((e = cudaMemcpyAsync(dst + off, p->dout[s], bytes, cudaMemcpyDeviceToHost, p->streams[s])) != cudaSuccess)
      return pipe_fail(e, "device-to-host copy");
  }
  for (int i = 0; i < depth; ++i) {
    if ((e = cudaEventRecord(p->done[i], p->streams[i])) != cudaSuccess) return pipe_fail(e, "fft_pipeline_exec");
    if ((e = cudaStreamWaitEvent(user, p->done[i], 0)) != cudaSuccess) return pipe_fail(e, "fft_pipeline_exec");
  }
  return FFT_OK;
}

fft_status fft_pipeline_destroy(fft_pipeline *p) {
  if (!p) return FFT_OK;
  DeviceScope scope(p->view.device);
  release(p);
  return FFT_OK;
}

}  // extern "C"
