// CUDA-graph orchestration of the kernel-split variant: the currents and
// amplitudes launches of every chunk are captured once, on two internal
// streams, into one graph:
//   currents(c) -> amplitudes(c)            (the records of chunk c)
//   amplitudes(c) -> currents(c + 2)        (the two chunk buffers alternate)
// so currents(c + 1) may run beside amplitudes(c).  The instantiated graph is
// kept with its key (every launch argument) and replayed on the caller's
// stream while the key matches; one cached graph, guarded by a mutex.
#include <cstring>
#include <mutex>
#include <vector>

#include "launch.h"

namespace mg {

namespace {

struct SplitGraphCache {
  std::mutex mu;
  std::vector<char> key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t s0 = nullptr, sa = nullptr, sb = nullptr;
  cudaEvent_t fork = nullptr, eva = nullptr, evb[2] = {nullptr, nullptr};
};

SplitGraphCache& cache() {
  static SplitGraphCache c;
  return c;
}

cudaError_t make_streams(SplitGraphCache& c) {
  if (c.s0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&c.s0, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithFlags(&c.sa, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithFlags(&c.sb, cudaStreamNonBlocking)) != cudaSuccess) return e;
  for (cudaEvent_t* ev : {&c.fork, &c.eva, &c.evb[0], &c.evb[1]})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaSuccess;
}

// the launches of one batch into the capture begun on c.s0
cudaError_t record_batch(SplitGraphCache& c, int64_t nevt, int64_t chunk, void* buf0, void* buf1,
                         const SplitOps& ops) {
  cudaError_t e;
  if ((e = cudaEventRecord(c.fork, c.s0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c.sa, c.fork, 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c.sb, c.fork, 0)) != cudaSuccess) return e;
  const int64_t nchunk = (nevt + chunk - 1) / chunk;
  for (int64_t k = 0; k < nchunk; ++k) {
    const int64_t first = k * chunk, last = first + chunk < nevt ? first + chunk : nevt;
    void* buf = (k & 1) ? buf1 : buf0;
    if (k >= 2 && (e = cudaStreamWaitEvent(c.sa, c.evb[k & 1], 0)) != cudaSuccess) return e;
    if ((e = ops.currents(first, last, buf, c.sa)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c.eva, c.sa)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.sb, c.eva, 0)) != cudaSuccess) return e;
    if ((e = ops.amplitudes(first, last, buf, c.sb)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c.evb[k & 1], c.sb)) != cudaSuccess) return e;
  }
  // join both streams back into the capturing stream
  if ((e = cudaEventRecord(c.eva, c.sa)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c.s0, c.eva, 0)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c.evb[0], c.sb)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(c.s0, c.evb[0], 0);
}

}  // namespace

cudaError_t run_split_graph(const void* key, size_t key_bytes, int64_t nevt, int64_t chunk, void* buf0, void* buf1,
                            const SplitOps& ops, cudaStream_t s) {
  SplitGraphCache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  const bool hit = c.exec && c.key.size() == key_bytes && std::memcmp(c.key.data(), key, key_bytes) == 0;
  if (!hit) {
    cudaError_t e;
    if (c.exec) {
      cudaGraphExecDestroy(c.exec);
      c.exec = nullptr;
      c.key.clear();
    }
    if ((e = make_streams(c)) != cudaSuccess) return e;
    if ((e = ops.prepare()) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(c.s0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t rec = record_batch(c, nevt, chunk, buf0, buf1, ops);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c.s0, &graph);
    if (rec != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();  // the launch error is reported through the return value
      return rec != cudaSuccess ? rec : e;
    }
    e = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c.exec = nullptr;
      return e;
    }
    c.key.assign(static_cast<const char*>(key), static_cast<const char*>(key) + key_bytes);
  }
  return cudaGraphLaunch(c.exec, s);
}

}  // namespace mg
