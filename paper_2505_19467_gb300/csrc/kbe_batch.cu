// Batched systems: many independent Kadanoff-Baym systems of uneven size
// advanced together on one GPU.
//
// Every admitted system is an ordinary handle on its own stream, forked from
// the caller's stream with an event and joined back after each call, so the
// kernels of different systems overlap on the GPU (a small system's launches
// fill SMs that a large system's tail leaves idle). Steps are enqueued one
// time step of all systems at a time, so no system runs far ahead of the
// others; with graphs on (kbe_batch_set_graphs) each system instead replays
// the call's steps as one captured graph on its own stream. Admission is by
// device memory: systems are taken in order while their allocation fits the
// budget; the others are reported as not admitted.
#include <cstdio>
#include <string>
#include <vector>

#include "kbe_internal.cuh"

struct kbe_batch {
  cudaStream_t main = nullptr;
  std::vector<kbe_handle *> sys;    // nullptr for systems not admitted
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<int> nt_max;
  std::vector<int> cur;             // host copy of each system's current row
  cudaEvent_t fork = nullptr;
  bool graphs = false;              // each system replays its captured steps (kbe_set_graphs)
};

namespace {

kbe_status batch_fail(kbe_status s, const std::string &msg) {
  kbe::set_last_error(msg);
  return s;
}

void destroy_all(kbe_batch *b) {
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (b->sys[i]) kbe_destroy(b->sys[i]);
    if (b->streams[i]) cudaStreamDestroy(b->streams[i]);
    if (b->done[i]) cudaEventDestroy(b->done[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
}

// streams of the admitted systems wait for the caller's prior work
cudaError_t fork_from_main(kbe_batch *b) {
  cudaError_t e = cudaEventRecord(b->fork, b->main);
  for (size_t i = 0; e == cudaSuccess && i < b->sys.size(); ++i)
    if (b->sys[i]) e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
  return e;
}

// the caller's stream waits for every admitted system
cudaError_t join_to_main(kbe_batch *b) {
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; e == cudaSuccess && i < b->sys.size(); ++i)
    if (b->sys[i]) {
      e = cudaEventRecord(b->done[i], b->streams[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->done[i], 0);
    }
  return e;
}

}  // namespace

extern "C" {

kbe_status kbe_batch_create(int nsys, const kbe_config *cfgs, void *stream, size_t budget_bytes,
                            kbe_batch **out, int *admitted) {
  if (nsys < 1 || !cfgs || !out) return batch_fail(KBE_ERR_ARG, "batch_create: bad arguments");
  *out = nullptr;
  size_t budget = budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
    budget = fr > ((size_t)2 << 30) ? fr - ((size_t)2 << 30) : 0;
  }
  kbe_batch *b = new kbe_batch();
  b->main = (cudaStream_t)stream;
  b->sys.assign((size_t)nsys, nullptr);
  b->streams.assign((size_t)nsys, nullptr);
  b->done.assign((size_t)nsys, nullptr);
  b->nt_max.assign((size_t)nsys, 0);
  b->cur.assign((size_t)nsys, -1);
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return batch_fail(KBE_ERR_CUDA, "batch_create: event");
  }
  size_t used = 0;
  for (int i = 0; i < nsys; ++i) {
    if (admitted) admitted[i] = 0;
    const size_t need = kbe_memory_bytes(&cfgs[i]);
    if (need == 0) {
      destroy_all(b);
      delete b;
      return batch_fail(KBE_ERR_ARG, "batch_create: invalid config for system " + std::to_string(i));
    }
    if (used + need > budget) continue;   // not admitted: does not fit
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[(size_t)i], cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      destroy_all(b);
      delete b;
      return batch_fail(KBE_ERR_CUDA, "batch_create: stream / event");
    }
    kbe_handle *h = nullptr;
    kbe_status s = kbe_create(&cfgs[i], st, &h);
    if (s == KBE_ERR_OOM) {   // the estimate was optimistic: leave it out
      cudaStreamDestroy(st);
      cudaEventDestroy(b->done[(size_t)i]);
      b->done[(size_t)i] = nullptr;
      cudaGetLastError();
      continue;
    }
    if (s != KBE_OK) {
      cudaStreamDestroy(st);
      destroy_all(b);
      delete b;
      return s;
    }
    b->sys[(size_t)i] = h;
    b->streams[(size_t)i] = st;
    b->nt_max[(size_t)i] = cfgs[i].nt_max;
    used += need;
    if (admitted) admitted[i] = 1;
  }
  *out = b;
  return KBE_OK;
}

kbe_status kbe_batch_destroy(kbe_batch *b) {
  if (!b) return KBE_ERR_ARG;
  cudaStreamSynchronize(b->main);
  destroy_all(b);
  delete b;
  return KBE_OK;
}

kbe_handle *kbe_batch_system(kbe_batch *b, int i) {
  if (!b || i < 0 || i >= (int)b->sys.size()) return nullptr;
  return b->sys[(size_t)i];
}

kbe_status kbe_batch_reset(kbe_batch *b) {
  if (!b) return KBE_ERR_ARG;
  cudaError_t e = fork_from_main(b);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_reset: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (!b->sys[i]) continue;
    kbe_status s = kbe_reset(b->sys[i]);
    if (s != KBE_OK) return s;
    b->cur[i] = 0;
  }
  e = join_to_main(b);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_reset: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_batch_step(kbe_batch *b, int nsteps) {
  if (!b || nsteps < 0) return batch_fail(KBE_ERR_ARG, "batch_step: bad arguments");
  cudaError_t e = fork_from_main(b);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
  if (b->graphs) {   // independent systems: each runs its steps as one replayed graph on its stream
    for (size_t i = 0; i < b->sys.size(); ++i) {
      if (!b->sys[i] || b->cur[i] < 0) continue;
      const int k = nsteps < b->nt_max[i] - b->cur[i] ? nsteps : b->nt_max[i] - b->cur[i];
      if (k <= 0) continue;
      kbe_status s = kbe_step(b->sys[i], k);
      if (s != KBE_OK) return s;
      b->cur[i] += k;
    }
    e = join_to_main(b);
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
    return KBE_OK;
  }
  for (int t = 0; t < nsteps; ++t) {
    bool any = false;
    for (size_t i = 0; i < b->sys.size(); ++i) {
      if (!b->sys[i] || b->cur[i] < 0 || b->cur[i] >= b->nt_max[i]) continue;
      kbe_status s = kbe_step(b->sys[i], 1);
      if (s != KBE_OK) return s;
      b->cur[i] += 1;
      any = true;
    }
    if (!any) break;
  }
  e = join_to_main(b);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_batch_set_graphs(kbe_batch *b, int enable) {
  if (!b) return KBE_ERR_ARG;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (!b->sys[i]) continue;
    kbe_status s = kbe_set_graphs(b->sys[i], enable);
    if (s != KBE_OK) return s;
  }
  b->graphs = enable != 0;
  return KBE_OK;
}

kbe_status kbe_batch_synchronize(kbe_batch *b) {
  if (!b) return KBE_ERR_ARG;
  kbe_status first = KBE_OK;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (!b->sys[i]) continue;
    kbe_status s = kbe_synchronize(b->sys[i]);
    if (s != KBE_OK && first == KBE_OK) first = s;
  }
  return first;
}

}  // extern "C"
