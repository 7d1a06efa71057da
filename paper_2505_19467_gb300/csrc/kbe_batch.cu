// Batched systems: many independent Kadanoff-Baym systems of uneven size
// advanced together on one GPU.
//
// Every admitted system is an ordinary handle on its own stream, forked from
// the caller's stream with an event and joined back after each call, so the
// kernels of different systems overlap on the GPU (a small system's launches
// fill SMs that a large system's tail leaves idle). Steps are enqueued one
// time step of all systems at a time, so no system runs far ahead of the
// others. With graphs on (kbe_batch_set_graphs) and a non-default stream, one
// call's steps of every system are captured into a single graph (each system's
// kernels on its own stream inside it, forked from and joined to the caller's
// stream) and later calls with the same row, count and ring order replay it
// with one launch; on the default stream each system replays its own graph.
// Admission is by
// device memory: systems are taken in order while their allocation fits the
// budget; the others are reported as not admitted.
#include <cstdio>
#include <map>
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
  bool graphs = false;              // replay captured steps (kbe_batch_set_graphs)
  kbe::GraphCache<std::vector<long>> gcache;   // one graph per call shape of the batch
};

namespace {

kbe_status batch_fail(kbe_status s, const std::string &msg) {
  kbe::set_last_error(msg);
  return s;
}

void drop_batch_graphs(kbe_batch *b) { b->gcache.clear(); }

// a cached batch graph whose key holds an outdated input generation of one of
// its systems can never be replayed again (key: nsteps, then per stepped
// system i, row, count, ring order, generation)
void drop_stale_batch_graphs(kbe_batch *b) {
  b->gcache.drop_if([b](const std::vector<long> &key) {
    for (size_t q = 1; q + 4 < key.size(); q += 5) {
      const size_t i = (size_t)key[q];
      if (i >= b->sys.size() || !b->sys[i]) return true;
      int ring = 0;
      unsigned gen = 0;
      kbe::step_key(b->sys[i], &ring, &gen);
      if ((long)gen != key[q + 4]) return true;
    }
    return false;
  });
}

void destroy_all(kbe_batch *b) {
  drop_batch_graphs(b);
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

// steps of every system for one kbe_batch_step call (k_i each)
std::vector<int> step_counts(const kbe_batch *b, int nsteps) {
  std::vector<int> k(b->sys.size(), 0);
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (!b->sys[i] || b->cur[i] < 0) continue;
    const int left = b->nt_max[i] - b->cur[i];
    k[i] = nsteps < left ? nsteps : left;
  }
  return k;
}

// one graph for the whole batch: captured on the caller's stream, each system
// forked onto its own stream inside the capture and joined back
kbe_status batch_graph_step(kbe_batch *b, int nsteps) {
  // the graph runs on the caller's stream: order it after work enqueued on a
  // system's own stream outside the batch calls (kbe_set_* on a borrowed handle)
  cudaError_t ej = join_to_main(b);
  if (ej != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(ej));
  const std::vector<int> k = step_counts(b, nsteps);
  std::vector<long> key{nsteps};
  for (size_t i = 0; i < b->sys.size(); ++i) {
    if (!b->sys[i] || k[i] <= 0) continue;
    kbe_status s = kbe::step_check(b->sys[i], k[i]);
    if (s != KBE_OK) return s;
    int ring = 0;
    unsigned gen = 0;
    kbe::step_key(b->sys[i], &ring, &gen);
    key.insert(key.end(), {(long)i, (long)b->cur[i], (long)k[i], (long)ring, (long)gen});
  }
  cudaGraphExec_t exec = b->gcache.find(key);
  if (!exec) {
    drop_stale_batch_graphs(b);
    for (size_t i = 0; i < b->sys.size(); ++i)
      if (b->sys[i] && k[i] > 0) {
        kbe_status s = kbe::step_prepare(b->sys[i]);
        if (s != KBE_OK) return s;
      }
    cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    kbe_status s = KBE_OK;
    e = cudaEventRecord(b->fork, b->main);
    for (size_t i = 0; i < b->sys.size() && s == KBE_OK && e == cudaSuccess; ++i) {
      if (!b->sys[i] || k[i] <= 0) continue;
      e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (e == cudaSuccess) s = kbe::step_record(b->sys[i], k[i]);
      if (s == KBE_OK && e == cudaSuccess) e = cudaEventRecord(b->done[i], b->streams[i]);
      if (s == KBE_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->done[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->main, &graph);
    if (s != KBE_OK || e != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (s != KBE_OK) return s;
      return batch_fail(KBE_ERR_CUDA, std::string("batch graph capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    b->gcache.put(key, exec);
  }
  cudaError_t e = cudaGraphLaunch(exec, b->main);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (b->sys[i] && k[i] > 0) {
      kbe::step_advance(b->sys[i], k[i]);
      b->cur[i] += k[i];
    }
  return KBE_OK;
}

bool batch_capturable(const kbe_batch *b) {
  if (b->main == nullptr) return false;   // the legacy default stream cannot be captured
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (b->sys[i] && !kbe::step_capturable(b->sys[i])) return false;
  return true;
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
  cudaError_t e;
  if (b->graphs && batch_capturable(b)) {
    kbe_status s = batch_graph_step(b, nsteps);
    if (s != KBE_OK) return s;
    e = fork_from_main(b);   // later work on a system's own stream follows the replayed graph
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
    return KBE_OK;
  }
  e = fork_from_main(b);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
  if (b->graphs) {   // default stream: each system replays its own graph on its stream
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
  cudaError_t e = cudaStreamSynchronize(b->main);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_set_graphs: ") + cudaGetErrorString(e));
  drop_batch_graphs(b);
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
