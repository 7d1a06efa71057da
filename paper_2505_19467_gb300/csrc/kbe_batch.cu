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
// In the persistent mode (kbe_batch_set_persistent, FP64 histories) the steps
// are enqueued stage-major: every system runs its step up to its next collision
// sweep on its own stream, then ONE persistent launch per sweep class (N_b,
// quadrature, kernel form) and lane (the systems of a class alternate between
// two lanes), on that lane's own stream, runs the sweeps of the lane's
// systems, walking the concatenation of their block lists (each system's
// blocks at its own autotuned split), and the systems continue from there; a
// launch waits only for its own lane's systems. With graphs on and a
// non-default stream the whole call is again one captured graph.
// Admission is by
// device memory: systems are taken in order while their allocation fits the
// budget; the others are reported as not admitted.
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

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
  bool persistent = false;          // stage-major steps, batched sweeps (kbe_batch_set_persistent)
  long sweep_launches = 0;          // persistent sweep launches enqueued (for reporting)
  std::map<int, cudaStream_t> class_streams;   // persistent mode: one stream per sweep class
  std::vector<int> classes_used;    // the classes the current call launched on (joined at its end)
  cudaEvent_t class_done = nullptr;
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
  for (auto &cs : b->class_streams) cudaStreamDestroy(cs.second);
  b->class_streams.clear();
  if (b->class_done) cudaEventDestroy(b->class_done);
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

// the sweep class of a job: the jobs of one class share one persistent launch
int sweep_class(const kbe::SweepJob &j) { return (j.nb * 2 + j.quad) * 2 + j.f64m; }
constexpr int kClassLanes = 2;

cudaError_t class_stream(kbe_batch *b, int cls, cudaStream_t *out) {
  bool seen = false;
  for (int c : b->classes_used) seen = seen || c == cls;
  if (!seen) b->classes_used.push_back(cls);
  auto it = b->class_streams.find(cls);
  if (it != b->class_streams.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (!b->class_done) e = cudaEventCreateWithFlags(&b->class_done, cudaEventDisableTiming);
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  b->class_streams[cls] = st;
  *out = st;
  return cudaSuccess;
}

// the caller's stream waits for the class streams the call launched on (a
// capture must rejoin them; a class stream the call did not use is not part
// of the capture and must not be waited on inside it)
cudaError_t join_classes(kbe_batch *b) {
  cudaError_t e = cudaSuccess;
  for (int c : b->classes_used) {
    cudaStream_t cs = b->class_streams[c];
    if (e == cudaSuccess) e = cudaEventRecord(b->class_done, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->class_done, 0);
  }
  b->classes_used.clear();
  return e;
}

// the steps k[i] of every system, stage-major: per time step, each system's
// segments up to its next collision sweep on its own stream; at each cut the
// systems that stopped there are grouped by sweep class (N_b, quadrature,
// form), each class's sweeps run as one launch on the class's stream once
// its systems have arrived, and its systems continue after it. Systems with
// fewer steps or segments drop out of the later cuts. Ends with the systems'
// and the classes' streams ahead of the caller's (join_to_main and
// join_classes follow).
kbe_status persistent_enqueue(kbe_batch *b, const std::vector<int> &k) {
  const size_t ns = b->sys.size();
  b->classes_used.clear();
  int kmax = 0;
  for (size_t i = 0; i < ns; ++i)
    if (b->sys[i] && k[i] > kmax) kmax = k[i];
  std::vector<kbe::SweepJob> jobs(ns);
  std::vector<kbe::SweepJob> group;
  std::vector<size_t> who;
  for (int t = 0; t < kmax; ++t) {
    int segs = 0;
    for (size_t i = 0; i < ns; ++i) {
      if (!b->sys[i] || t >= k[i]) continue;
      kbe_status s = step_segment_check(b->sys[i]);
      if (s != KBE_OK) return s;
      const int c = step_segment_count(b->sys[i]);
      if (c > segs) segs = c;
    }
    for (int seg = 0; seg < segs; ++seg) {
      group.clear();
      who.clear();
      for (size_t i = 0; i < ns; ++i) {
        if (!b->sys[i] || t >= k[i] || seg >= step_segment_count(b->sys[i])) continue;
        bool has = false;
        kbe_status s = step_segment(b->sys[i], seg, &jobs[i], &has);
        if (s != KBE_OK) return s;
        if (has) {
          group.push_back(jobs[i]);
          who.push_back(i);
        }
      }
      if (group.empty()) continue;
      // one launch per sweep class (N_b, quadrature, form) and lane, each on
      // its own stream: the systems of a class alternate between kClassLanes
      // lanes, and a launch waits only for the systems of its own lane
      std::vector<char> taken(group.size(), 0);
      for (size_t q0 = 0; q0 < group.size(); ++q0) {
        if (taken[q0]) continue;
        const int base = sweep_class(group[q0]);
        std::vector<kbe::SweepJob> lane_jobs[kClassLanes];
        std::vector<size_t> lane_who[kClassLanes];
        int rank = 0;
        for (size_t q = q0; q < group.size(); ++q)
          if (!taken[q] && sweep_class(group[q]) == base) {
            taken[q] = 1;
            lane_jobs[rank % kClassLanes].push_back(group[q]);
            lane_who[rank % kClassLanes].push_back(who[q]);
            ++rank;
          }
        for (int ln = 0; ln < kClassLanes; ++ln) {
          if (lane_jobs[ln].empty()) continue;
          const std::vector<kbe::SweepJob> &sub = lane_jobs[ln];
          const std::vector<size_t> &subw = lane_who[ln];
          cudaStream_t cs = nullptr;
          cudaError_t e = class_stream(b, base * kClassLanes + ln, &cs);
          for (size_t q = 0; q < subw.size() && e == cudaSuccess; ++q) {
            e = cudaEventRecord(b->done[subw[q]], b->streams[subw[q]]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->done[subw[q]], 0);
          }
          int nl = 0;
          if (e == cudaSuccess) e = kbe::launch_sweep_batch(sub.data(), (int)sub.size(), cs, &nl);
          if (e == cudaSuccess) e = cudaEventRecord(b->class_done, cs);
          for (size_t q = 0; q < subw.size() && e == cudaSuccess; ++q)
            e = cudaStreamWaitEvent(b->streams[subw[q]], b->class_done, 0);
          if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch sweep: ") + cudaGetErrorString(e));
          b->sweep_launches += nl;
        }
      }
    }
  }
  return KBE_OK;
}

// one graph for the whole batch: captured on the caller's stream, each system
// forked onto its own stream inside the capture and joined back
kbe_status batch_graph_step(kbe_batch *b, int nsteps) {
  // the graph runs on the caller's stream: order it after work enqueued on a
  // system's own stream outside the batch calls (kbe_set_* on a borrowed handle)
  cudaError_t ej = join_to_main(b);
  if (ej != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(ej));
  const std::vector<int> k = step_counts(b, nsteps);
  std::vector<long> key{2L * nsteps + (b->persistent ? 1 : 0)};
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
    if (b->persistent) {   // stage-major; the host-side step state is put back after the capture
      std::vector<kbe::StepMark> mk(b->sys.size());
      for (size_t i = 0; i < b->sys.size() && e == cudaSuccess; ++i)
        if (b->sys[i] && k[i] > 0) {
          mk[i] = kbe::step_mark(b->sys[i]);
          e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        }
      const long nl0 = b->sweep_launches;
      if (e == cudaSuccess) s = persistent_enqueue(b, k);
      b->sweep_launches = nl0;
      for (size_t i = 0; i < b->sys.size(); ++i)
        if (b->sys[i] && k[i] > 0) {
          kbe::step_rewind(b->sys[i], mk[i]);
          if (s == KBE_OK && e == cudaSuccess) e = cudaEventRecord(b->done[i], b->streams[i]);
          if (s == KBE_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->done[i], 0);
        }
      if (s == KBE_OK && e == cudaSuccess) e = join_classes(b);
    } else {
      for (size_t i = 0; i < b->sys.size() && s == KBE_OK && e == cudaSuccess; ++i) {
        if (!b->sys[i] || k[i] <= 0) continue;
        e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        if (e == cudaSuccess) s = kbe::step_record(b->sys[i], k[i]);
        if (s == KBE_OK && e == cudaSuccess) e = cudaEventRecord(b->done[i], b->streams[i]);
        if (s == KBE_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->done[i], 0);
      }
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
  struct Range {   // an NVTX range over the call (timeline tools)
    Range() { nvtxRangePushA("kbe: batch step"); }
    ~Range() { nvtxRangePop(); }
  } range;
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
  if (b->persistent) {   // stage-major, eagerly enqueued
    const std::vector<int> k = step_counts(b, nsteps);
    kbe_status s = persistent_enqueue(b, k);
    for (size_t i = 0; i < b->sys.size(); ++i)
      if (b->sys[i] && k[i] > 0) b->cur[i] = kbe::step_mark(b->sys[i]).n;
    if (s != KBE_OK) return s;
    e = join_to_main(b);
    if (e == cudaSuccess) e = join_classes(b);
    if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_step: ") + cudaGetErrorString(e));
    return KBE_OK;
  }
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

kbe_status kbe_batch_set_persistent(kbe_batch *b, int enable) {
  if (!b) return KBE_ERR_ARG;
  if (enable)
    for (size_t i = 0; i < b->sys.size(); ++i)
      if (b->sys[i] && !kbe::step_capturable(b->sys[i]))
        return batch_fail(KBE_ERR_UNSUPPORTED, "batch_set_persistent: a system has profiling or an injected fault on");
  for (size_t i = 0; enable && i < b->sys.size(); ++i)
    if (b->sys[i] && kbe::handle_precision(b->sys[i]) != KBE_PREC_FP64)
      return batch_fail(KBE_ERR_UNSUPPORTED, "batch_set_persistent: the batched sweep needs FP64 histories");
  cudaError_t e = cudaStreamSynchronize(b->main);
  if (e != cudaSuccess) return batch_fail(KBE_ERR_CUDA, std::string("batch_set_persistent: ") + cudaGetErrorString(e));
  drop_batch_graphs(b);
  b->persistent = enable != 0;
  return KBE_OK;
}

long kbe_batch_sweep_launches(const kbe_batch *b) { return b ? b->sweep_launches : -1; }

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
