// kbe_op_sigma_row_noalloc: the second-Born self-energy row (same operation
// as kbe_op_sigma_row) with its scratch held inside the library instead of
// being passed in by the caller.
//
// Some callers cannot allocate device memory at the point where they need
// the self-energy: hosts that hand the whole GPU to their own allocator (a
// framework's caching pool that has already reserved the device memory, so a
// raw cudaMalloc may fail or fragment it), latency-critical loops where
// cudaMalloc / cudaFree would synchronise the device, and plug-in or embedded
// hosts whose device-memory budget is fixed when they start. For them this
// entry point uses one fixed, file-scope device array and allocates nothing.
//
// The array costs kNoAllocScratchBytes of device memory on every GPU that
// loads the library, for the life of the process. It is shared by all calls:
// calls whose work overlaps on the GPU (several streams, several host
// threads) race on it and must be serialised by the caller. Nothing in it has
// to start at zero: every scratch element a call reads was written earlier in
// the same call (forward transform, then band products), so the stale
// contents left by the previous call are never used.
#include <mutex>
#include <string>

#include "kbe_internal.cuh"

static constexpr size_t kNoAllocScratchBytes = KBE_NOALLOC_SCRATCH_BYTES;
static_assert(kNoAllocScratchBytes % sizeof(double2) == 0, "scratch size");

// In host code this name only stands in for the device array; its device
// address comes from cudaGetSymbolAddress (once per device, below).
static __device__ __align__(256) double2 g_sigma_scratch[kNoAllocScratchBytes / sizeof(double2)];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, resolved on the
// first call for that device (the device must be current; done before any
// stream capture by calling this entry point once first).
cudaError_t scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sigma_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// the message is read back with kbe_last_error(NULL)
kbe_status noalloc_fail(kbe_status s, const std::string &msg) {
  kbe::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" kbe_status kbe_op_sigma_row_noalloc(const kbe_mesh *m, const double *v, int n, double Un,
                                               const double *Ul_dev, const void *Grow_dev,
                                               void *Sigma_dev, void *stream) {
  if (!m || !v || n < 0 || !Grow_dev || !Sigma_dev || !kbe::sweep_supported(m->nb) || m->L[0] < 1 ||
      m->L[1] < 1 || (long)m->L[0] * m->L[1] > kbe::kMaxNk)
    return noalloc_fail(KBE_ERR_ARG, "op_sigma_row_noalloc: bad arguments");
  const kbe::Mesh mm{m->nb, m->L[0], m->L[1], m->L[0] * m->L[1]};
  const size_t need = kbe::sigma_workspace_bytes(mm, n);
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(KBE_ERR_ARG, "op_sigma_row_noalloc: this row needs " + std::to_string(need) +
                                         " bytes of scratch; the built-in array holds " +
                                         std::to_string(kNoAllocScratchBytes) +
                                         " (use kbe_op_sigma_row with caller scratch)");
  void *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return noalloc_fail(KBE_ERR_CUDA, std::string("op_sigma_row_noalloc: scratch address: ") +
                                          cudaGetErrorString(e));
  e = kbe::sigma_row(mm, v, n, Un, Ul_dev, (const double2 *)Grow_dev, (double2 *)Sigma_dev,
                     (double2 *)scratch, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return noalloc_fail(KBE_ERR_CUDA, std::string("op_sigma_row_noalloc: ") + cudaGetErrorString(e));
  return KBE_OK;
}
