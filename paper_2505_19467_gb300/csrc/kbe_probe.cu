// Arithmetic-throughput probe: the FP64 and FP32 fused multiply-add rates this
// device sustains, measured with CUDA events. They are the denominators of the
// roofline fractions of the ALU-bound sweep forms (the FP64 sweep is bound by
// the FP64 pipe, the double-float and complex64 forms by the FP32 pipe).
//
// Each thread runs 4, 8 or 16 independent FMA chains for `iters` rounds, in
// two forms (accumulation with register operands, and iteration), on a grid of
// 4 or 8 CTAs of 256 threads per SM; the largest rate of the twelve
// configurations is the result (a single one can sit below the pipe's rate on
// dependency latency or operand handling). The chains' values are folded into one store that the
// compiler cannot remove (it happens only if the sum is exactly a sentinel
// that finite inputs never reach).
#include <string>

#include "kbe_internal.cuh"

namespace {

constexpr int kThreads = 256;

// CHAINS independent chains per thread, `iters` rounds, in one of two forms:
// ACC = 1 accumulates (acc = fma(p, q, acc), register operands, as the sweep
// uses the pipe), ACC = 0 iterates x = fma(x, a, b). Both stay bounded.
template <class T, int CHAINS, int ACC>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T a, T b, T *sink) {
  T x[CHAINS], p[CHAINS];
  const T q = b * (T)(1 + (threadIdx.x & 1));
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    p[c] = a * (T)(c + 1);
  }
#pragma unroll 8   // iters is a multiple of 8: the loop's own instructions stay negligible
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = ACC ? fma(p[c], q, x[c]) : fma(x[c], (T)0.999, q);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == (T)-12345.678) *sink = s;
}

// best of three timed runs (after one untimed) of one configuration, GFLOP/s
template <class T, int CHAINS, int ACC>
cudaError_t probe_config(int ctas_per_sm, T *sink, cudaEvent_t e0, cudaEvent_t e1, double *gflops) {
  const unsigned blocks = (unsigned)(kbe::device_sms() * ctas_per_sm);
  // ~80 ms per FP64 run, ~20 ms per FP32 run at the nominal rates
  const int iters = (sizeof(T) == 8 ? (1 << 20) : (1 << 24)) / (CHAINS * ctas_per_sm);
  const T a = (T)1e-3, b = (T)1e-3;   // x stays ~ 1 in both forms: no overflow or subnormals
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      fma_probe_kernel<T, CHAINS, ACC><<<blocks, kThreads>>>(iters, a, b, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) *gflops = 2.0 * CHAINS * (double)iters * kThreads * blocks / (best * 1e-3) / 1e9;
  return e;
}

// the largest rate over chain counts and occupancies (a single configuration
// can sit below the pipe's rate on dependency latency or issue)
template <class T>
cudaError_t run_probe(double *gflops) {
  T *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int occ : {4, 8}) {
    double g[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = probe_config<T, 4, 1>(occ, sink, e0, e1, &g[0]);
    if (e == cudaSuccess) e = probe_config<T, 8, 1>(occ, sink, e0, e1, &g[1]);
    if (e == cudaSuccess) e = probe_config<T, 16, 1>(occ, sink, e0, e1, &g[2]);
    if (e == cudaSuccess) e = probe_config<T, 4, 0>(occ, sink, e0, e1, &g[3]);
    if (e == cudaSuccess) e = probe_config<T, 8, 0>(occ, sink, e0, e1, &g[4]);
    if (e == cudaSuccess) e = probe_config<T, 16, 0>(occ, sink, e0, e1, &g[5]);
    for (double x : g) best = x > best ? x : best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return e;
  *gflops = best;
  return cudaSuccess;
}

}  // namespace

extern "C" kbe_status kbe_measure_fma_peaks(double *fp64_gflops, double *fp32_gflops) {
  cudaError_t e = cudaSuccess;
  if (fp64_gflops) e = run_probe<double>(fp64_gflops);
  if (e == cudaSuccess && fp32_gflops) e = run_probe<float>(fp32_gflops);
  if (e != cudaSuccess) {
    kbe::set_last_error(std::string("measure_fma_peaks: ") + cudaGetErrorString(e));
    return KBE_ERR_CUDA;
  }
  return KBE_OK;
}
