// Arithmetic-throughput probe: the FP64 and FP32 fused multiply-add rates this
// device sustains, measured with CUDA events. They are the denominators of the
// roofline fractions of the ALU-bound sweep forms (the FP64 sweep is bound by
// the FP64 pipe, the double-float and complex64 forms by the FP32 pipe).
//
// Each thread runs kChains independent FMA chains (enough to cover the pipe's
// latency) for `iters` rounds; the grid is a multiple of the SM count with
// several CTAs per SM. The chains' values are folded into one store that the
// compiler cannot remove (it happens only if the sum is exactly a sentinel
// that finite inputs never reach).
#include <string>

#include "kbe_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T a, T b, T *sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.678) *sink = s;
}

template <class T>
cudaError_t run_probe(double *gflops) {
  const int sms = kbe::device_sms();
  const unsigned blocks = (unsigned)sms * 8;
  const int iters = sizeof(T) == 8 ? (1 << 14) : (1 << 18);   // ~50 ms and ~20 ms per run
  T *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a and b keep x bounded (|a| < 1): no overflow, no subnormals
  const T a = (T)0.999, b = (T)1e-4;
  float best = 1e30f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {   // the first round is a warm-up
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      fma_probe_kernel<T><<<blocks, kThreads>>>(iters, a, b, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kChains * (double)iters * kThreads * blocks;
  *gflops = flops / (best * 1e-3) / 1e9;
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
