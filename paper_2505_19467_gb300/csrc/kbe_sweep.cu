// (a2) Collision integrals on the new time row (Eq. 6 of the paper, read in
// the left Sigma * G form, trapezoid quadrature):
//   I^x(n,j) = sum_{l=0}^{n} w^(n)_l [S^>(n,l) - S^<(n,l)] G^x(l,j)
//            + sum_{l=0}^{j} w^(j)_l  S^x(n,l) [G^<(l,j) - G^>(l,j)]
// for j = 0..n and x in {<, >}. The history holds G only for l >= j; above
// the diagonal G(l,j) = -G(j,l)^+ (the paper keeps G^> below and G^< above
// the diagonal for the same reason).
//
// Work per evaluation: 3 N_b^3 complex multiply-adds per stored block and k,
// i.e. 24 n^2 N_b^3 n_k flops for n^2 N_b^2 n_k complex numbers read: about
// 1.5 N_b flop per byte in FP64, far right of the FP64 ridge on GB300 (the
// FP64 pipe is ~1.2 TFLOP/s against ~7 TB/s of HBM). The kernel is therefore
// written to keep the FP64 pipe busy: every thread owns one (k, a) output row
// of both components in registers and streams the l sum; the N_b threads
// sharing a k read the same block through L1.
#include "kbe_internal.cuh"

namespace kbe {

namespace {

template <int NB>
__global__ void __launch_bounds__(128) sweep_f64_kernel(const double2 *__restrict__ H,
                                                        const double2 *__restrict__ Sig,
                                                        double2 *__restrict__ Iout, int n, int nk,
                                                        double dt) {
  const int j = blockIdx.x;
  const int idx = blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= NB * nk) return;
  const int a = idx / nk;
  const int k = idx - a * nk;
  const size_t blk = (size_t)NB * NB * nk;

  double2 accL[NB], accG[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) accL[b] = accG[b] = make_double2(0.0, 0.0);

  for (int l = 0; l <= n; ++l) {
    const double2 *sl = Sig + (size_t)l * 2 * blk + (size_t)a * NB * nk + k;   // S^<(n,l)_{a,.}
    const double2 *sg = sl + blk;
    const double w1 = trap_weight(n, l, dt);
    const double w2 = (l <= j) ? trap_weight(j, l, dt) : 0.0;
    const bool lower = (l >= j);
    const double2 *gl = H + (lower ? tri(l, j) : tri(j, l)) * 2 * blk + k;
    const double2 *gg = gl + blk;
#pragma unroll 1
    for (int c = 0; c < NB; ++c) {
      const double2 s_l = sl[(size_t)c * nk];
      const double2 s_g = sg[(size_t)c * nk];
      const double2 a1 = c_scale(w1, c_sub(s_g, s_l));
      const double2 a2l = c_scale(w2, s_l);
      const double2 a2g = c_scale(w2, s_g);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        double2 Bl, Bg;
        if (lower) {   // G(l,j)_cb stored directly
          Bl = gl[(size_t)(c * NB + b) * nk];
          Bg = gg[(size_t)(c * NB + b) * nk];
        } else {       // G(l,j)_cb = -conj(G(j,l)_bc)
          Bl = c_neg(c_conj(gl[(size_t)(b * NB + c) * nk]));
          Bg = c_neg(c_conj(gg[(size_t)(b * NB + c) * nk]));
        }
        accL[b] = c_fma(a1, Bl, accL[b]);
        accG[b] = c_fma(a1, Bg, accG[b]);
        if (w2 != 0.0) {
          const double2 d = c_sub(Bl, Bg);
          accL[b] = c_fma(a2l, d, accL[b]);
          accG[b] = c_fma(a2g, d, accG[b]);
        }
      }
    }
  }
  double2 *il = Iout + (size_t)j * 2 * blk + (size_t)a * NB * nk + k;
  double2 *ig = il + blk;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    il[(size_t)b * nk] = accL[b];
    ig[(size_t)b * nk] = accG[b];
  }
}

template <int NB>
cudaError_t sweep_nb(const Mesh &m, int n, double dt, const double2 *H, const double2 *Sig,
                     double2 *I, cudaStream_t st) {
  const int threads = 128;
  dim3 grid(n + 1, (NB * m.nk + threads - 1) / threads);
  sweep_f64_kernel<NB><<<grid, threads, 0, st>>>(H, Sig, I, n, m.nk, dt);
  return cudaGetLastError();
}

}  // namespace

bool sweep_supported(int nb) {
  switch (nb) {
    case 1: case 2: case 3: case 4: case 6: case 8: case 12: case 16: return true;
    default: return false;
  }
}

cudaError_t launch_sweep(const Mesh &m, int n, double dt, int precision, const double2 *H,
                         const double2 *Sig, double2 *I, cudaStream_t st) {
  if (precision != KBE_PREC_FP64) return cudaErrorInvalidValue;
  switch (m.nb) {
    case 1: return sweep_nb<1>(m, n, dt, H, Sig, I, st);
    case 2: return sweep_nb<2>(m, n, dt, H, Sig, I, st);
    case 3: return sweep_nb<3>(m, n, dt, H, Sig, I, st);
    case 4: return sweep_nb<4>(m, n, dt, H, Sig, I, st);
    case 6: return sweep_nb<6>(m, n, dt, H, Sig, I, st);
    case 8: return sweep_nb<8>(m, n, dt, H, Sig, I, st);
    case 12: return sweep_nb<12>(m, n, dt, H, Sig, I, st);
    case 16: return sweep_nb<16>(m, n, dt, H, Sig, I, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kbe
