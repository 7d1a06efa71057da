// (a1) Second-Born self-energy on the new time row (Eq. 7 of the paper).
//
// The paper evaluates Eq. 7 as k-space sums: the direct term in two
// O(n_k^2) steps (polarisability Eq. 8, then the contraction Eq. 9) and the
// exchange term by the O(n_k^3) loop of Algorithm 2. Both terms are
// convolutions over the mesh, so with G(R) = (1/n_k) sum_k e^{ik.R} G(k) they
// become point-wise products in real space:
//   Sigma^<_jm(R) = -U_n U_l sum_ab v_ja v_mb [ G^<_jm G^<_ab conj(G^>_ab)
//                                              - G^<_jb conj(G^>_ab) G^<_am ](R)
// using G^x(k; t_l, t_n) = -G^x(k; t_n, t_l)^+, i.e. G'_ba(-R) = -conj(G_ab(R)).
// Sigma^> is the same with < and > exchanged. The row is handled in three
// launches over all n+1 time pairs at once (the paper's single-launch row):
//   1. forward DFT of every (l, x, a, b) array,
//   2. band products per (l, j, R),
//   3. inverse DFT into the Sigma row.
// Cost per pair: O(N_b^2 n_k (L0 + L1)) for the DFTs and O(N_b^3 n_k) for the
// products, against O(N_b^4 n_k^3) for Algorithm 2.
#include "kbe_internal.cuh"

namespace kbe {

namespace {

// Separable 2-D DFT of length-n_k arrays (mesh L0 x L1, k = k0 * L1 + k1):
//   out[R] = scale * sum_k exp(sign * i * 2 pi (k0 R0 / L0 + k1 R1 / L1)) in[k].
// One CTA per array (grid-stride over arrays); the array and the half-way
// result live in shared memory together with the twiddle tables.
__global__ void dft_rows_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                                long narr, int L0, int L1, int sign, double scale) {
  extern __shared__ double2 sm[];
  const int nk = L0 * L1;
  double2 *x = sm;
  double2 *t = x + nk;
  double2 *tw0 = t + nk;
  double2 *tw1 = tw0 + L0;
  for (int i = threadIdx.x; i < L0; i += blockDim.x) {
    double s, c;
    sincospi(2.0 * i / L0, &s, &c);
    tw0[i] = make_double2(c, sign * s);
  }
  for (int i = threadIdx.x; i < L1; i += blockDim.x) {
    double s, c;
    sincospi(2.0 * i / L1, &s, &c);
    tw1[i] = make_double2(c, sign * s);
  }
  for (long arr = blockIdx.x; arr < narr; arr += gridDim.x) {
    const double2 *src = in + arr * nk;
    __syncthreads();
    for (int e = threadIdx.x; e < nk; e += blockDim.x) x[e] = src[e];
    __syncthreads();
    for (int e = threadIdx.x; e < nk; e += blockDim.x) {
      const int k0 = e / L1, R1 = e - (e / L1) * L1;
      double2 acc = make_double2(0.0, 0.0);
      int ph = 0;
      for (int k1 = 0; k1 < L1; ++k1) {
        acc = c_fma(tw1[ph], x[k0 * L1 + k1], acc);
        ph += R1;
        if (ph >= L1) ph -= L1;
      }
      t[e] = acc;
    }
    __syncthreads();
    double2 *dst = out + arr * nk;
    for (int e = threadIdx.x; e < nk; e += blockDim.x) {
      const int R0 = e / L1, R1 = e - (e / L1) * L1;
      double2 acc = make_double2(0.0, 0.0);
      int ph = 0;
      for (int k0 = 0; k0 < L0; ++k0) {
        acc = c_fma(tw0[ph], t[k0 * L1 + R1], acc);
        ph += R0;
        if (ph >= L0) ph -= L0;
      }
      dst[e] = c_scale(scale, acc);
    }
  }
}

struct VMat {
  double v[kMaxNb * kMaxNb];
};

// Real-space second-Born products for one (l, j, R): all m, both components.
template <int NB>
__global__ void __launch_bounds__(128) sigma_products_kernel(const double2 *__restrict__ GR,
                                                             double2 *__restrict__ SR, int n, int nk,
                                                             double Un, const double *__restrict__ Ul,
                                                             VMat vm) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)(n + 1) * NB * nk;
  if (idx >= total) return;
  const int R = (int)(idx % nk);
  const long t = idx / nk;
  const int j = (int)(t % NB);
  const int l = (int)(t / NB);
  const size_t blk = (size_t)NB * NB * nk;
  const double2 *gl = GR + (size_t)l * 2 * blk + R;
  const double2 *gg = gl + blk;
  const double fac = -Un * (Ul ? Ul[l] : Un);
  double2 *sl = SR + (size_t)l * 2 * blk + (size_t)j * NB * nk + R;
  double2 *sg = sl + blk;
#pragma unroll 1
  for (int m = 0; m < NB; ++m) {
    double2 QL = make_double2(0, 0), QG = make_double2(0, 0);
    double2 EL = make_double2(0, 0), EG = make_double2(0, 0);
#pragma unroll 1
    for (int a = 0; a < NB; ++a) {
      const double vja = vm.v[j * NB + a];
      if (vja == 0.0) continue;
      double2 zl = make_double2(0, 0), yl = make_double2(0, 0), yg = make_double2(0, 0);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const double vmb = vm.v[m * NB + b];
        if (vmb == 0.0) continue;
        const double2 gl_ab = gl[(size_t)(a * NB + b) * nk];
        const double2 gg_ab = gg[(size_t)(a * NB + b) * nk];
        const double2 gl_jb = gl[(size_t)(j * NB + b) * nk];
        const double2 gg_jb = gg[(size_t)(j * NB + b) * nk];
        zl = c_add(zl, c_scale(vmb, c_mulc(gl_ab, gg_ab)));   // M_ab = G^<_ab conj(G^>_ab)
        yl = c_add(yl, c_scale(vmb, c_mulc(gl_jb, gg_ab)));   // G^<_jb conj(G^>_ab)
        yg = c_add(yg, c_scale(vmb, c_mulc(gg_jb, gl_ab)));   // G^>_jb conj(G^<_ab)
      }
      QL = c_add(QL, c_scale(vja, zl));
      QG = c_add(QG, c_scale(vja, c_conj(zl)));              // M^>_ab = conj(M^<_ab)
      EL = c_fma(c_scale(vja, gl[(size_t)(a * NB + m) * nk]), yl, EL);
      EG = c_fma(c_scale(vja, gg[(size_t)(a * NB + m) * nk]), yg, EG);
    }
    const double2 gl_jm = gl[(size_t)(j * NB + m) * nk];
    const double2 gg_jm = gg[(size_t)(j * NB + m) * nk];
    sl[(size_t)m * nk] = c_scale(fac, c_sub(c_mul(gl_jm, QL), EL));
    sg[(size_t)m * nk] = c_scale(fac, c_sub(c_mul(gg_jm, QG), EG));
  }
}

template <int NB>
cudaError_t products_nb(const Mesh &m, const VMat &vm, int n, double Un, const double *Ul,
                        const double2 *GR, double2 *SR, cudaStream_t st) {
  const long total = (long)(n + 1) * NB * m.nk;
  const int threads = 128;
  const long blocks = (total + threads - 1) / threads;
  sigma_products_kernel<NB><<<(unsigned)blocks, threads, 0, st>>>(GR, SR, n, m.nk, Un, Ul, vm);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dft_rows(const double2 *in, double2 *out, long narr, int L0, int L1, int sign,
                            double scale, cudaStream_t st) {
  if (narr <= 0) return cudaSuccess;
  const int nk = L0 * L1;
  const size_t smem = sizeof(double2) * (2 * (size_t)nk + L0 + L1);
  static size_t attr_bytes = 48 * 1024;  // default opt-in limit
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(dft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  int threads = nk >= 256 ? 256 : ((nk + 31) / 32) * 32;
  long blocks = narr < 152L * 32 ? narr : 152L * 32;
  dft_rows_kernel<<<(unsigned)blocks, threads, smem, st>>>(in, out, narr, L0, L1, sign, scale);
  return cudaGetLastError();
}

cudaError_t launch_sigma_products(const Mesh &m, const double *v, int n, double Un,
                                  const double *Ul_dev, const double2 *GR, double2 *SR,
                                  cudaStream_t st) {
  VMat vm;
  for (int i = 0; i < kMaxNb * kMaxNb; ++i) vm.v[i] = 0.0;
  for (int i = 0; i < m.nb * m.nb; ++i) vm.v[i] = v[i];
  switch (m.nb) {
    case 1: return products_nb<1>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 2: return products_nb<2>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 3: return products_nb<3>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 4: return products_nb<4>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 6: return products_nb<6>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 8: return products_nb<8>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 12: return products_nb<12>(m, vm, n, Un, Ul_dev, GR, SR, st);
    case 16: return products_nb<16>(m, vm, n, Un, Ul_dev, GR, SR, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t sigma_workspace_bytes(const Mesh &m, int n) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  return 2 * (size_t)(n + 1) * 2 * blk * sizeof(double2);
}

cudaError_t sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                      const double2 *Grow, double2 *Sig, double2 *work, cudaStream_t st) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const long narr = (long)(n + 1) * 2 * m.nb * m.nb;
  double2 *GR = work;
  double2 *SR = work + (size_t)(n + 1) * 2 * blk;
  cudaError_t e = launch_dft_rows(Grow, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st);
  if (e != cudaSuccess) return e;
  e = launch_sigma_products(m, v_host, n, Un, Ul_dev, GR, SR, st);
  if (e != cudaSuccess) return e;
  return launch_dft_rows(SR, Sig, narr, m.L0, m.L1, -1, 1.0, st);
}

}  // namespace kbe
