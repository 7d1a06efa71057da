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
// Cost per pair: O(N_b^2 n_k log n_k) for power-of-two meshes (FFT), else
// O(N_b^2 n_k (L0 + L1)), and O(N_b^3 n_k) for the products, against
// O(N_b^4 n_k^3) for Algorithm 2.
#include <mutex>

#include "kbe_internal.cuh"

namespace kbe {

namespace {

// Separable 2-D DFT of length-n_k arrays (mesh L0 x L1, k = k0 * L1 + k1):
//   out[R] (+)= scale * sum_k exp(sign * i * 2 pi (k0 R0 / L0 + k1 R1 / L1)) in[k]
// (added to out when accumulating).
// One array at a time per CTA (grid-stride over arrays), in shared memory.
// An axis whose length is a power of two is transformed in place by a
// radix-2 FFT (bit reversal, then log2 L butterfly stages; O(L log L));
// other lengths use the direct sum over that axis (O(L^2)). The twiddle
// tables e^{sign 2 pi i m / L} are built once per CTA.

__device__ __forceinline__ bool is_pow2(int L) { return L > 0 && (L & (L - 1)) == 0; }

// in-place FFT of `count` sequences of length L, element i of sequence q at
// x[q * qstride + i * stride]; tw[m] = e^{sign 2 pi i m / L}
__device__ void fft_axis(double2 *x, int L, int stride, int count, int qstride, const double2 *tw) {
  int logL = 0;
  while ((1 << logL) < L) ++logL;
  const int total = count * L;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {   // bit reversal
    const int q = e / L, i = e - q * L;
    const int r = __brev(i) >> (32 - logL);
    if (logL > 0 && i < r) {
      double2 *p = x + q * qstride;
      const double2 t = p[i * stride];
      p[i * stride] = p[r * stride];
      p[r * stride] = t;
    }
  }
  __syncthreads();
  for (int len = 2; len <= L; len <<= 1) {
    const int half = len >> 1, step = L / len, nbf = count * (L >> 1);
    for (int e = threadIdx.x; e < nbf; e += blockDim.x) {
      const int q = e / (L >> 1), bq = e - q * (L >> 1);
      const int grp = bq / half, pos = bq - grp * half;
      double2 *p = x + q * qstride;
      const int i = grp * len + pos, j = i + half;
      const double2 u = p[i * stride];
      const double2 t = c_mul(tw[pos * step], p[j * stride]);
      p[i * stride] = c_add(u, t);
      p[j * stride] = c_sub(u, t);
    }
    __syncthreads();
  }
}

// direct transform of `count` sequences of length L (x -> tmp -> x)
__device__ void dft_axis(double2 *x, double2 *tmp, int L, int stride, int count, int qstride,
                         const double2 *tw) {
  const int total = count * L;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e / L, R = e - q * L;
    const double2 *p = x + q * qstride;
    double2 acc = make_double2(0.0, 0.0);
    int ph = 0;
    for (int kk = 0; kk < L; ++kk) {
      acc = c_fma(tw[ph], p[kk * stride], acc);
      ph += R;
      if (ph >= L) ph -= L;
    }
    tmp[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e / L, R = e - q * L;
    x[q * qstride + R * stride] = tmp[e];
  }
  __syncthreads();
}

__global__ void dft_rows_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                                long narr, int L0, int L1, int sign, double scale, int accumulate,
                                const int *__restrict__ skip) {
  if (skip && *skip) return;
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
    if (L1 > 1) {   // axis 1: L0 contiguous sequences of length L1
      if (is_pow2(L1)) fft_axis(x, L1, 1, L0, L1, tw1);
      else dft_axis(x, t, L1, 1, L0, L1, tw1);
    }
    if (L0 > 1) {   // axis 0: L1 sequences of length L0, stride L1
      if (is_pow2(L0)) fft_axis(x, L0, L1, L1, 1, tw0);
      else dft_axis(x, t, L0, L1, L1, 1, tw0);
    }
    double2 *dst = out + arr * nk;
    if (accumulate)
      for (int e = threadIdx.x; e < nk; e += blockDim.x) dst[e] = c_add(dst[e], c_scale(scale, x[e]));
    else
      for (int e = threadIdx.x; e < nk; e += blockDim.x) dst[e] = c_scale(scale, x[e]);
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
                                                             VMat vm, const int *__restrict__ skip) {
  if (skip && *skip) return;
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

// The products for the pair pattern v = 1 - delta (every pair of distinct bands
// interacts; the paper's two-band bar at N_b = 2). Then the sums over a != j and
// b != m collapse: with T = G^< G^>^+ (per R), the direct sum is
// tr T - r_j - c_m + M_jm (row and column sums of M_ab = G^<_ab conj(G^>_ab)),
// the exchange sum (T G^<)_jm - T_jj G^<_jm - G^<_jm (c_m - M_jm), and with
// T_jj = r_j everything but two terms cancels:
//   Sigma^<(R) = fac [tr(T) G^< - T G^<],   Sigma^> = fac [tr(T)* G^> - T^+ G^>]
// (T^+ = G^> G^<^+): two N_b x N_b products per (l, R) instead of the O(N_b^4)
// double sums. One thread per (l, j, R) forms row j of both.
template <int NB>
__global__ void __launch_bounds__(128) sigma_products_pair_kernel(const double2 *__restrict__ GR,
                                                                  double2 *__restrict__ SR, int n, int nk,
                                                                  double Un, const double *__restrict__ Ul,
                                                                  const int *__restrict__ skip) {
  if (skip && *skip) return;
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
#define AT(M, r, c) M[(size_t)((r) * NB + (c)) * nk]
  double2 tr = make_double2(0, 0);   // tr(G^< G^>^+) = sum_ab G^<_ab conj(G^>_ab)
  double2 Tl[NB], Tg[NB];            // row j of T = G^< G^>^+ and of T^+ = G^> G^<^+
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    double2 sl = make_double2(0, 0), sg = make_double2(0, 0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const double2 xab = AT(gl, a, b), yab = AT(gg, a, b);
      tr = c_add(tr, c_mulc(xab, yab));
      sl = c_add(sl, c_mulc(AT(gl, j, b), yab));
      sg = c_add(sg, c_mulc(AT(gg, j, b), xab));
    }
    Tl[a] = sl;
    Tg[a] = sg;
  }
  double2 *sl = SR + (size_t)l * 2 * blk + (size_t)j * NB * nk + R;
  double2 *sg = sl + blk;
#pragma unroll 1
  for (int m = 0; m < NB; ++m) {
    double2 pl = make_double2(0, 0), pg = make_double2(0, 0);
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      pl = c_fma(Tl[a], AT(gl, a, m), pl);
      pg = c_fma(Tg[a], AT(gg, a, m), pg);
    }
    sl[(size_t)m * nk] = c_scale(fac, c_sub(c_mul(tr, AT(gl, j, m)), pl));
    sg[(size_t)m * nk] = c_scale(fac, c_sub(c_mul(c_conj(tr), AT(gg, j, m)), pg));
  }
#undef AT
}

template <int NB>
cudaError_t products_nb(const Mesh &m, const VMat &vm, int n, double Un, const double *Ul,
                        const double2 *GR, double2 *SR, cudaStream_t st, const int *skip) {
  bool pair = NB >= 3;   // v = 1 - delta exactly (at N_b <= 2 the two forms time the same)
  for (int a = 0; a < NB; ++a)
    for (int b = 0; b < NB; ++b) pair = pair && vm.v[a * NB + b] == (a == b ? 0.0 : 1.0);
  if (pair) {
    const long total = (long)(n + 1) * NB * m.nk;
    sigma_products_pair_kernel<NB><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(GR, SR, n, m.nk, Un, Ul, skip);
    return cudaGetLastError();
  }
  const long total = (long)(n + 1) * NB * m.nk;
  const int threads = 128;
  const long blocks = (total + threads - 1) / threads;
  sigma_products_kernel<NB><<<(unsigned)blocks, threads, 0, st>>>(GR, SR, n, m.nk, Un, Ul, vm, skip);
  return cudaGetLastError();
}

}  // namespace

namespace {
size_t dft_smem_bytes(int L0, int L1) {
  return sizeof(double2) * (2 * (size_t)L0 * L1 + L0 + L1);
}
}  // namespace

// raise the DFT kernel's dynamic shared-memory limit for this mesh (a host-side
// attribute of the current device's context, done before any stream capture
// that launches it); the raised limit is kept per device, under a lock
cudaError_t dft_prepare(int L0, int L1) {
  constexpr size_t kDefault = 48 * 1024;   // no opt-in needed below this
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static size_t raised[kMaxDev] = {};
  const size_t smem = dft_smem_bytes(L0, L1);
  if (smem <= kDefault) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (smem > raised[dev]) {
    e = cudaFuncSetAttribute(dft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    raised[dev] = smem;
  }
  return cudaSuccess;
}

cudaError_t launch_dft_rows(const double2 *in, double2 *out, long narr, int L0, int L1, int sign,
                            double scale, cudaStream_t st, bool accumulate, const int *skip) {
  if (narr <= 0) return cudaSuccess;
  const int nk = L0 * L1;
  const size_t smem = dft_smem_bytes(L0, L1);
  cudaError_t pe = dft_prepare(L0, L1);
  if (pe != cudaSuccess) return pe;
  int threads = nk >= 256 ? 256 : ((nk + 31) / 32) * 32;
  const long cap = (long)device_sms() * 8;
  long blocks = narr < cap ? narr : cap;
  dft_rows_kernel<<<(unsigned)blocks, threads, smem, st>>>(in, out, narr, L0, L1, sign, scale,
                                                            accumulate ? 1 : 0, skip);
  return cudaGetLastError();
}

cudaError_t launch_sigma_products(const Mesh &m, const double *v, int n, double Un,
                                  const double *Ul_dev, const double2 *GR, double2 *SR,
                                  cudaStream_t st, const int *skip) {
  VMat vm;
  for (int i = 0; i < kMaxNb * kMaxNb; ++i) vm.v[i] = 0.0;
  for (int i = 0; i < m.nb * m.nb; ++i) vm.v[i] = v[i];
  switch (m.nb) {
    case 1: return products_nb<1>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 2: return products_nb<2>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 3: return products_nb<3>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 4: return products_nb<4>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 6: return products_nb<6>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 8: return products_nb<8>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 12: return products_nb<12>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 16: return products_nb<16>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    default: return cudaErrorInvalidValue;
  }
}

size_t sigma_workspace_bytes(const Mesh &m, int n) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  return 2 * (size_t)(n + 1) * 2 * blk * sizeof(double2);
}

cudaError_t sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                      const double2 *Grow, double2 *Sig, double2 *work, cudaStream_t st, const int *skip) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const long narr = (long)(n + 1) * 2 * m.nb * m.nb;
  double2 *GR = work;
  double2 *SR = work + (size_t)(n + 1) * 2 * blk;
  cudaError_t e = launch_dft_rows(Grow, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st, false, skip);
  if (e != cudaSuccess) return e;
  e = launch_sigma_products(m, v_host, n, Un, Ul_dev, GR, SR, st, skip);
  if (e != cudaSuccess) return e;
  return launch_dft_rows(SR, Sig, narr, m.L0, m.L1, -1, 1.0, st, false, skip);
}

}  // namespace kbe
