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
// A CTA transforms P arrays at a time (P n_k <= 512 points; grid-stride over
// the groups of arrays) in shared memory, so that each barrier of the
// transform covers P arrays' work. An axis whose length is a power of two is
// transformed in place by a radix-2 FFT (bit reversal, then log2 L butterfly
// stages; O(L log L)); other lengths use the direct sum over that axis
// (O(L^2)). The twiddle tables e^{sign 2 pi i m / L} are built once per CTA.
// C is the arithmetic type (double2, or float2 for the complex64 form).

__device__ __forceinline__ bool is_pow2(int L) { return L > 0 && (L & (L - 1)) == 0; }

// sequence q of an axis pass: groups of gsize sequences (one group per array,
// gstride apart), qstride apart within a group; element i at + i * stride
__device__ __forceinline__ int seq_base(int q, int gsize, int qstride, int gstride) {
  const int g = q / gsize;
  return g * gstride + (q - g * gsize) * qstride;
}

// in-place FFT of `count` sequences of length L; tw[m] = e^{sign 2 pi i m / L}
template <class C>
__device__ void fft_axis(C *x, int L, int stride, int count, int gsize, int qstride, int gstride, const C *tw) {
  int logL = 0;
  while ((1 << logL) < L) ++logL;
  const int total = count * L;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {   // bit reversal
    const int q = e / L, i = e - q * L;
    const int r = __brev(i) >> (32 - logL);
    if (logL > 0 && i < r) {
      C *p = x + seq_base(q, gsize, qstride, gstride);
      const C t = p[i * stride];
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
      C *p = x + seq_base(q, gsize, qstride, gstride);
      const int i = grp * len + pos, j = i + half;
      const C u = p[i * stride];
      const C t = c_mul(tw[pos * step], p[j * stride]);
      p[i * stride] = c_add(u, t);
      p[j * stride] = c_sub(u, t);
    }
    __syncthreads();
  }
}

// direct transform of `count` sequences of length L (x -> tmp -> x)
template <class C>
__device__ void dft_axis(C *x, C *tmp, int L, int stride, int count, int gsize, int qstride, int gstride,
                         const C *tw) {
  const int total = count * L;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e / L, R = e - q * L;
    const C *p = x + seq_base(q, gsize, qstride, gstride);
    C acc = c_scale(0, tw[0]);
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
    x[seq_base(q, gsize, qstride, gstride) + R * stride] = tmp[e];
  }
  __syncthreads();
}

__device__ __forceinline__ void store_as(double2 *p, double2 v) { *p = v; }
__device__ __forceinline__ void store_as(double2 *p, float2 v) { *p = make_double2(v.x, v.y); }
__device__ __forceinline__ void store_as(float2 *p, float2 v) { *p = v; }
__device__ __forceinline__ void add_as(double2 *p, double2 v) { *p = c_add(*p, v); }
__device__ __forceinline__ void add_as(double2 *p, float2 v) { *p = c_add(*p, make_double2(v.x, v.y)); }
__device__ __forceinline__ void add_as(float2 *p, float2 v) { *p = c_add(*p, v); }

// P arrays per CTA iteration (a power of two when n_k is one)
__host__ __device__ __forceinline__ int dft_group(int nk) {
  int P = 1;
  while (2 * P * nk <= 512) P *= 2;
  return P;
}

// Axes of at most kRegDft points, or of 16, are transformed one sequence per thread in
// registers: a CTA loads a group of PR arrays into shared memory (rows padded
// to L1 + 1 points, so that the row pass is close to conflict-free), each
// thread transforms whole rows, then whole columns, and the group is stored;
// three barriers per group instead of two per FFT stage. The butterflies and
// the direct sums are the shared-memory path's, in the same order, so both
// paths give the same bits.
constexpr int kRegDft = 12;   // and 16 (a power of two: radix-2 in registers)
__host__ __device__ __forceinline__ bool dft_axis_in_registers(int L) { return L <= kRegDft || L == 16; }
__host__ __device__ __forceinline__ bool dft_in_registers(int L0, int L1) {
  return dft_axis_in_registers(L0) && dft_axis_in_registers(L1);
}
__host__ __device__ __forceinline__ int dft_group_reg(int L0, int L1) {
  const int nk = L0 * L1, padded = L0 * (L1 + 1);
  const int a = 2048 / nk, b = 2560 / padded;
  const int P = a < b ? a : b;
  return P > 0 ? P : 1;
}

// one sequence of L points at p[i * stride], in place, in registers
template <class C, int L>
__device__ __forceinline__ void seq_transform(C *p, int stride, const C *tw) {
  C v[L];
  if constexpr ((L & (L - 1)) == 0) {
    constexpr int logL = L == 1 ? 0 : (L == 2 ? 1 : (L == 4 ? 2 : (L == 8 ? 3 : 4)));
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] = p[(logL ? (int)(__brev((unsigned)i) >> (32 - logL)) : 0) * stride];
#pragma unroll
    for (int len = 2; len <= L; len <<= 1) {
      const int half = len >> 1, step = L / len;
#pragma unroll
      for (int grp = 0; grp < L / len; ++grp)
#pragma unroll
        for (int pos = 0; pos < half; ++pos) {
          const int i = grp * len + pos, j = i + half;
          const C u = v[i];
          const C t = c_mul(tw[pos * step], v[j]);
          v[i] = c_add(u, t);
          v[j] = c_sub(u, t);
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i) p[i * stride] = v[i];
  } else {   // direct sum; every output is stored as it is formed (the inputs are all in v)
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] = p[i * stride];
#pragma unroll
    for (int R = 0; R < L; ++R) {
      C acc = c_scale(0, tw[0]);
#pragma unroll
      for (int kk = 0; kk < L; ++kk) acc = c_fma(tw[(R * kk) % L], v[kk], acc);
      p[R * stride] = acc;
    }
  }
}

template <class C>
__device__ __forceinline__ void seq_transform_any(int L, C *p, int stride, const C *tw) {
  switch (L) {
    case 2: seq_transform<C, 2>(p, stride, tw); break;
    case 3: seq_transform<C, 3>(p, stride, tw); break;
    case 4: seq_transform<C, 4>(p, stride, tw); break;
    case 5: seq_transform<C, 5>(p, stride, tw); break;
    case 6: seq_transform<C, 6>(p, stride, tw); break;
    case 7: seq_transform<C, 7>(p, stride, tw); break;
    case 8: seq_transform<C, 8>(p, stride, tw); break;
    case 9: seq_transform<C, 9>(p, stride, tw); break;
    case 10: seq_transform<C, 10>(p, stride, tw); break;
    case 11: seq_transform<C, 11>(p, stride, tw); break;
    case 12: seq_transform<C, 12>(p, stride, tw); break;
    case 16: seq_transform<C, 16>(p, stride, tw); break;
    default: break;   // L = 1: nothing to do
  }
}

__device__ __forceinline__ float2 load_as(const float2 &v, float2 *) { return v; }
__device__ __forceinline__ float2 load_as(const double2 &v, float2 *) {
  return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
__device__ __forceinline__ double2 load_as(const double2 &v, double2 *) { return v; }

// element e of array A of the input; pair_nb2 > 0: the input is a row of
// (G^<, dG) pairs (arrays [l][x][a b], x = 1 holding dG = G^< - G^>), read as
// (G^<, G^> = G^< - dG)
template <class C, class Tin>
__device__ __forceinline__ C load_in(const Tin *__restrict__ src, long e, long A, long nk, int pair_nb2) {
  const C v = load_as(src[e], (C *)nullptr);
  if (pair_nb2 > 0 && (A / pair_nb2) % 2 == 1) return c_sub(load_as(src[e - (long)pair_nb2 * nk], (C *)nullptr), v);
  return v;
}

template <class C, class Tin, class Tout>
__global__ void dft_rows_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, long narr, int L0, int L1,
                                int sign, double scale, int accumulate, const int *__restrict__ skip,
                                int pair_nb2) {
  if (skip && *skip) return;
  extern __shared__ double2 sm_d2[];
  C *sm = reinterpret_cast<C *>(sm_d2);
  const int nk = L0 * L1;
  const bool reg = dft_in_registers(L0, L1);
  const int P = reg ? dft_group_reg(L0, L1) : dft_group(nk);
  const int W = reg ? L1 + 1 : L1;   // row pitch in shared memory (points)
  C *x = sm;
  C *t = x + (size_t)P * L0 * W;
  C *tw0 = reg ? t : t + P * nk;
  C *tw1 = tw0 + L0;
  for (int i = threadIdx.x; i < L0; i += blockDim.x) {
    double s, c;
    sincospi(2.0 * i / L0, &s, &c);
    tw0[i] = c_from<C>(make_double2(c, sign * s));
  }
  for (int i = threadIdx.x; i < L1; i += blockDim.x) {
    double s, c;
    sincospi(2.0 * i / L1, &s, &c);
    tw1[i] = c_from<C>(make_double2(c, sign * s));
  }
  const C sc = c_from<C>(make_double2(scale, 0.0));
  const long ngroups = (narr + P - 1) / P;
  for (long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long arr0 = grp * P;
    const int pa = (int)(narr - arr0 < P ? narr - arr0 : P);   // arrays in this group
    const Tin *src = in + arr0 * nk;
    Tout *dst = out + arr0 * nk;
    __syncthreads();
    if (reg) {
      for (int e = threadIdx.x; e < pa * nk; e += blockDim.x) {
        const int row = e / L1;   // (array, k0)
        x[row * W + (e - row * L1)] = load_in<C>(src, e, arr0 + e / nk, nk, pair_nb2);
      }
      __syncthreads();
      if (L1 > 1)   // axis 1: rows (array, k0), contiguous
        for (int q = threadIdx.x; q < pa * L0; q += blockDim.x) seq_transform_any<C>(L1, x + q * W, 1, tw1);
      __syncthreads();
      if (L0 > 1)   // axis 0: columns (array, k1), pitch W
        for (int q = threadIdx.x; q < pa * L1; q += blockDim.x) {
          const int arr = q / L1, k1 = q - arr * L1;
          seq_transform_any<C>(L0, x + arr * L0 * W + k1, W, tw0);
        }
      __syncthreads();
      for (int e = threadIdx.x; e < pa * nk; e += blockDim.x) {
        const int row = e / L1;
        const C v = c_mul(sc, x[row * W + (e - row * L1)]);
        if (accumulate) add_as(dst + e, v);
        else store_as(dst + e, v);
      }
      continue;
    }
    for (int e = threadIdx.x; e < pa * nk; e += blockDim.x) x[e] = load_in<C>(src, e, arr0 + e / nk, nk, pair_nb2);
    __syncthreads();
    if (L1 > 1) {   // axis 1: L0 contiguous sequences of length L1 per array
      if (is_pow2(L1)) fft_axis<C>(x, L1, 1, pa * L0, L0, L1, nk, tw1);
      else dft_axis<C>(x, t, L1, 1, pa * L0, L0, L1, nk, tw1);
    }
    if (L0 > 1) {   // axis 0: L1 sequences of length L0, stride L1, per array
      if (is_pow2(L0)) fft_axis<C>(x, L0, L1, pa * L1, L1, 1, nk, tw0);
      else dft_axis<C>(x, t, L0, L1, pa * L1, L1, 1, nk, tw0);
    }
    if (accumulate)
      for (int e = threadIdx.x; e < pa * nk; e += blockDim.x) add_as(dst + e, c_mul(sc, x[e]));
    else
      for (int e = threadIdx.x; e < pa * nk; e += blockDim.x) store_as(dst + e, c_mul(sc, x[e]));
  }
}

struct VMat {
  double v[kMaxNb * kMaxNb];
};

template <class C>
struct RealOf;
template <>
struct RealOf<double2> {
  using T = double;
};
template <>
struct RealOf<float2> {
  using T = float;
};

// Real-space second-Born products for one (l, j, R): all m, both components.
template <class C, int NB>
__global__ void __launch_bounds__(128) sigma_products_kernel(const C *__restrict__ GR, C *__restrict__ SR, int n,
                                                             int nk, double Un, const double *__restrict__ Ul,
                                                             VMat vm, const int *__restrict__ skip) {
  using R = typename RealOf<C>::T;
  if (skip && *skip) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)(n + 1) * NB * nk;
  if (idx >= total) return;
  const int Rp = (int)(idx % nk);
  const long t = idx / nk;
  const int j = (int)(t % NB);
  const int l = (int)(t / NB);
  const size_t blk = (size_t)NB * NB * nk;
  const C *gl = GR + (size_t)l * 2 * blk + Rp;
  const C *gg = gl + blk;
  const R fac = (R)(-Un * (Ul ? Ul[l] : Un));
  const C zero = c_from<C>(make_double2(0.0, 0.0));
  C *sl = SR + (size_t)l * 2 * blk + (size_t)j * NB * nk + Rp;
  C *sg = sl + blk;
#pragma unroll 1
  for (int m = 0; m < NB; ++m) {
    C QL = zero, QG = zero, EL = zero, EG = zero;
#pragma unroll 1
    for (int a = 0; a < NB; ++a) {
      const R vja = (R)vm.v[j * NB + a];
      if (vja == (R)0) continue;
      C zl = zero, yl = zero, yg = zero;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const R vmb = (R)vm.v[m * NB + b];
        if (vmb == (R)0) continue;
        const C gl_ab = gl[(size_t)(a * NB + b) * nk];
        const C gg_ab = gg[(size_t)(a * NB + b) * nk];
        const C gl_jb = gl[(size_t)(j * NB + b) * nk];
        const C gg_jb = gg[(size_t)(j * NB + b) * nk];
        zl = c_add(zl, c_scale(vmb, c_mulc(gl_ab, gg_ab)));   // M_ab = G^<_ab conj(G^>_ab)
        yl = c_add(yl, c_scale(vmb, c_mulc(gl_jb, gg_ab)));   // G^<_jb conj(G^>_ab)
        yg = c_add(yg, c_scale(vmb, c_mulc(gg_jb, gl_ab)));   // G^>_jb conj(G^<_ab)
      }
      QL = c_add(QL, c_scale(vja, zl));
      QG = c_add(QG, c_scale(vja, c_conj(zl)));              // M^>_ab = conj(M^<_ab)
      EL = c_fma(c_scale(vja, gl[(size_t)(a * NB + m) * nk]), yl, EL);
      EG = c_fma(c_scale(vja, gg[(size_t)(a * NB + m) * nk]), yg, EG);
    }
    const C gl_jm = gl[(size_t)(j * NB + m) * nk];
    const C gg_jm = gg[(size_t)(j * NB + m) * nk];
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
template <class C, int NB>
__global__ void __launch_bounds__(128) sigma_products_pair_kernel(const C *__restrict__ GR, C *__restrict__ SR,
                                                                  int n, int nk, double Un,
                                                                  const double *__restrict__ Ul,
                                                                  const int *__restrict__ skip) {
  using R = typename RealOf<C>::T;
  if (skip && *skip) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)(n + 1) * NB * nk;
  if (idx >= total) return;
  const int Rp = (int)(idx % nk);
  const long t = idx / nk;
  const int j = (int)(t % NB);
  const int l = (int)(t / NB);
  const size_t blk = (size_t)NB * NB * nk;
  const C *gl = GR + (size_t)l * 2 * blk + Rp;
  const C *gg = gl + blk;
  const R fac = (R)(-Un * (Ul ? Ul[l] : Un));
  const C zero = c_from<C>(make_double2(0.0, 0.0));
#define AT(M, r, c) M[(size_t)((r) * NB + (c)) * nk]
  C tr = zero;        // tr(G^< G^>^+) = sum_ab G^<_ab conj(G^>_ab)
  C Tl[NB], Tg[NB];   // row j of T = G^< G^>^+ and of T^+ = G^> G^<^+
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    C sl = zero, sg = zero;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const C xab = AT(gl, a, b), yab = AT(gg, a, b);
      tr = c_add(tr, c_mulc(xab, yab));
      sl = c_add(sl, c_mulc(AT(gl, j, b), yab));
      sg = c_add(sg, c_mulc(AT(gg, j, b), xab));
    }
    Tl[a] = sl;
    Tg[a] = sg;
  }
  C *sl = SR + (size_t)l * 2 * blk + (size_t)j * NB * nk + Rp;
  C *sg = sl + blk;
#pragma unroll 1
  for (int m = 0; m < NB; ++m) {
    C pl = zero, pg = zero;
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

template <class C, int NB>
cudaError_t products_nb(const Mesh &m, const VMat &vm, int n, double Un, const double *Ul, const C *GR, C *SR,
                        cudaStream_t st, const int *skip) {
  bool pair = NB >= 3;   // v = 1 - delta exactly (at N_b <= 2 the two forms time the same)
  for (int a = 0; a < NB; ++a)
    for (int b = 0; b < NB; ++b) pair = pair && vm.v[a * NB + b] == (a == b ? 0.0 : 1.0);
  const long total = (long)(n + 1) * NB * m.nk;
  const unsigned blocks = (unsigned)((total + 127) / 128);
  if (pair)
    sigma_products_pair_kernel<C, NB><<<blocks, 128, 0, st>>>(GR, SR, n, m.nk, Un, Ul, skip);
  else
    sigma_products_kernel<C, NB><<<blocks, 128, 0, st>>>(GR, SR, n, m.nk, Un, Ul, vm, skip);
  return cudaGetLastError();
}

template <class C>
cudaError_t products_any(const Mesh &m, const double *v, int n, double Un, const double *Ul_dev, const C *GR, C *SR,
                         cudaStream_t st, const int *skip) {
  VMat vm;
  for (int i = 0; i < kMaxNb * kMaxNb; ++i) vm.v[i] = 0.0;
  for (int i = 0; i < m.nb * m.nb; ++i) vm.v[i] = v[i];
  switch (m.nb) {
    case 1: return products_nb<C, 1>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 2: return products_nb<C, 2>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 3: return products_nb<C, 3>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 4: return products_nb<C, 4>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 6: return products_nb<C, 6>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 8: return products_nb<C, 8>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 12: return products_nb<C, 12>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    case 16: return products_nb<C, 16>(m, vm, n, Un, Ul_dev, GR, SR, st, skip);
    default: return cudaErrorInvalidValue;
  }
}

size_t dft_smem_bytes(int L0, int L1, size_t csize) {
  const int nk = L0 * L1;
  if (dft_in_registers(L0, L1)) return csize * ((size_t)dft_group_reg(L0, L1) * L0 * (L1 + 1) + L0 + L1);
  return csize * (2 * (size_t)dft_group(nk) * nk + L0 + L1);
}

template <class C, class Tin, class Tout>
cudaError_t dft_prepare_t(int L0, int L1) {
  constexpr size_t kDefault = 48 * 1024;   // no opt-in needed below this
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static size_t raised[kMaxDev] = {};
  const size_t smem = dft_smem_bytes(L0, L1, sizeof(C));
  if (smem <= kDefault) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (smem > raised[dev]) {
    e = cudaFuncSetAttribute(dft_rows_kernel<C, Tin, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    raised[dev] = smem;
  }
  return cudaSuccess;
}

template <class C, class Tin, class Tout>
cudaError_t dft_launch(const Tin *in, Tout *out, long narr, int L0, int L1, int sign, double scale, cudaStream_t st,
                       bool accumulate, const int *skip, int pair_nb2 = 0) {
  if (narr <= 0) return cudaSuccess;
  const int nk = L0 * L1;
  const bool reg = dft_in_registers(L0, L1);
  const int P = reg ? dft_group_reg(L0, L1) : dft_group(nk);
  cudaError_t pe = dft_prepare_t<C, Tin, Tout>(L0, L1);
  if (pe != cudaSuccess) return pe;
  const int pts = reg ? P * (L0 > L1 ? L0 : L1) : P * nk;   // the register path: sequences per pass
  const int threads = pts >= 256 ? 256 : ((pts + 31) / 32) * 32;
  const long groups = (narr + P - 1) / P, cap = (long)device_sms() * 8;
  const long blocks = groups < cap ? groups : cap;
  dft_rows_kernel<C, Tin, Tout><<<(unsigned)blocks, threads, dft_smem_bytes(L0, L1, sizeof(C)), st>>>(
      in, out, narr, L0, L1, sign, scale, accumulate ? 1 : 0, skip, pair_nb2);
  return cudaGetLastError();
}

}  // namespace

// raise the DFT kernels' dynamic shared-memory limits for this mesh (host-side
// attributes of the current device's context, done before any stream capture
// that launches them); the raised limits are kept per device, under a lock
cudaError_t dft_prepare(int L0, int L1) {
  cudaError_t e = dft_prepare_t<double2, double2, double2>(L0, L1);
  if (e == cudaSuccess) e = dft_prepare_t<float2, double2, float2>(L0, L1);
  if (e == cudaSuccess) e = dft_prepare_t<float2, float2, double2>(L0, L1);
  if (e == cudaSuccess) e = dft_prepare_t<float2, float2, float2>(L0, L1);
  return e;
}

cudaError_t launch_dft_rows(const double2 *in, double2 *out, long narr, int L0, int L1, int sign,
                            double scale, cudaStream_t st, bool accumulate, const int *skip) {
  return dft_launch<double2, double2, double2>(in, out, narr, L0, L1, sign, scale, st, accumulate, skip);
}

cudaError_t launch_sigma_products(const Mesh &m, const double *v, int n, double Un,
                                  const double *Ul_dev, const double2 *GR, double2 *SR,
                                  cudaStream_t st, const int *skip) {
  return products_any<double2>(m, v, n, Un, Ul_dev, GR, SR, st, skip);
}

size_t sigma_workspace_bytes(const Mesh &m, int n) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  return 2 * (size_t)(n + 1) * 2 * blk * sizeof(double2);
}

cudaError_t sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                      const double2 *Grow, double2 *Sig, double2 *work, cudaStream_t st, const int *skip,
                      bool fp32, const float2 *Hrow32, bool sig32) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const long narr = (long)(n + 1) * 2 * m.nb * m.nb;
  if (fp32) {   // complex64 transforms and products (half the workspace)
    float2 *GR = (float2 *)work;
    float2 *SR = GR + (size_t)(n + 1) * 2 * blk;
    cudaError_t e = Hrow32 ? dft_launch<float2, float2, float2>(Hrow32, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st,
                                                                false, skip, m.nb * m.nb)
                           : dft_launch<float2, double2, float2>(Grow, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st,
                                                                 false, skip);
    if (e != cudaSuccess) return e;
    e = products_any<float2>(m, v_host, n, Un, Ul_dev, GR, SR, st, skip);
    if (e != cudaSuccess) return e;
    if (sig32) return dft_launch<float2, float2, float2>(SR, (float2 *)Sig, narr, m.L0, m.L1, -1, 1.0, st, false, skip);
    return dft_launch<float2, float2, double2>(SR, Sig, narr, m.L0, m.L1, -1, 1.0, st, false, skip);
  }
  double2 *GR = work;
  double2 *SR = work + (size_t)(n + 1) * 2 * blk;
  cudaError_t e = launch_dft_rows(Grow, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st, false, skip);
  if (e != cudaSuccess) return e;
  e = launch_sigma_products(m, v_host, n, Un, Ul_dev, GR, SR, st, skip);
  if (e != cudaSuccess) return e;
  return launch_dft_rows(SR, Sig, narr, m.L0, m.L1, -1, 1.0, st, false, skip);
}

}  // namespace kbe
