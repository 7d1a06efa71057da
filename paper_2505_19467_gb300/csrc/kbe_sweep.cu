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
// FP64 pipe is ~1.2 TFLOP/s against ~7 TB/s of HBM, and the FP32 pipe ~61x
// the FP64 one). Three arithmetic forms share one thread mapping -- every
// thread owns one (k, a) output row of both components and streams the l
// sum; the N_b threads sharing a k read the same block through L1:
//   FP64 : complex128 history, DFMA.
//   DF64 : history as FP32 (hi, lo) pairs; each real product x*y is split
//          exactly (p = fl(xh*yh), e = fma(xh, yh, -p) + xh*yl + xl*yh) and
//          accumulated with an error-free TwoSum into a (hi, lo) pair:
//          ~2^-44 relative accuracy at FP32-pipe speed.
//   C64  : complex64 history, FP32 partial products per l, partial sums
//          added into a compensated (TwoSum) accumulator.
// For DF64 / C64 the Sigma row is first turned into three coefficient rows
// C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<, C2^> = dt S^> in the history's
// storage; the term-2 weights w^(j)_l / dt are then exact powers of two.
#include "kbe_internal.cuh"

namespace kbe {

namespace {

// ---------------------------------------------------------------- FP64 ----
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

// ---------------------------------------------------------------- DF64 ----
// A complex double-float is float4 {re_hi, re_lo, im_hi, im_lo}. The explicit
// _rn intrinsics keep the compiler from contracting the error-free
// transformations into FMAs.

// (ah, al) += (xh + xl) * (yh + yl), dropping xl * yl (2^-48 relative)
__device__ __forceinline__ void df_mac(float &ah, float &al, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float pe = __fmaf_rn(xh, yh, -p);
  pe = __fmaf_rn(xh, yl, pe);
  pe = __fmaf_rn(xl, yh, pe);
  const float s = __fadd_rn(ah, p);
  const float bb = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, pe));
}

// acc += X * Y (complex double-float)
__device__ __forceinline__ void cdf_mac(float4 &acc, const float4 &X, const float4 &Y) {
  df_mac(acc.x, acc.y, X.x, X.y, Y.x, Y.y);
  df_mac(acc.x, acc.y, -X.z, -X.w, Y.z, Y.w);
  df_mac(acc.z, acc.w, X.x, X.y, Y.z, Y.w);
  df_mac(acc.z, acc.w, X.z, X.w, Y.x, Y.y);
}

// (sh, sl) = (ah + al) - (bh + bl), renormalised with TwoSum
__device__ __forceinline__ void df_sub(float &sh, float &sl, float ah, float al, float bh, float bl) {
  const float s = __fsub_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
  e = __fadd_rn(e, __fsub_rn(al, bl));
  const float t = __fadd_rn(s, e);
  const float tb = __fsub_rn(t, s);
  sl = __fadd_rn(__fsub_rn(s, __fsub_rn(t, tb)), __fsub_rn(e, tb));
  sh = t;
}

__device__ __forceinline__ float4 cdf_sub(const float4 &A, const float4 &B) {
  float4 r;
  df_sub(r.x, r.y, A.x, A.y, B.x, B.y);
  df_sub(r.z, r.w, A.z, A.w, B.z, B.w);
  return r;
}

__device__ __forceinline__ float4 cdf_negconj(const float4 &A) {
  return make_float4(-A.x, -A.y, A.z, A.w);
}

__device__ __forceinline__ float4 cdf_scale2(float f, const float4 &A) {   // f a power of two
  return make_float4(f * A.x, f * A.y, f * A.z, f * A.w);
}

__device__ __forceinline__ double2 cdf_to_double(const float4 &A) {
  return make_double2((double)A.x + (double)A.y, (double)A.z + (double)A.w);
}

// term-2 weight w^(j)_l / dt: 0 above the diagonal or for j = 0, 1/2 at the
// trapezoid ends, 1 inside
__device__ __forceinline__ float term2_factor(int j, int l) {
  if (j == 0 || l > j) return 0.f;
  return (l == 0 || l == j) ? 0.5f : 1.f;
}

template <int NB>
__global__ void __launch_bounds__(128) sweep_df64_kernel(const float4 *__restrict__ H,
                                                         const float4 *__restrict__ Cf,
                                                         double2 *__restrict__ Iout, int n,
                                                         int nk) {
  const int j = blockIdx.x;
  const int idx = blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= NB * nk) return;
  const int a = idx / nk;
  const int k = idx - a * nk;
  const size_t blk = (size_t)NB * NB * nk;

  float4 accL[NB], accG[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) accL[b] = accG[b] = make_float4(0.f, 0.f, 0.f, 0.f);

  for (int l = 0; l <= n; ++l) {
    const float4 *c1 = Cf + (size_t)l * 3 * blk + (size_t)a * NB * nk + k;
    const float4 *c2l = c1 + blk;
    const float4 *c2g = c1 + 2 * blk;
    const float f = term2_factor(j, l);
    const bool lower = (l >= j);
    const float4 *gl = H + (lower ? tri(l, j) : tri(j, l)) * 2 * blk + k;
    const float4 *gg = gl + blk;
#pragma unroll 1
    for (int c = 0; c < NB; ++c) {
      const float4 A1 = c1[(size_t)c * nk];
      float4 B2l = make_float4(0.f, 0.f, 0.f, 0.f), B2g = B2l;
      if (f != 0.f) {
        B2l = cdf_scale2(f, c2l[(size_t)c * nk]);
        B2g = cdf_scale2(f, c2g[(size_t)c * nk]);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float4 Gl, Gg;
        if (lower) {
          Gl = gl[(size_t)(c * NB + b) * nk];
          Gg = gg[(size_t)(c * NB + b) * nk];
        } else {
          Gl = cdf_negconj(gl[(size_t)(b * NB + c) * nk]);
          Gg = cdf_negconj(gg[(size_t)(b * NB + c) * nk]);
        }
        cdf_mac(accL[b], A1, Gl);
        cdf_mac(accG[b], A1, Gg);
        if (f != 0.f) {
          const float4 D = cdf_sub(Gl, Gg);
          cdf_mac(accL[b], B2l, D);
          cdf_mac(accG[b], B2g, D);
        }
      }
    }
  }
  double2 *il = Iout + (size_t)j * 2 * blk + (size_t)a * NB * nk + k;
  double2 *ig = il + blk;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    il[(size_t)b * nk] = cdf_to_double(accL[b]);
    ig[(size_t)b * nk] = cdf_to_double(accG[b]);
  }
}

// ----------------------------------------------------------------- C64 ----
__device__ __forceinline__ float2 cf_fma(float2 a, float2 b, float2 acc) {
  return make_float2(__fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, acc.x)),
                     __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, acc.y)));
}

// (h, c) += p with an error-free TwoSum; c collects the rounding errors
__device__ __forceinline__ void comp_add(float &h, float &c, float p) {
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  c = __fadd_rn(c, e);
}

template <int NB>
__global__ void __launch_bounds__(128) sweep_c64_kernel(const float2 *__restrict__ H,
                                                        const float2 *__restrict__ Cf,
                                                        double2 *__restrict__ Iout, int n,
                                                        int nk) {
  const int j = blockIdx.x;
  const int idx = blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= NB * nk) return;
  const int a = idx / nk;
  const int k = idx - a * nk;
  const size_t blk = (size_t)NB * NB * nk;

  float4 accL[NB], accG[NB];   // {re, re_comp, im, im_comp}
#pragma unroll
  for (int b = 0; b < NB; ++b) accL[b] = accG[b] = make_float4(0.f, 0.f, 0.f, 0.f);

  for (int l = 0; l <= n; ++l) {
    const float2 *c1 = Cf + (size_t)l * 3 * blk + (size_t)a * NB * nk + k;
    const float2 *c2l = c1 + blk;
    const float2 *c2g = c1 + 2 * blk;
    const float f = term2_factor(j, l);
    const bool lower = (l >= j);
    const float2 *gl = H + (lower ? tri(l, j) : tri(j, l)) * 2 * blk + k;
    const float2 *gg = gl + blk;
    float2 pL[NB], pG[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) pL[b] = pG[b] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int c = 0; c < NB; ++c) {
      const float2 A1 = c1[(size_t)c * nk];
      float2 B2l = make_float2(0.f, 0.f), B2g = B2l;
      if (f != 0.f) {
        const float2 u = c2l[(size_t)c * nk], w = c2g[(size_t)c * nk];
        B2l = make_float2(f * u.x, f * u.y);
        B2g = make_float2(f * w.x, f * w.y);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float2 Gl, Gg;
        if (lower) {
          Gl = gl[(size_t)(c * NB + b) * nk];
          Gg = gg[(size_t)(c * NB + b) * nk];
        } else {
          const float2 u = gl[(size_t)(b * NB + c) * nk], w = gg[(size_t)(b * NB + c) * nk];
          Gl = make_float2(-u.x, u.y);
          Gg = make_float2(-w.x, w.y);
        }
        pL[b] = cf_fma(A1, Gl, pL[b]);
        pG[b] = cf_fma(A1, Gg, pG[b]);
        if (f != 0.f) {
          const float2 D = make_float2(Gl.x - Gg.x, Gl.y - Gg.y);
          pL[b] = cf_fma(B2l, D, pL[b]);
          pG[b] = cf_fma(B2g, D, pG[b]);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      comp_add(accL[b].x, accL[b].y, pL[b].x);
      comp_add(accL[b].z, accL[b].w, pL[b].y);
      comp_add(accG[b].x, accG[b].y, pG[b].x);
      comp_add(accG[b].z, accG[b].w, pG[b].y);
    }
  }
  double2 *il = Iout + (size_t)j * 2 * blk + (size_t)a * NB * nk + k;
  double2 *ig = il + blk;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    il[(size_t)b * nk] = cdf_to_double(accL[b]);
    ig[(size_t)b * nk] = cdf_to_double(accG[b]);
  }
}

// --------------------------------------------------- packing and coefficients
__device__ __forceinline__ float4 split_df(double2 x) {
  const float rh = __double2float_rn(x.x), ih = __double2float_rn(x.y);
  return make_float4(rh, __double2float_rn(x.x - (double)rh), ih, __double2float_rn(x.y - (double)ih));
}

__global__ void pack_kernel(int prec, const double2 *__restrict__ src, void *__restrict__ dst,
                            size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const double2 x = src[i];
    if (prec == KBE_PREC_DF64) ((float4 *)dst)[i] = split_df(x);
    else if (prec == KBE_PREC_C64) ((float2 *)dst)[i] = make_float2((float)x.x, (float)x.y);
    else ((double2 *)dst)[i] = x;
  }
}

// coefficient rows [l][3][a][c][k]: C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<, C2^> = dt S^>
__global__ void coef_kernel(int prec, const double2 *__restrict__ Sig, void *__restrict__ Cf, int n,
                            int nk, int nb2, double dt) {
  const size_t blk = (size_t)nb2 * nk;
  const size_t total = (size_t)(n + 1) * blk;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t l = i / blk, r = i - l * blk;
    const double2 sl = Sig[(l * 2) * blk + r], sg = Sig[(l * 2 + 1) * blk + r];
    const double w1 = trap_weight(n, (int)l, dt);
    const double2 v[3] = {c_scale(w1, c_sub(sg, sl)), c_scale(dt, sl), c_scale(dt, sg)};
    for (int q = 0; q < 3; ++q) {
      const size_t o = (l * 3 + q) * blk + r;
      if (prec == KBE_PREC_DF64) ((float4 *)Cf)[o] = split_df(v[q]);
      else ((float2 *)Cf)[o] = make_float2((float)v[q].x, (float)v[q].y);
    }
  }
}

template <int NB>
cudaError_t sweep_nb(const Mesh &m, int n, double dt, int prec, const void *H, const double2 *Sig,
                     const void *Cf, double2 *I, cudaStream_t st) {
  const int threads = 128;
  dim3 grid(n + 1, (NB * m.nk + threads - 1) / threads);
  if (prec == KBE_PREC_FP64)
    sweep_f64_kernel<NB><<<grid, threads, 0, st>>>((const double2 *)H, Sig, I, n, m.nk, dt);
  else if (prec == KBE_PREC_DF64)
    sweep_df64_kernel<NB><<<grid, threads, 0, st>>>((const float4 *)H, (const float4 *)Cf, I, n, m.nk);
  else
    sweep_c64_kernel<NB><<<grid, threads, 0, st>>>((const float2 *)H, (const float2 *)Cf, I, n, m.nk);
  return cudaGetLastError();
}

unsigned grid_for(size_t count) {
  size_t b = (count + 255) / 256;
  return (unsigned)(b < 152 * 64 ? (b ? b : 1) : 152 * 64);
}

}  // namespace

bool sweep_supported(int nb) {
  switch (nb) {
    case 1: case 2: case 3: case 4: case 6: case 8: case 12: case 16: return true;
    default: return false;
  }
}

bool precision_supported(int prec) {
  return prec == KBE_PREC_FP64 || prec == KBE_PREC_DF64 || prec == KBE_PREC_C64;
}

size_t history_elem_bytes(int prec) { return prec == KBE_PREC_C64 ? sizeof(float2) : 16; }

size_t sweep_workspace_bytes(const Mesh &m, int n, int prec) {
  if (prec == KBE_PREC_FP64) return 0;
  return (size_t)(n + 1) * 3 * m.nb * m.nb * m.nk * history_elem_bytes(prec);
}

cudaError_t launch_pack(int prec, const double2 *src, void *dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  pack_kernel<<<grid_for(count), 256, 0, st>>>(prec, src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const Mesh &m, int n, double dt, int precision, const void *H,
                         const double2 *Sig, double2 *I, void *work, cudaStream_t st) {
  if (!precision_supported(precision)) return cudaErrorInvalidValue;
  if (precision != KBE_PREC_FP64) {
    const size_t total = (size_t)(n + 1) * m.nb * m.nb * m.nk;
    coef_kernel<<<grid_for(total), 256, 0, st>>>(precision, Sig, work, n, m.nk, m.nb * m.nb, dt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  switch (m.nb) {
    case 1: return sweep_nb<1>(m, n, dt, precision, H, Sig, work, I, st);
    case 2: return sweep_nb<2>(m, n, dt, precision, H, Sig, work, I, st);
    case 3: return sweep_nb<3>(m, n, dt, precision, H, Sig, work, I, st);
    case 4: return sweep_nb<4>(m, n, dt, precision, H, Sig, work, I, st);
    case 6: return sweep_nb<6>(m, n, dt, precision, H, Sig, work, I, st);
    case 8: return sweep_nb<8>(m, n, dt, precision, H, Sig, work, I, st);
    case 12: return sweep_nb<12>(m, n, dt, precision, H, Sig, work, I, st);
    case 16: return sweep_nb<16>(m, n, dt, precision, H, Sig, work, I, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kbe
