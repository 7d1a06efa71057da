// (a2) Collision integrals on the new time row (Eq. 6 of the paper, read in
// the left Sigma * G form, trapezoid quadrature):
//   I^x(n,j) = sum_{l=0}^{n} w^(n)_l [S^>(n,l) - S^<(n,l)] G^x(l,j)
//            + sum_{l=0}^{j} w^(j)_l  S^x(n,l) [G^<(l,j) - G^>(l,j)]
// for j = 0..n and x in {<, >}. The history holds G only for l >= j; above
// the diagonal G(l,j) = -G(j,l)^+ (the paper keeps G^> below and G^< above
// the diagonal for the same reason). It stores, per block, G^< and
// dG = G^< - G^> (so that G^> never has to be formed). With
// C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<, C3 = dt S^> - C1 and f = w^(j)_l / dt
// the kernels accumulate X = I^< and Y = I^> - I^<:
//   X(n,j) = sum_l C1 G^<(l,j) + sum_{l<=j} f C2^< dG(l,j),
//   Y(n,j) = sum_{l<=j} (w^(j)_l - w^(n)_l) (S^> - S^<) dG(l,j) - sum_{l>j} C1 dG(l,j).
// Both quadratures give every interior node of [0, t_j] the weight dt, so Y
// takes only the nodes above the output and the few end nodes where the
// weights differ (there its coefficient is f (C3 - C2^<) + (f - 1) C1): two
// complex multiply-adds per element and node, three at the end nodes.
//
// Work per evaluation: ~2 N_b^3 complex multiply-adds per stored block, k and
// use (each block serves one column j as stored and one as an adjoint), i.e.
// ~16 n^2 N_b^3 n_k flops for n^2 N_b^2 n_k complex numbers read: about
// N_b flop per byte in FP64, far right of the FP64 ridge on GB300 (the
// FP64 pipe is ~1.2 TFLOP/s against ~7 TB/s of HBM, and the FP32 pipe ~61x
// the FP64 one). Three arithmetic forms share one kernel template: every
// thread owns one output element (k, a, b) of both components and streams
// the l sum (threads sharing k and b read the same block column through L1);
// when the grid would be too small to fill the GPU, the l range is split over
// several CTAs and the partial sums are reduced in FP64 by a second kernel:
//   FP64 : complex128 history, DFMA.
//   DF64 : history as FP32 (hi, lo) pairs; each real product x*y is split
//          exactly (p = fl(xh*yh), e = fma(xh, yh, -p) + xh*yl + xl*yh) and
//          accumulated with an error-free TwoSum into a (hi, lo) pair:
//          ~2^-44 relative accuracy at FP32-pipe speed.
//   C64  : complex64 history, FP32 partial sums over a group of nodes,
//          folded into a compensated (TwoSum) accumulator.
// The Sigma row is first turned into the three coefficient rows C1, C2^<, C3
// in the history's storage; the trapezoid's term-2 weights f are then exact
// powers of two (f = 1 inside, 1/2 at l = 0 and l = j).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kbe_internal.cuh"
#include "kbe_tma.cuh"

#ifndef KBE_SWEEP_MINB_F64
#define KBE_SWEEP_MINB_F64 2
#endif
#ifndef KBE_SWEEP_MINB_DF64
#define KBE_SWEEP_MINB_DF64 3
#endif
#ifndef KBE_SWEEP_MINB_C64
#define KBE_SWEEP_MINB_C64 2
#endif
#ifndef KBE_SWEEP_MINB_C64X2
#define KBE_SWEEP_MINB_C64X2 3   // picked by timing (pairs at 2 / 3 CTAs, single k at 2 / 4)
#endif
#ifndef KBE_SWEEP_C64_PAIRS
#define KBE_SWEEP_C64_PAIRS 1   // C64: two consecutive k per thread when n_k is even
#endif

namespace kbe {

namespace {

// ---------------------------------------------------------------- FP64 ----
// Every arithmetic form below provides, besides the complex operations, V (the
// complex values of consecutive k one stored element S carries) and store()
// (the I^< and I^> outputs of this thread; blkc = the component stride in
// complex numbers).
struct ArithF64 {
  using S = double2;   // stored complex
  using A = double2;   // accumulator
  static constexpr int V = 1;
  static constexpr bool kGrouped = false;   // end() after every node (no-op here)
  static constexpr int kUnrollSmallNb = 1;   // nodes per loop iteration at N_b <= 4
  static constexpr int kMinBlocks = KBE_SWEEP_MINB_F64;   // CTAs of 256 per SM (register cap)
  static __device__ __forceinline__ void zero(A &a) { a = make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void begin(A &) {}
  static __device__ __forceinline__ void end(A &) {}
  static __device__ __forceinline__ void mac(A &a, const S &x, const S &y) { a = c_fma(x, y, a); }
  static __device__ __forceinline__ S sub(const S &x, const S &y) { return c_sub(x, y); }
  static __device__ __forceinline__ S negconj(const S &x) { return make_double2(-x.x, x.y); }
  static __device__ __forceinline__ S neg(const S &x) { return make_double2(-x.x, -x.y); }
  static __device__ __forceinline__ S scale(float f, const S &x) { return c_scale((double)f, x); }
  static __device__ __forceinline__ S scale_w(double f, const S &x) { return c_scale(f, x); }
  static __device__ __forceinline__ S add(const S &x, const S &y) { return c_add(x, y); }
  static __device__ __forceinline__ void store(double2 *o, size_t blkc, const A &x, const A &y) {
    o[0] = x;
    o[blkc] = c_add(x, y);
  }
};

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

// (rh, rl) = (xh + xl) * f for a double weight f (split into two floats):
// the exact product of the high parts plus the cross terms, renormalised
__device__ __forceinline__ void df_mul_w(float &rh, float &rl, float xh, float xl, double f) {
  const float fh = __double2float_rn(f), fl = __double2float_rn(f - (double)fh);
  const float p = __fmul_rn(xh, fh);
  float e = __fmaf_rn(xh, fh, -p);
  e = __fmaf_rn(xh, fl, e);
  e = __fmaf_rn(xl, fh, e);
  const float s = __fadd_rn(p, e);
  rl = __fsub_rn(e, __fsub_rn(s, p));
  rh = s;
}

// (h, l) <- TwoSum(h, l): renormalise so that |l| <= ulp(h) / 2
__device__ __forceinline__ void df_renorm(float &h, float &l) {
  const float s = __fadd_rn(h, l);
  const float bb = __fsub_rn(s, h);
  l = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb));
  h = s;
}

struct ArithDF64 {
  using S = float4;
  using A = float4;
  static constexpr int V = 1;
  static constexpr bool kGrouped = false;   // renormalise after every node
  static constexpr int kUnrollSmallNb = 4;   // timed: +21 % at N_b = 4, a loss at N_b = 8
  static constexpr int kMinBlocks = KBE_SWEEP_MINB_DF64;
  static __device__ __forceinline__ void zero(A &a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void begin(A &) {}
  // after each memory-time node: keep the low word within a few ulps of the
  // high one, so its own FP32 rounding stays at the 2^-48 level over any n
  static __device__ __forceinline__ void end(A &a) {
    df_renorm(a.x, a.y);
    df_renorm(a.z, a.w);
  }
  static __device__ __forceinline__ void mac(A &acc, const S &X, const S &Y) {
    df_mac(acc.x, acc.y, X.x, X.y, Y.x, Y.y);
    df_mac(acc.x, acc.y, -X.z, -X.w, Y.z, Y.w);
    df_mac(acc.z, acc.w, X.x, X.y, Y.z, Y.w);
    df_mac(acc.z, acc.w, X.z, X.w, Y.x, Y.y);
  }
  static __device__ __forceinline__ S sub(const S &X, const S &Y) {
    float4 r;
    df_sub(r.x, r.y, X.x, X.y, Y.x, Y.y);
    df_sub(r.z, r.w, X.z, X.w, Y.z, Y.w);
    return r;
  }
  static __device__ __forceinline__ S negconj(const S &X) { return make_float4(-X.x, -X.y, X.z, X.w); }
  static __device__ __forceinline__ S neg(const S &X) { return make_float4(-X.x, -X.y, -X.z, -X.w); }
  static __device__ __forceinline__ S scale(float f, const S &X) {   // f a power of two: exact
    return make_float4(f * X.x, f * X.y, f * X.z, f * X.w);
  }
  static __device__ __forceinline__ S scale_w(double f, const S &X) {   // any weight, 2^-48 relative
    float4 r;
    df_mul_w(r.x, r.y, X.x, X.y, f);
    df_mul_w(r.z, r.w, X.z, X.w, f);
    return r;
  }
  static __device__ __forceinline__ S add(const S &X, const S &Y) {
    float4 r;
    df_sub(r.x, r.y, X.x, X.y, -Y.x, -Y.y);
    df_sub(r.z, r.w, X.z, X.w, -Y.z, -Y.w);
    return r;
  }
  static __device__ __forceinline__ double2 result(const A &a) {
    return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
  }
  static __device__ __forceinline__ void store(double2 *o, size_t blkc, const A &x, const A &y) {
    const double2 xr = result(x);
    o[0] = xr;
    o[blkc] = c_add(xr, result(y));
  }
};

// ----------------------------------------------------------------- C64 ----
// (h, c) += p with an error-free TwoSum; c collects the rounding errors
__device__ __forceinline__ void comp_add(float &h, float &c, float p) {
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  c = __fadd_rn(c, e);
}

struct AccC64 {
  float4 sum;    // {re, re_comp, im, im_comp}, compensated over l
  float2 part;   // plain FP32 partial of the current l
};

struct ArithC64 {
  using S = float2;
  using A = AccC64;
  static constexpr int V = 1;
  static constexpr bool kGrouped = true;    // the plain partial spans several nodes
  static constexpr int kUnrollSmallNb = 1;
  static constexpr int kMinBlocks = KBE_SWEEP_MINB_C64;
  static __device__ __forceinline__ void zero(A &a) { a.sum = make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void begin(A &a) { a.part = make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void end(A &a) {
    comp_add(a.sum.x, a.sum.y, a.part.x);
    comp_add(a.sum.z, a.sum.w, a.part.y);
  }
  static __device__ __forceinline__ void mac(A &a, const S &x, const S &y) {
    a.part = make_float2(__fmaf_rn(x.x, y.x, __fmaf_rn(-x.y, y.y, a.part.x)),
                         __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, a.part.y)));
  }
  static __device__ __forceinline__ S sub(const S &x, const S &y) { return make_float2(x.x - y.x, x.y - y.y); }
  static __device__ __forceinline__ S negconj(const S &x) { return make_float2(-x.x, x.y); }
  static __device__ __forceinline__ S neg(const S &x) { return make_float2(-x.x, -x.y); }
  static __device__ __forceinline__ S scale(float f, const S &x) { return make_float2(f * x.x, f * x.y); }
  static __device__ __forceinline__ S scale_w(double f, const S &x) {
    const float g = (float)f;
    return make_float2(g * x.x, g * x.y);
  }
  static __device__ __forceinline__ S add(const S &x, const S &y) { return make_float2(x.x + y.x, x.y + y.y); }
  static __device__ __forceinline__ double2 result(const A &a) {
    return make_double2((double)a.sum.x + (double)a.sum.y, (double)a.sum.z + (double)a.sum.w);
  }
  static __device__ __forceinline__ void store(double2 *o, size_t blkc, const A &x, const A &y) {
    const double2 xr = result(x);
    o[0] = xr;
    o[blkc] = c_add(xr, result(y));
  }
};

// C64 with two consecutive k per thread: one 16-byte load carries both
// complex64 values, halving the load instructions per multiply-add (the C64
// sweep is bound by load issue, not by the FP32 pipe); same arithmetic as
// ArithC64 on each half.
struct AccC64x2 {
  AccC64 h[2];
};

struct ArithC64x2 {
  using S = float4;
  using A = AccC64x2;
  static constexpr int V = 2;
  static constexpr bool kGrouped = true;
  static constexpr int kUnrollSmallNb = 1;
  static constexpr int kMinBlocks = KBE_SWEEP_MINB_C64X2;
  static __device__ __forceinline__ float2 lo(const S &x) { return make_float2(x.x, x.y); }
  static __device__ __forceinline__ float2 hi(const S &x) { return make_float2(x.z, x.w); }
  static __device__ __forceinline__ S join(const float2 &a, const float2 &b) { return make_float4(a.x, a.y, b.x, b.y); }
  static __device__ __forceinline__ void zero(A &a) { ArithC64::zero(a.h[0]); ArithC64::zero(a.h[1]); }
  static __device__ __forceinline__ void begin(A &a) { ArithC64::begin(a.h[0]); ArithC64::begin(a.h[1]); }
  static __device__ __forceinline__ void end(A &a) { ArithC64::end(a.h[0]); ArithC64::end(a.h[1]); }
  static __device__ __forceinline__ void mac(A &a, const S &x, const S &y) {
    ArithC64::mac(a.h[0], lo(x), lo(y));
    ArithC64::mac(a.h[1], hi(x), hi(y));
  }
  static __device__ __forceinline__ S sub(const S &x, const S &y) { return join(ArithC64::sub(lo(x), lo(y)), ArithC64::sub(hi(x), hi(y))); }
  static __device__ __forceinline__ S negconj(const S &x) { return make_float4(-x.x, x.y, -x.z, x.w); }
  static __device__ __forceinline__ S neg(const S &x) { return make_float4(-x.x, -x.y, -x.z, -x.w); }
  static __device__ __forceinline__ S scale(float f, const S &x) { return make_float4(f * x.x, f * x.y, f * x.z, f * x.w); }
  static __device__ __forceinline__ S scale_w(double f, const S &x) { return scale((float)f, x); }
  static __device__ __forceinline__ S add(const S &x, const S &y) {
    return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
  }
  static __device__ __forceinline__ void store(double2 *o, size_t blkc, const A &x, const A &y) {
    ArithC64::store(o, blkc, x.h[0], y.h[0]);
    ArithC64::store(o + 1, blkc, x.h[1], y.h[1]);
  }
};

// ------------------------------------------------------------ the sweep ----
// Nodes per compensated group. A node adds N_b products per output into the
// plain partial (begin() clears it, end() folds it into the compensated sum);
// the C64 forms fold only every G nodes, so that at most KBE_C64_COMP_TERMS
// products are summed in plain FP32 (their rounding stays ~1e-6 of the
// group's magnitude, below the complex64 storage error at the mixed form's
// accuracy bar) and the TwoSum costs 1/G of what a fold per node costs.
#ifndef KBE_C64_COMP_TERMS
#define KBE_C64_COMP_TERMS 32
#endif
template <class P, int NB>
__host__ __device__ constexpr int comp_group() {
  return P::kGrouped && NB < KBE_C64_COMP_TERMS ? KBE_C64_COMP_TERMS / NB : 1;
}

// counts the nodes of the current group; at the group's end folds the partials
template <class P, int G>
struct CompGroup {
  int left = G;
  __device__ __forceinline__ static void fold(typename P::A &x, typename P::A &y) {
    P::end(x);
    P::end(y);
    P::begin(x);
    P::begin(y);
  }
  __device__ __forceinline__ void node(typename P::A &x, typename P::A &y) {
    if constexpr (G == 1) {
      fold(x, y);
    } else {
      if (--left == 0) {
        left = G;
        fold(x, y);
      }
    }
  }
};

// One memory-time node l for this thread's element (k, a, b), accumulating
// X = I^< and Y = I^> - I^<: MODE 0 is a node above the output (l > j, or
// j = 0): X += C1 G^<, Y -= C1 dG; MODE 1 an interior node of [0, t_j], where
// both quadratures give weight dt and Y gets nothing: X += C1 G^< + C2^< dG;
// MODE 2 a trapezoid end node of [0, t_j] (l = 0 or l = j, f = 1/2).
// LOWER: the block (l, j) is stored (l >= j), else its adjoint -X(j, l)^+ is read.
template <class P, int NB, int MODE, bool LOWER>
__device__ __forceinline__ void sweep_node(const typename P::S *__restrict__ c1,
                                           const typename P::S *__restrict__ g, size_t blk, int nk,
                                           int b, typename P::A &accX, typename P::A &accY) {
  using S = typename P::S;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    const S A1 = c1[(size_t)c * nk];
    S Gl, D;
    if (LOWER) {   // G(l, j)_cb, dG(l, j)_cb stored directly
      Gl = g[(size_t)(c * NB + b) * nk];
      D = g[blk + (size_t)(c * NB + b) * nk];
    } else {       // X(l, j)_cb = -conj(X(j, l)_bc)
      Gl = P::negconj(g[(size_t)(b * NB + c) * nk]);
      D = P::negconj(g[blk + (size_t)(b * NB + c) * nk]);
    }
    P::mac(accX, A1, Gl);
    if (MODE == 0) {
      P::mac(accY, P::neg(A1), D);
    } else if (MODE == 1) {
      P::mac(accX, c1[blk + (size_t)c * nk], D);
    } else {   // f = 1/2: X += C2^< dG / 2, Y += (C3 - C2^< - C1) dG / 2
      const S K2 = c1[blk + (size_t)c * nk];
      P::mac(accX, P::scale(0.5f, K2), D);
      P::mac(accY, P::scale(0.5f, P::sub(P::sub(c1[2 * blk + (size_t)c * nk], K2), A1)), D);
    }
  }
}

// One node of [0, t_j] with a general weight f = w^(j)_l / dt (the Gregory end
// nodes): X += C1 G^< + f C2^< dG and Y += (f (C3 - C2^<) + (f - 1) C1) dG,
// the last coefficient being (w^(j)_l - w^(n)_l) (S^> - S^<).
template <class P, int NB, bool LOWER>
__device__ __forceinline__ void sweep_wnode(const typename P::S *__restrict__ c1,
                                            const typename P::S *__restrict__ g, size_t blk, int nk,
                                            int b, double f, typename P::A &accX, typename P::A &accY) {
  using S = typename P::S;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    const S A1 = c1[(size_t)c * nk];
    S Gl, D;
    if (LOWER) {
      Gl = g[(size_t)(c * NB + b) * nk];
      D = g[blk + (size_t)(c * NB + b) * nk];
    } else {
      Gl = P::negconj(g[(size_t)(b * NB + c) * nk]);
      D = P::negconj(g[blk + (size_t)(b * NB + c) * nk]);
    }
    const S K2 = c1[blk + (size_t)c * nk];
    P::mac(accX, A1, Gl);
    P::mac(accX, P::scale_w(f, K2), D);
    P::mac(accY, P::add(P::scale_w(f, P::sub(c1[2 * blk + (size_t)c * nk], K2)), P::scale_w(f - 1.0, A1)), D);
  }
}

// grid: x = tiles of the N_b^2 n_k output elements, y = output column j
// (0..n), z = split of the l range (lchunk values each). The tiles of one
// column are adjacent in launch order, so they share its blocks through L2.
// out is the I row when gridDim.z == 1, else the partial-sum scratch
// [z][j][x][a][b][k]. The l range [l0, l1) is walked as three branch-free
// runs: interior nodes 0 < l < j (adjoint blocks), nodes above l > j (stored
// blocks), then the two end nodes l = 0 and l = j.
// one CTA's work, block (bx, by, bz) of `threads` threads (the batched
// persistent kernel calls it for blocks of many systems)
template <class P, int NB, int QUAD>
__device__ __forceinline__ void sweep_block(const typename P::S *__restrict__ H, const typename P::S *__restrict__ Cf,
                                            double2 *__restrict__ out, int n, int nk, int lchunk, int bx, int by,
                                            int bz, int threads) {
  using S = typename P::S;
  const int j = by;
  if ((int)threadIdx.x >= threads) return;
  const int idx = bx * threads + threadIdx.x;
  if (idx >= NB * NB * nk) return;
  const int k = idx % nk;
  const int ab = idx / nk;
  const int a = ab / NB, b = ab - (ab / NB) * NB;
  const int l0 = bz * lchunk;
  const int l1 = min(n + 1, l0 + lchunk);
  const size_t blk = (size_t)NB * NB * nk;
  const S *cbase = Cf + (size_t)a * NB * nk + k;   // C1(l)_{a, .} at cbase + 3 l blk
  const S *hbase = H + k;

  typename P::A accX, accY;   // I^< and I^> - I^<
  P::zero(accX);
  P::zero(accY);
  P::begin(accX);
  P::begin(accY);
  CompGroup<P, comp_group<P, NB>()> grp;
  // interior of [0, t_j] with weight 1: 0 < l < j (trapezoid), 3 <= l <= j - 3 (Gregory)
  const int ia = QUAD == kQuadTrapezoid ? 1 : 3, ib = QUAD == kQuadTrapezoid ? j : j - 2;
  constexpr int U = NB <= 4 ? P::kUnrollSmallNb : 1;
  if (j > 0) {
#pragma unroll U
    for (int l = max(l0, ia); l < min(l1, ib); ++l) {
      sweep_node<P, NB, 1, false>(cbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk, blk, nk, b,
                                  accX, accY);
      grp.node(accX, accY);
    }
  }
#pragma unroll U
  for (int l = max(l0, j == 0 ? 0 : j + 1); l < l1; ++l) {   // above the output
    sweep_node<P, NB, 0, true>(cbase + (size_t)l * 3 * blk, hbase + tri(l, j) * 2 * blk, blk, nk, b,
                               accX, accY);
    grp.node(accX, accY);
  }
  if (j > 0 && QUAD == kQuadTrapezoid) {
    if (l0 == 0) {   // end node l = 0 (adjoint block, 0 < j)
      sweep_node<P, NB, 2, false>(cbase, hbase + tri(j, 0) * 2 * blk, blk, nk, b, accX, accY);
      grp.node(accX, accY);
    }
    if (j >= l0 && j < l1) {   // end node l = j (diagonal block)
      sweep_node<P, NB, 2, true>(cbase + (size_t)j * 3 * blk, hbase + tri(j, j) * 2 * blk, blk, nk, b,
                                 accX, accY);
      grp.node(accX, accY);
    }
  } else if (j > 0) {   // Gregory: the three nodes at each end (every node for j <= 4)
    const int ns = j >= 5 ? 6 : j + 1;
    for (int s = 0; s < ns; ++s) {
      const int l = (j >= 5 && s >= 3) ? j - 5 + s : s;
      if (l < l0 || l >= l1) continue;
      const double f = quad_omega(kQuadGregory, j, l);
      if (l == j)
        sweep_wnode<P, NB, true>(cbase + (size_t)l * 3 * blk, hbase + tri(j, j) * 2 * blk, blk, nk, b, f,
                                 accX, accY);
      else
        sweep_wnode<P, NB, false>(cbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk, blk, nk, b, f,
                                  accX, accY);
      grp.node(accX, accY);
    }
  }
  P::end(accX);   // the last, partly filled group
  P::end(accY);
  // outputs in complex numbers: nk, blk and k above count stored elements S
  const size_t blkc = blk * P::V;
  double2 *o = out + ((size_t)bz * (n + 1) + j) * 2 * blkc + (size_t)ab * nk * P::V + (size_t)k * P::V;
  P::store(o, blkc, accX, accY);
}

template <class P, int NB, int QUAD>
__global__ void __launch_bounds__(256, P::kMinBlocks) sweep_kernel(const typename P::S *__restrict__ H,
                                                    const typename P::S *__restrict__ Cf,
                                                    double2 *__restrict__ out, int n, int nk,
                                                    int lchunk, const int *__restrict__ skip) {
  if (skip && *skip) return;
  sweep_block<P, NB, QUAD>(H, Cf, out, n, nk, lchunk, blockIdx.x, blockIdx.y, blockIdx.z, blockDim.x);
}

// ---------------------------------------------- C64, register-blocked ----
// At N_b <= 2 a thread owns one k and all N_b^2 outputs (a, b) of both
// components: each stored value and each coefficient is loaded once per node
// and feeds N_b multiply-adds, against one per load in the per-element form
// (whose loads, not its FP32 arithmetic, bound it at small N_b). Same
// arithmetic and node classes as sweep_kernel.
template <class P, int NB, int MODE, bool LOWER>
__device__ __forceinline__ void blocked_node(const typename P::S *__restrict__ cf,
                                             const typename P::S *__restrict__ g, size_t blk, int nk, double f,
                                             typename P::A *X, typename P::A *Y) {
  using S = typename P::S;
  S Gm[NB * NB], Dm[NB * NB];   // X(l, j)_cb, dG(l, j)_cb
#pragma unroll
  for (int c = 0; c < NB; ++c)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (LOWER) {
        Gm[c * NB + b] = g[(size_t)(c * NB + b) * nk];
        Dm[c * NB + b] = g[blk + (size_t)(c * NB + b) * nk];
      } else {
        Gm[c * NB + b] = P::negconj(g[(size_t)(b * NB + c) * nk]);
        Dm[c * NB + b] = P::negconj(g[blk + (size_t)(b * NB + c) * nk]);
      }
    }
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const S A1 = cf[(size_t)(a * NB + c) * nk];
      S K2, KY;
      if (MODE == 0) {            // above the output
        KY = P::neg(A1);
      } else if (MODE == 1) {     // interior of [0, t_j]
        K2 = cf[blk + (size_t)(a * NB + c) * nk];
      } else {                    // weighted node (f), Y coefficient f (C3 - C2^<) + (f - 1) C1
        const S k2 = cf[blk + (size_t)(a * NB + c) * nk], k3 = cf[2 * blk + (size_t)(a * NB + c) * nk];
        K2 = P::scale_w(f, k2);
        KY = P::add(P::scale_w(f, P::sub(k3, k2)), P::scale_w(f - 1.0, A1));
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        P::mac(X[a * NB + b], A1, Gm[c * NB + b]);
        if (MODE != 0) P::mac(X[a * NB + b], K2, Dm[c * NB + b]);
        if (MODE != 1) P::mac(Y[a * NB + b], KY, Dm[c * NB + b]);
      }
    }
}

template <class P, int NB>
__device__ __forceinline__ void blocked_fold(typename P::A *X, typename P::A *Y) {
#pragma unroll
  for (int e = 0; e < NB * NB; ++e) CompGroup<P, 1>::fold(X[e], Y[e]);
}

// grid: x = tiles of n_k, y = output column j, z = split of the l range; out as
// for sweep_kernel
#ifndef KBE_BLOCKED_THREADS
#define KBE_BLOCKED_THREADS 128
#endif
#ifndef KBE_BLOCKED_MINB
#define KBE_BLOCKED_MINB 3   // 168 registers without spills at N_b = 2
#endif
template <class P, int NB, int QUAD>
__global__ void __launch_bounds__(KBE_BLOCKED_THREADS, KBE_BLOCKED_MINB) sweep_blocked_kernel(const typename P::S *__restrict__ H,
                                                               const typename P::S *__restrict__ Cf,
                                                               double2 *__restrict__ out, int n, int nk,
                                                               int lchunk, const int *__restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NB2 = NB * NB, G = comp_group<P, NB>();
  const int j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int l0 = blockIdx.z * lchunk;
  const int l1 = min(n + 1, l0 + lchunk);
  const size_t blk = (size_t)NB2 * nk;
  const typename P::S *cbase = Cf + k, *hbase = H + k;
  typename P::A X[NB2], Y[NB2];   // I^< and I^> - I^< for every (a, b)
#pragma unroll
  for (int e = 0; e < NB2; ++e) {
    P::zero(X[e]);
    P::zero(Y[e]);
    P::begin(X[e]);
    P::begin(Y[e]);
  }
  int left = G;
  auto tick = [&]() {
    if (--left == 0) {
      left = G;
      blocked_fold<P, NB>(X, Y);
    }
  };
  const int ia = QUAD == kQuadTrapezoid ? 1 : 3, ib = QUAD == kQuadTrapezoid ? j : j - 2;
  if (j > 0)
    for (int l = max(l0, ia); l < min(l1, ib); ++l) {   // interior, adjoint blocks
      blocked_node<P, NB, 1, false>(cbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk, blk, nk, 1.0, X, Y);
      tick();
    }
  for (int l = max(l0, j == 0 ? 0 : j + 1); l < l1; ++l) {   // above the output
    blocked_node<P, NB, 0, true>(cbase + (size_t)l * 3 * blk, hbase + tri(l, j) * 2 * blk, blk, nk, 1.0, X, Y);
    tick();
  }
  if (j > 0) {   // the end nodes: l = 0 and l = j (trapezoid), three at each end (Gregory)
    const int ns = QUAD == kQuadTrapezoid ? 2 : (j >= 5 ? 6 : j + 1);
    for (int s = 0; s < ns; ++s) {
      const int l = QUAD == kQuadTrapezoid ? (s == 0 ? 0 : j) : ((j >= 5 && s >= 3) ? j - 5 + s : s);
      if (l < l0 || l >= l1) continue;
      const double f = quad_omega(QUAD, j, l);
      if (l == j)
        blocked_node<P, NB, 2, true>(cbase + (size_t)l * 3 * blk, hbase + tri(j, j) * 2 * blk, blk, nk, f, X, Y);
      else
        blocked_node<P, NB, 2, false>(cbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk, blk, nk, f, X, Y);
    }
  }
  blocked_fold<P, NB>(X, Y);
  double2 *o = out + ((size_t)blockIdx.z * (n + 1) + j) * 2 * blk + k;
#pragma unroll
  for (int e = 0; e < NB2; ++e) P::store(o + (size_t)e * nk, blk, X[e], Y[e]);
}

// ------------------------------------------- FP64, three-multiplication --
// The FP64 sweep is bound by the FP64 pipe, so it pays to spend fewer DFMAs.
// A complex product needs three real multiplications:
//   A B = (P1 - P2) + i (P3 - P1 - P2),  P1 = Ar Br, P2 = Ai Bi,
//   P3 = (Ar + Ai)(Br + Bi),
// and the sums of products over a column's nodes can be kept as the three
// sums P1, P2, P3. The extra additions are shared: coef_kernel stores
// Ar + Ai of every coefficient (Cs), and a thread owns one column b of the
// output for every row a, so the sum Br + Bi of each history element it
// loads feeds N_b products. 6 N_b DFMAs per output and node (X and Y, or the
// two products of an interior node) instead of 8 N_b. Exact algebra; only
// the rounding differs. Same node classes and launch shape as sweep_kernel.
template <int NB>
struct F64m {
  double p[3][NB];   // P1, P2, P3 of rows a
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int a = 0; a < NB; ++a) p[t][a] = 0.0;
  }
  // += (or -= when NEG) A B for row a; as = Ar + Ai, bs = Br + Bi
  template <bool NEG>
  __device__ __forceinline__ void mac(int a, double2 A, double as, double2 B, double bs) {
    const double s = NEG ? -1.0 : 1.0;
    p[0][a] = fma(s * A.x, B.x, p[0][a]);
    p[1][a] = fma(s * A.y, B.y, p[1][a]);
    p[2][a] = fma(s * as, bs, p[2][a]);
  }
  __device__ __forceinline__ double2 value(int a) const {
    return make_double2(p[0][a] - p[1][a], p[2][a] - p[0][a] - p[1][a]);
  }
};

// one node: B = the block's column b as used (G, dG of (l, j); LOWER: stored,
// else -conj of the stored (j, l)), the coefficient planes at node l
template <int NB, int MODE, bool LOWER>
__device__ __forceinline__ void f64m_node(const double2 *__restrict__ cf, const double *__restrict__ cs,
                                          const double2 *__restrict__ g, size_t blk, int nk, int b, double f,
                                          F64m<NB> &X, F64m<NB> &Y) {
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double2 G, D;
    if (LOWER) {
      G = g[(size_t)(c * NB + b) * nk];
      D = g[blk + (size_t)(c * NB + b) * nk];
    } else {
      const double2 g0 = g[(size_t)(b * NB + c) * nk], d0 = g[blk + (size_t)(b * NB + c) * nk];
      G = make_double2(-g0.x, g0.y);
      D = make_double2(-d0.x, d0.y);
    }
    const double gs = G.x + G.y, ds = D.x + D.y;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const size_t o = (size_t)(a * NB + c) * nk;
      const double2 A1 = cf[o];
      const double a1s = cs[o];
      X.template mac<false>(a, A1, a1s, G, gs);
      if (MODE == 0) {   // above the output: Y -= C1 dG
        Y.template mac<true>(a, A1, a1s, D, ds);
      } else if (MODE == 1) {   // interior of [0, t_j]: X += C2^< dG
        X.template mac<false>(a, cf[blk + o], cs[blk + o], D, ds);
      } else {   // weighted node: X += f C2^< dG, Y += (f (C3 - C2^<) + (f - 1) C1) dG
        const double2 k2 = cf[blk + o], k3 = cf[2 * blk + o];
        const double2 K2 = make_double2(f * k2.x, f * k2.y);
        const double2 KY = make_double2(f * (k3.x - k2.x) + (f - 1.0) * A1.x, f * (k3.y - k2.y) + (f - 1.0) * A1.y);
        X.template mac<false>(a, K2, K2.x + K2.y, D, ds);
        Y.template mac<false>(a, KY, KY.x + KY.y, D, ds);
      }
    }
  }
}

constexpr int kF64mThreads = 128;
// CTAs per SM the register cap aims for: N_b >= 6 keeps its 6 N_b accumulators
// and the unrolled node in registers at 2 (the FP64 pipe needs few warps)
__host__ __device__ constexpr int f64m_minb(int NB) { return NB >= 6 ? 2 : 4; }

// grid: x = k tiles of 128 / N_b, y = output column j, z = split of the l range;
// thread (kk, b) with b fastest (the N_b lanes of one k read each coefficient
// together); out as for sweep_kernel
template <int NB, int QUAD>
__device__ __forceinline__ void f64m_block(const double2 *__restrict__ H, const double2 *__restrict__ Cf,
                                           const double *__restrict__ Cs, double2 *__restrict__ out, int n, int nk,
                                           int lchunk, int bx, int by, int bz) {
  constexpr int KT = kF64mThreads / NB;
  if ((int)threadIdx.x >= KT * NB) return;
  const int b = threadIdx.x % NB, kk = threadIdx.x / NB;
  const int k = bx * KT + kk;
  if (k >= nk) return;
  const int j = by;
  const int l0 = bz * lchunk;
  const int l1 = min(n + 1, l0 + lchunk);
  const size_t blk = (size_t)NB * NB * nk;
  const double2 *cbase = Cf + k;
  const double *sbase = Cs + k;
  const double2 *hbase = H + k;
  F64m<NB> X, Y;   // I^< and I^> - I^< of column b
  X.zero();
  Y.zero();
  const int ia = QUAD == kQuadTrapezoid ? 1 : 3, ib = QUAD == kQuadTrapezoid ? j : j - 2;
  if (j > 0)
    for (int l = max(l0, ia); l < min(l1, ib); ++l)   // interior of [0, t_j], adjoint blocks
      f64m_node<NB, 1, false>(cbase + (size_t)l * 3 * blk, sbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk,
                              blk, nk, b, 1.0, X, Y);
  for (int l = max(l0, j == 0 ? 0 : j + 1); l < l1; ++l)   // above the output, stored blocks
    f64m_node<NB, 0, true>(cbase + (size_t)l * 3 * blk, sbase + (size_t)l * 3 * blk, hbase + tri(l, j) * 2 * blk,
                           blk, nk, b, 1.0, X, Y);
  if (j > 0) {   // the end nodes: l = 0 and l = j (trapezoid), three at each end (Gregory)
    const int ns = QUAD == kQuadTrapezoid ? 2 : (j >= 5 ? 6 : j + 1);
    for (int t = 0; t < ns; ++t) {
      const int l = QUAD == kQuadTrapezoid ? (t == 0 ? 0 : j) : ((j >= 5 && t >= 3) ? j - 5 + t : t);
      if (l < l0 || l >= l1) continue;
      const double f = quad_omega(QUAD, j, l);
      if (l == j)
        f64m_node<NB, 2, true>(cbase + (size_t)l * 3 * blk, sbase + (size_t)l * 3 * blk, hbase + tri(j, j) * 2 * blk,
                               blk, nk, b, f, X, Y);
      else
        f64m_node<NB, 2, false>(cbase + (size_t)l * 3 * blk, sbase + (size_t)l * 3 * blk, hbase + tri(j, l) * 2 * blk,
                                blk, nk, b, f, X, Y);
    }
  }
  double2 *o = out + ((size_t)bz * (n + 1) + j) * 2 * blk + k;
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    const double2 x = X.value(a), y = Y.value(a);
    o[(size_t)(a * NB + b) * nk] = x;
    o[blk + (size_t)(a * NB + b) * nk] = c_add(x, y);
  }
}

template <int NB, int QUAD>
__global__ void __launch_bounds__(kF64mThreads, f64m_minb(NB)) sweep_f64m_kernel(const double2 *__restrict__ H,
                                                                      const double2 *__restrict__ Cf,
                                                                      const double *__restrict__ Cs,
                                                                      double2 *__restrict__ out, int n, int nk,
                                                                      int lchunk, const int *__restrict__ skip) {
  if (skip && *skip) return;
  f64m_block<NB, QUAD>(H, Cf, Cs, out, n, nk, lchunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

// I = sum over the z partial rows (FP64)
__global__ void reduce_partials_kernel(const double2 *__restrict__ part, double2 *__restrict__ I,
                                       size_t count, int nz, const int *__restrict__ skip) {
  if (skip && *skip) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    double2 s = part[i];
    for (int z = 1; z < nz; ++z) s = c_add(s, part[(size_t)z * count + i]);
    I[i] = s;
  }
}

// --------------------------------------------------- packing and coefficients
// nblocks blocks [2][nb][nb][nk] of (G^<, G^>) in FP64 -> (G^<, dG = G^< - G^>)
// in the history storage (dG formed in FP64 before rounding)
// (nb, nk, row: the mesh and the row of the blocks, used by the F16X2 layout)
__global__ void pack_kernel(int prec, const double2 *__restrict__ src, void *__restrict__ dst,
                            size_t nblocks, size_t blk, const int *__restrict__ skip, int nb, int nk, int row,
                            int cap) {
  if (skip && *skip) return;
  const size_t count = nblocks * blk;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t bq = i / blk, r = i - bq * blk;
    const size_t o0 = bq * 2 * blk + r, o1 = o0 + blk;
    const double2 gl = src[o0];
    pack_store(prec, dst, o0, o1, gl, c_sub(gl, src[o1]), nb, nk, row, cap);
  }
}

// one component of nblk blocks into [j][k][a][b] (the getters' layout): from
// the FP64 working row (G^<, G^>) when fp64 != NULL, else from the history's
// (G^<, dG) storage of precision prec (G^> = G^< - dG)
// (row, cap: the row of the blocks and the rows the storage holds, used by the
// F16X2 layout, for which packed is the storage start)
__global__ void row_out_kernel(int prec, const double2 *__restrict__ fp64, const void *__restrict__ packed,
                               size_t nblk, int nb, int nk, int which, double2 *__restrict__ out, int row,
                               int cap) {
  const size_t blk = (size_t)nb * nb * nk, count = nblk * blk;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = i / blk, r = i - j * blk;   // r = (k nb + a) nb + b
    const int k = (int)(r / ((size_t)nb * nb)), ab = (int)(r - (size_t)k * nb * nb);
    const size_t s0 = j * 2 * blk + (size_t)ab * nk + k, s1 = s0 + blk;
    double2 v;
    if (fp64) {
      v = fp64[which ? s1 : s0];
    } else {
      double2 gl, dg;
      if (prec == KBE_PREC_F16X2) {
        const int a = ab / nb, b = ab - a * nb;
        gl = f16x2_get((const __half *)packed, row, (int)j, k, 0, a, b, nb, cap);
        dg = f16x2_get((const __half *)packed, row, (int)j, k, 1, a, b, nb, cap);
      } else if (prec == KBE_PREC_DF64) {
        const float4 a = ((const float4 *)packed)[s0], b = ((const float4 *)packed)[s1];
        gl = make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
        dg = make_double2((double)b.x + (double)b.y, (double)b.z + (double)b.w);
      } else if (prec == KBE_PREC_C64) {
        const float2 a = ((const float2 *)packed)[s0], b = ((const float2 *)packed)[s1];
        gl = make_double2(a.x, a.y);
        dg = make_double2(b.x, b.y);
      } else {
        gl = ((const double2 *)packed)[s0];
        dg = ((const double2 *)packed)[s1];
      }
      v = which ? c_sub(gl, dg) : gl;
    }
    out[i] = v;
  }
}

// coefficient rows [l][3][a][c][k]: C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<, C3 = dt S^> - C1
// (FP64 also stores re + im of every coefficient in Cs, [l][3][a][c][k], for the
// three-multiplication products of sweep_f64m_kernel)
// cmax (may be NULL, zeroed before the launch): the largest |re|, |im| of C1
// and C2^< over the row, as the bits of a non-negative float (the scale of the
// tensor-core sweep's FP16 coefficient pairs)
__global__ void coef_kernel(int prec, const double2 *__restrict__ Sig, void *__restrict__ Cf, int n,
                            int nk, int nb2, double dt, const int *__restrict__ skip, int quad,
                            double *__restrict__ Cs, unsigned *__restrict__ cmax, int sig32 = 0) {
  if (skip && *skip) return;
  const size_t blk = (size_t)nb2 * nk;
  const size_t total = (size_t)(n + 1) * blk;
  double big = 0.0;
  if (prec == KBE_PREC_C64 || prec == KBE_PREC_F16X2) {
    // complex64 coefficients from FP32 arithmetic (their Sigma row is complex64
    // values held in FP64): GB300's FP64 pipe made this kernel FP64-bound
    const float fdt = (float)dt;
    float fbig = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
      const size_t l = i / blk, r = i - l * blk;
      float2 sl, sg;
      if (sig32) {   // the row as complex64 (sigma_row's sig32)
        sl = ((const float2 *)Sig)[(l * 2) * blk + r];
        sg = ((const float2 *)Sig)[(l * 2 + 1) * blk + r];
      } else {
        const double2 dl = Sig[(l * 2) * blk + r], dg = Sig[(l * 2 + 1) * blk + r];
        sl = make_float2((float)dl.x, (float)dl.y);
        sg = make_float2((float)dg.x, (float)dg.y);
      }
      const float w1 = (float)(dt * quad_omega(quad, n, (int)l));
      const float2 c1 = make_float2(w1 * (sg.x - sl.x), w1 * (sg.y - sl.y));
      const float2 c2 = make_float2(fdt * sl.x, fdt * sl.y);
      const float2 c3 = make_float2(fmaf(fdt, sg.x, -c1.x), fmaf(fdt, sg.y, -c1.y));
      float2 *cf = (float2 *)Cf;
      cf[(l * 3) * blk + r] = c1;
      cf[(l * 3 + 1) * blk + r] = c2;
      cf[(l * 3 + 2) * blk + r] = c3;
      fbig = fmaxf(fbig, fmaxf(fmaxf(fabsf(c1.x), fabsf(c1.y)), fmaxf(fabsf(c2.x), fabsf(c2.y))));
    }
    if (cmax) {   // blockDim is a multiple of 32
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) fbig = fmaxf(fbig, __shfl_xor_sync(0xffffffffu, fbig, off));
      if ((threadIdx.x & 31) == 0 && fbig > 0.f) atomicMax(cmax, __float_as_uint(fbig));
    }
    return;
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t l = i / blk, r = i - l * blk;
    const double2 sl = Sig[(l * 2) * blk + r], sg = Sig[(l * 2 + 1) * blk + r];
    const double w1 = dt * quad_omega(quad, n, (int)l);
    const double2 c1 = c_scale(w1, c_sub(sg, sl));
    const double2 v[3] = {c1, c_scale(dt, sl), c_sub(c_scale(dt, sg), c1)};
    for (int q = 0; q < 3; ++q) {
      const size_t o = (l * 3 + q) * blk + r;
      if (prec == KBE_PREC_DF64) ((float4 *)Cf)[o] = split_df(v[q]);
      else if (prec == KBE_PREC_C64 || prec == KBE_PREC_F16X2)
        ((float2 *)Cf)[o] = make_float2((float)v[q].x, (float)v[q].y);
      else ((double2 *)Cf)[o] = v[q];
      if (Cs) Cs[o] = v[q].x + v[q].y;
    }
    big = fmax(big, fmax(fmax(fabs(v[0].x), fabs(v[0].y)), fmax(fabs(v[1].x), fabs(v[1].y))));
  }
  if (cmax) {   // blockDim is a multiple of 32
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, off));
    if ((threadIdx.x & 31) == 0 && big > 0.0) atomicMax(cmax, __float_as_uint((float)big));
  }
}


// ------------------------------------------------ C64, staged through smem --
// The C64 sweep is bound by load latency, not by the FP32 pipe. This form
// stages every memory-time node's operands in shared memory ahead of use: a
// CTA of 128 threads owns KT consecutive k for all outputs (a, b) of one
// column j, and for each node l copies the three coefficient rows (C1, C2^<,
// C3 for all (a, c)) and the block X(l, j) (G^< and dG, both orientations
// come from the same stored block) for its k range into a ring of kStages
// buffers with 16-byte cp.async copies, kStages - 1 nodes ahead of the
// arithmetic (zero-filled past n_k). Each thread keeps NBB <= 4 outputs
// (a, b..b+NBB) of both components in registers, so one shared-memory load
// of a coefficient feeds NBB multiply-adds. The waits are cp.async group
// waits and barriers only. Same C64 arithmetic as ArithC64 (FP32 products
// summed over groups of comp_group nodes, the groups folded into a
// TwoSum-compensated sum). The TMA variant below replaces the per-thread
// copies and is the one used when a tensor map can be encoded.
#ifndef KBE_STAGED_STAGES
#define KBE_STAGED_STAGES 3   // timed: 4 stages (2 CTAs/SM) 9 % slower, 2 stages no better
#endif
#ifndef KBE_STAGED_MINB
#define KBE_STAGED_MINB 3
#endif
#ifndef KBE_STAGED_TARGET
#define KBE_STAGED_TARGET 12  // CTAs per SM the l-split aims for (timed: 3, 6, 12 within 3 %)
#endif
constexpr int kStagedThreads = 128;
constexpr int kStages = KBE_STAGED_STAGES;

__host__ __device__ constexpr int staged_nbb(int NB) { return NB < 4 ? NB : 4; }
__host__ __device__ constexpr int staged_kt(int NB) { return kStagedThreads / (NB * (NB / staged_nbb(NB))); }
__host__ __device__ constexpr size_t staged_stage_elems(int NB) { return (size_t)5 * NB * NB * staged_kt(NB); }

bool staged_supported(int nb) { return nb == 1 || nb == 2 || nb == 4 || nb == 8 || nb == 16; }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;   // 0: zero-fill, nothing read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// copy node l's operands for k in [k0, k0 + KT) into one stage buffer:
// [q][a][c][kk] coefficient rows (q = C1, C2^<, C3), then [x][r][s][kk] of the
// stored block (x = G^<, dG), as float2 pairs (16 bytes)
template <int NB>
__device__ __forceinline__ void staged_issue(float2 *st, const float2 *__restrict__ Cf,
                                             const float2 *__restrict__ H, int l, size_t tblk, int k0,
                                             int nk) {
  constexpr int KT = staged_kt(NB), NB2 = NB * NB, CH = KT / 2;   // 16-byte chunks per row
  const size_t blk = (size_t)NB2 * nk;
  const float2 *csrc = Cf + (size_t)l * 3 * blk;
  const float2 *hsrc = H + tblk * 2 * blk;
  constexpr int nrow = 5 * NB2;                                     // 3 NB^2 + 2 NB^2 rows
  for (int e = threadIdx.x; e < nrow * CH; e += kStagedThreads) {
    const int row = e / CH, ch = e - row * CH;
    const int kk = 2 * ch, kg = k0 + kk;
    const bool valid = kg < nk;   // n_k even: a chunk is wholly inside or wholly past the end
    const float2 *src = row < 3 * NB2 ? csrc + (size_t)row * nk : hsrc + (size_t)(row - 3 * NB2) * nk;
    cp_async16(st + (size_t)row * KT + kk, valid ? src + kg : src, valid);
  }
}

// one node on the staged operands, into X = I^< and Y = I^> - I^<. KIND 0:
// above the output (stored block): X += C1 G^<, Y -= C1 dG; 3: interior of
// [0, t_j] (adjoint block, both quadratures weigh it dt): X += C1 G^< + C2^< dG;
// 1 (stored diagonal block) and 2 (adjoint block): a node of weight f = w^(j)_l / dt,
// X += C1 G^< + f C2^< dG, Y += (f (C3 - C2^<) + (f - 1) C1) dG
template <int NB, int KIND>
__device__ __forceinline__ void staged_node(const float2 *st, int kk, int a, int b0, float f, AccC64 *accX,
                                            AccC64 *accY) {
  constexpr int KT = staged_kt(NB), NBB = staged_nbb(NB), NB2 = NB * NB;
  const float2 *c1 = st + (size_t)(0 * NB2 + a * NB) * KT + kk;
  const float2 *c2 = st + (size_t)(1 * NB2 + a * NB) * KT + kk;
  const float2 *c3 = st + (size_t)(2 * NB2 + a * NB) * KT + kk;
  const float2 *gl = st + (size_t)(3 * NB2) * KT + kk;
  const float2 *dg = st + (size_t)(4 * NB2) * KT + kk;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    const float2 A1 = c1[(size_t)c * KT];
    float2 K2 = make_float2(0.f, 0.f), KY = make_float2(0.f, 0.f);
    if (KIND == 0) {
      KY = make_float2(-A1.x, -A1.y);
    } else if (KIND == 3) {
      K2 = c2[(size_t)c * KT];
    } else {
      const float2 k2 = c2[(size_t)c * KT], k3 = c3[(size_t)c * KT];
      K2 = make_float2(f * k2.x, f * k2.y);
      KY = make_float2(f * (k3.x - k2.x) + (f - 1.0f) * A1.x, f * (k3.y - k2.y) + (f - 1.0f) * A1.y);
    }
#pragma unroll
    for (int q = 0; q < NBB; ++q) {
      const int b = b0 + q;
      float2 G, D;
      if (KIND >= 2) {   // X(l, j)_cb = -conj(G(j, l)_bc)
        const float2 g = gl[(size_t)(b * NB + c) * KT], d = dg[(size_t)(b * NB + c) * KT];
        G = make_float2(-g.x, g.y);
        D = make_float2(-d.x, d.y);
      } else {
        G = gl[(size_t)(c * NB + b) * KT];
        D = dg[(size_t)(c * NB + b) * KT];
      }
      ArithC64::mac(accX[q], A1, G);
      if (KIND != 0) ArithC64::mac(accX[q], K2, D);
      if (KIND != 3) ArithC64::mac(accY[q], KY, D);
    }
  }
}

// the staged kernels' compensated groups (comp_group nodes each) over their NBB outputs
template <int NB>
struct StagedGroup {
  static constexpr int G = comp_group<ArithC64, NB>();
  int left = G;
  __device__ __forceinline__ static void fold(AccC64 *accX, AccC64 *accY) {
#pragma unroll
    for (int q = 0; q < staged_nbb(NB); ++q) {
      ArithC64::end(accX[q]);
      ArithC64::end(accY[q]);
      ArithC64::begin(accX[q]);
      ArithC64::begin(accY[q]);
    }
  }
  __device__ __forceinline__ void node(AccC64 *accX, AccC64 *accY) {
    if (--left == 0) {
      left = G;
      fold(accX, accY);
    }
  }
};

// node l of output column j: above the output, interior of [0, t_j], or a
// weighted node (stored diagonal / adjoint end node)
template <int NB, int QUAD>
__device__ __forceinline__ void staged_any_node(const float2 *st, int kk, int a, int b0, int j, int l,
                                                AccC64 *accX, AccC64 *accY) {
  if (l > j || j == 0) {
    staged_node<NB, 0>(st, kk, a, b0, 1.0f, accX, accY);
  } else if (QUAD == kQuadTrapezoid ? (l > 0 && l < j) : (l >= 3 && l <= j - 3)) {
    staged_node<NB, 3>(st, kk, a, b0, 1.0f, accX, accY);
  } else {
    const float f = (float)quad_omega(QUAD, j, l);
    if (l == j) staged_node<NB, 1>(st, kk, a, b0, f, accX, accY);
    else staged_node<NB, 2>(st, kk, a, b0, f, accX, accY);
  }
}

// grid: x = k tiles of KT, y = output column j (0..n), z = split of the l range
template <int NB, int QUAD>
__global__ void __launch_bounds__(kStagedThreads, KBE_STAGED_MINB)
    sweep_c64_staged_kernel(const float2 *__restrict__ H, const float2 *__restrict__ Cf, double2 *__restrict__ out,
                            int n, int nk, int lchunk, const int *__restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float4 staged_smem4[];
  float2 *smem = reinterpret_cast<float2 *>(staged_smem4);
  constexpr int KT = staged_kt(NB), NBB = staged_nbb(NB);
  const int tid = threadIdx.x;
  const int kk = tid % KT, rest = tid / KT;
  const int a = rest % NB, b0 = (rest / NB) * NBB;
  const int k0 = blockIdx.x * KT;
  const int j = blockIdx.y;
  const int l0 = blockIdx.z * lchunk;
  const int l1 = min(n + 1, l0 + lchunk);
  const int nodes = max(l1 - l0, 0);
  AccC64 accX[NBB], accY[NBB];   // I^< and I^> - I^<
#pragma unroll
  for (int q = 0; q < NBB; ++q) {
    ArithC64::zero(accX[q]);
    ArithC64::zero(accY[q]);
    ArithC64::begin(accX[q]);
    ArithC64::begin(accY[q]);
  }
  StagedGroup<NB> grp;
  // node i is l = l0 + i; its block is stored at (l, j) when l >= j, else (j, l)
  auto tblk = [&](int l) -> size_t { return l >= j ? tri(l, j) : tri(j, l); };
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nodes) staged_issue<NB>(smem + (size_t)s * staged_stage_elems(NB), Cf, H, l0 + s, tblk(l0 + s), k0, nk);
    cp_async_commit();
  }
  for (int i = 0; i < nodes; ++i) {
    const int ahead = i + kStages - 1;
    if (ahead < nodes)
      staged_issue<NB>(smem + (size_t)(ahead % kStages) * staged_stage_elems(NB), Cf, H, l0 + ahead, tblk(l0 + ahead),
                       k0, nk);
    cp_async_commit();
    cp_async_wait<kStages - 1>();   // this thread's copies of node i have landed
    __syncthreads();                // and everybody else's
    const float2 *st = smem + (size_t)(i % kStages) * staged_stage_elems(NB);
    staged_any_node<NB, QUAD>(st, kk, a, b0, j, l0 + i, accX, accY);
    grp.node(accX, accY);
    __syncthreads();                // the stage may be refilled next iteration
  }
  StagedGroup<NB>::fold(accX, accY);   // the last, partly filled group
  const int k = k0 + kk;
  if (k >= nk) return;
  const size_t blk = (size_t)NB * NB * nk;
  double2 *o = out + ((size_t)blockIdx.z * (n + 1) + j) * 2 * blk + k;
#pragma unroll
  for (int q = 0; q < NBB; ++q) ArithC64::store(o + (size_t)(a * NB + b0 + q) * nk, blk, accX[q], accY[q]);
}


// The same staged sweep with TMA copies: one thread issues, per node, a 3-D
// tensor copy of the coefficient rows (box 2KT floats x N_b^2 x 3 rows of
// [l][q][a][c][k]) and a 4-D one of the stored block (box 2KT x N_b^2 x 2
// components x 1 block of [tri][x][r][s][k]) into the stage, completing on
// that stage's mbarrier; the hardware zero-fills past n_k. The shared-memory
// layout is the cp.async form's, so the arithmetic is shared. Every wait on
// an mbarrier is bounded: past the limit the kernel marks kDevTimeout in the
// status word and stops after waiting (bounded) for its copies in flight; if
// that wait runs out too it also marks kDevTimeoutDrain (a copy may still be
// writing into shared memory the CTA gives up).

template <int NB, int QUAD>
__global__ void __launch_bounds__(kStagedThreads, KBE_STAGED_MINB)
    sweep_c64_tma_kernel(const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmH,
                         double2 *__restrict__ out, int n, int nk, int lchunk, const int *__restrict__ skip,
                         int *status, int drop_first) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) float4 tma_smem4[];
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ int failed;
  float2 *smem = reinterpret_cast<float2 *>(tma_smem4);
  constexpr int KT = staged_kt(NB), NBB = staged_nbb(NB), NB2 = NB * NB;
  constexpr unsigned kBytesC = 3u * NB2 * KT * sizeof(float2), kBytesH = 2u * NB2 * KT * sizeof(float2);
  const int tid = threadIdx.x;
  const int kk = tid % KT, rest = tid / KT;
  const int a = rest % NB, b0 = (rest / NB) * NBB;
  const int k0 = blockIdx.x * KT;
  const int j = blockIdx.y;
  const int l0 = blockIdx.z * lchunk;
  const int l1 = min(n + 1, l0 + lchunk);
  const int nodes = max(l1 - l0, 0);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // drop_first (fault injection for the timeout test): the first CTA omits
  // its first node's copies, so that its waits run out
  const bool drop = drop_first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  auto issue = [&](int i) {   // node i into stage i % kStages (thread 0)
    if (drop && i == 0) return;
    const int l = l0 + i, s = i % kStages;
    const int tb = (int)(l >= j ? tri(l, j) : tri(j, l));
    float2 *st = smem + (size_t)s * staged_stage_elems(NB);
    mbar_expect_tx(&bar[s], kBytesC + kBytesH);
    tma_load_3d(st, &tmC, 2 * k0, 0, 3 * l, &bar[s]);
    tma_load_4d(st + (size_t)3 * NB2 * KT, &tmH, 2 * k0, 0, 0, tb, &bar[s]);
  };
  AccC64 accX[NBB], accY[NBB];   // I^< and I^> - I^<
#pragma unroll
  for (int q = 0; q < NBB; ++q) {
    ArithC64::zero(accX[q]);
    ArithC64::zero(accY[q]);
    ArithC64::begin(accX[q]);
    ArithC64::begin(accY[q]);
  }
  StagedGroup<NB> grp;
  if (tid == 0)
    for (int i = 0; i < kStages - 1 && i < nodes; ++i) issue(i);
  int issued = min(kStages - 1, nodes);
  for (int i = 0; i < nodes; ++i) {
    if (tid == 0 && issued < nodes && issued == i + kStages - 1) {
      issue(issued);
    }
    issued = min(i + kStages, nodes);
    const int s = i % kStages;
    if (!mbar_wait(&bar[s], (unsigned)((i / kStages) & 1), kMbarWaitLimit)) failed = 1;
    __syncthreads();
    if (failed) {   // a copy did not arrive: flag it, let the in-flight ones land, stop
      if (tid == 0) {
        int st = kDevTimeout;
        for (int q = i; q < issued; ++q) {
          if (drop && q == 0) continue;   // never issued (fault injection): nothing in flight
          if (!mbar_wait(&bar[q % kStages], (unsigned)((q / kStages) & 1), kMbarWaitLimit)) st |= kDevTimeoutDrain;
        }
        if (status) atomicOr(status, st);
      }
      __syncthreads();
      return;
    }
    const float2 *st = smem + (size_t)s * staged_stage_elems(NB);
    staged_any_node<NB, QUAD>(st, kk, a, b0, j, l0 + i, accX, accY);
    grp.node(accX, accY);
    __syncthreads();   // stage s is free for the copy issued next iteration
  }
  StagedGroup<NB>::fold(accX, accY);   // the last, partly filled group
  const int k = k0 + kk;
  if (k >= nk) return;
  const size_t blk = (size_t)NB2 * nk;
  double2 *o = out + ((size_t)blockIdx.z * (n + 1) + j) * 2 * blk + k;
#pragma unroll
  for (int q = 0; q < NBB; ++q) ArithC64::store(o + (size_t)(a * NB + b0 + q) * nk, blk, accX[q], accY[q]);
}

// tensor maps of the coefficient rows (rows 0..n) and the stored triangle (rows
// 0..n) of a C64 sweep; false when the driver cannot encode them
template <int NB>
bool staged_tensor_maps(const void *Cf, const void *H, int n, int nk, CUtensorMap *tmC, CUtensorMap *tmH) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  constexpr int KT = staged_kt(NB), NB2 = NB * NB;
  const cuuint64_t row = (cuuint64_t)2 * nk * sizeof(float);   // one (a, c) row of k, bytes
  {
    const cuuint64_t dim[3] = {(cuuint64_t)2 * nk, (cuuint64_t)NB2, (cuuint64_t)3 * (n + 1)};
    const cuuint64_t stride[2] = {row, row * NB2};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * KT), (cuuint32_t)NB2, 3};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(Cf), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t ntri = (cuuint64_t)tri(n, n) + 1;
    const cuuint64_t dim[4] = {(cuuint64_t)2 * nk, (cuuint64_t)NB2, 2, ntri};
    const cuuint64_t stride[3] = {row, row * NB2, row * NB2 * 2};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * KT), (cuuint32_t)NB2, 2, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(tmH, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(H), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// shared-memory limits of the staged kernels, raised once per device (the
// attribute belongs to the current device's context), under a lock
template <int NB>
cudaError_t staged_prepare() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  tensor_map_encoder();   // resolve the driver entry point outside any stream capture
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  const int bytes = (int)(kStages * staged_stage_elems(NB) * sizeof(float2));
  e = cudaFuncSetAttribute(sweep_c64_staged_kernel<NB, kQuadTrapezoid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_c64_staged_kernel<NB, kQuadGregory>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_c64_tma_kernel<NB, kQuadTrapezoid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_c64_tma_kernel<NB, kQuadGregory>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

unsigned grid_for(size_t count) {
  const size_t b = (count + 255) / 256, cap = (size_t)device_sms() * 64;
  return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

// l-split: enough CTAs to give every SM ~8 resident CTAs; the number of
// partial rows nz (n+1) stays below 2(n+1) + 1024
constexpr int kTargetPerSm = 8;

struct SweepShape {
  dim3 grid;
  int threads, lchunk, nz;
};

#ifndef KBE_SWEEP_C64_TMA
#define KBE_SWEEP_C64_TMA 1      // the staged sweep's copies by TMA (else per-thread cp.async)
#endif
#ifndef KBE_SWEEP_C64_STAGED
#define KBE_SWEEP_C64_STAGED 1   // C64: the shared-memory staged sweep where it applies
#endif

// the C64 staged form: N_b in {4, 8, 16} and n_k even (16-byte copies); at
// N_b <= 2 a node is too little arithmetic for two barriers (timed: the
// paper's two-band shape 5.56 ms staged against 5.23 ms for the pair form)
bool use_staged(const Mesh &m, int prec) {
  return KBE_SWEEP_C64_STAGED && prec == KBE_PREC_C64 && staged_supported(m.nb) && m.nb >= 4 &&
         m.nk % 2 == 0;
}

// C64 at N_b <= 2: one thread per k owns all N_b^2 outputs
#ifndef KBE_SWEEP_C64_BLOCKED
#define KBE_SWEEP_C64_BLOCKED 1
#endif
bool use_blocked(const Mesh &m, int prec) { return KBE_SWEEP_C64_BLOCKED && prec == KBE_PREC_C64 && m.nb <= 2; }

// V: complex values of consecutive k per thread (the C64 pair form)
int sweep_width(const Mesh &m, int prec) {
  return (KBE_SWEEP_C64_PAIRS && prec == KBE_PREC_C64 && m.nk % 2 == 0) ? 2 : 1;
}

int staged_kt_of(int nb) {
  switch (nb) {
    case 1: return staged_kt(1);
    case 2: return staged_kt(2);
    case 4: return staged_kt(4);
    case 8: return staged_kt(8);
    default: return staged_kt(16);
  }
}

// ---- l-split of the memory-time range (autotuned per shape) ----------------
// The number of CTAs sharing one output column's l range is chosen so that the
// grid reaches about `target` CTAs per SM; kbe_autotune times candidate
// targets per (form, quadrature, N_b, n_k, row bucket) and keeps the best for
// the process. Every choice obeys nz <= nz_cap(n), which sizes the workspace.
int nz_cap(int n) { return min(n + 1, 2 + 1024 / (n + 1)); }
int row_bucket(int n) {
  int b = 0;
  while ((2 << b) <= n + 1 && b < 30) ++b;
  return b;   // floor(log2(n + 1))
}
using TuneKey = std::tuple<int, int, int, int, int>;   // precision, quadrature, nb, nk, bucket
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

int tuned_target(int prec, int quad, const Mesh &m, int n, int fallback) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey(prec, quad, m.nb, m.nk, row_bucket(n)));
  return it == g_tune.end() ? fallback : it->second;
}

long split_count(long base, int n, int target) {
  long nz = ((long)device_sms() * target + base - 1) / base;
  if (nz > nz_cap(n)) nz = nz_cap(n);
  return nz < 1 ? 1 : nz;
}

// l-split of the staged form: enough CTAs for ~target resident per SM
SweepShape staged_shape(const Mesh &m, int n, int target = KBE_STAGED_TARGET) {
  SweepShape sh;
  sh.threads = kStagedThreads;
  const int kt = staged_kt_of(m.nb);
  const long tx = (m.nk + kt - 1) / kt;
  const long base = (long)(n + 1) * tx;
  long nz = split_count(base, n, target);
  sh.lchunk = (int)((n + 1 + nz - 1) / nz);
  sh.nz = (int)((n + 1 + sh.lchunk - 1) / sh.lchunk);
  sh.grid = dim3((unsigned)tx, n + 1, (unsigned)sh.nz);
  return sh;
}

SweepShape sweep_shape(const Mesh &m, int n, int V = 1, int target = kTargetPerSm, int maxthreads = 256) {
  SweepShape sh;
  const long elems = (long)m.nb * m.nb * (m.nk / V);
  sh.threads = elems >= maxthreads ? maxthreads : (int)((elems + 31) / 32) * 32;
  const long ty = (elems + sh.threads - 1) / sh.threads;
  const long base = (long)(n + 1) * ty;
  long nz = split_count(base, n, target);   // at least one l per split, bounded scratch
  sh.lchunk = (int)((n + 1 + nz - 1) / nz);
  sh.nz = (int)((n + 1 + sh.lchunk - 1) / sh.lchunk);
  sh.grid = dim3((unsigned)ty, n + 1, (unsigned)sh.nz);
  return sh;
}

template <class P> struct PrecOf;
template <> struct PrecOf<ArithF64> { static constexpr int v = KBE_PREC_FP64; };
template <> struct PrecOf<ArithDF64> { static constexpr int v = KBE_PREC_DF64; };
template <> struct PrecOf<ArithC64> { static constexpr int v = KBE_PREC_C64; };
template <> struct PrecOf<ArithC64x2> { static constexpr int v = KBE_PREC_C64; };

template <class P, int NB>
cudaError_t sweep_nb(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, double2 *part,
                     cudaStream_t st, const int *skip, int quad) {
  const SweepShape sh = sweep_shape(m, n, P::V, tuned_target(PrecOf<P>::v, quad, m, n, kTargetPerSm));
  double2 *out = sh.nz > 1 ? part : I;
  const int nkS = m.nk / P::V;   // stored elements per (a, b) array
  if (quad == kQuadGregory)
    sweep_kernel<P, NB, kQuadGregory><<<sh.grid, sh.threads, 0, st>>>(
        (const typename P::S *)H, (const typename P::S *)Cf, out, n, nkS, sh.lchunk, skip);
  else
    sweep_kernel<P, NB, kQuadTrapezoid><<<sh.grid, sh.threads, 0, st>>>(
        (const typename P::S *)H, (const typename P::S *)Cf, out, n, nkS, sh.lchunk, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sh.nz == 1) return e;
  const size_t count = (size_t)(n + 1) * 2 * m.nb * m.nb * m.nk;
  reduce_partials_kernel<<<grid_for(count), 256, 0, st>>>(part, I, count, sh.nz, skip);
  return cudaGetLastError();
}

// the three-multiplication FP64 sweep (N_b <= 8): k tiles of 128 / N_b, split as sweep_kernel

template <int NB>
cudaError_t sweep_f64m(const Mesh &m, int n, const void *H, const void *Cf, const double *Cs, double2 *I,
                       double2 *part, cudaStream_t st, const int *skip, int quad) {
  constexpr int KT = kF64mThreads / NB;
  SweepShape sh;
  sh.threads = kF64mThreads;
  const long tx = (m.nk + KT - 1) / KT;
  const long nz = split_count((long)(n + 1) * tx, n, tuned_target(KBE_PREC_FP64, quad, m, n, kTargetPerSm));
  sh.lchunk = (int)((n + 1 + nz - 1) / nz);
  sh.nz = (int)((n + 1 + sh.lchunk - 1) / sh.lchunk);
  sh.grid = dim3((unsigned)tx, n + 1, (unsigned)sh.nz);
  double2 *out = sh.nz > 1 ? part : I;
  if (quad == kQuadGregory)
    sweep_f64m_kernel<NB, kQuadGregory><<<sh.grid, sh.threads, 0, st>>>((const double2 *)H, (const double2 *)Cf, Cs,
                                                                         out, n, m.nk, sh.lchunk, skip);
  else
    sweep_f64m_kernel<NB, kQuadTrapezoid><<<sh.grid, sh.threads, 0, st>>>((const double2 *)H, (const double2 *)Cf, Cs,
                                                                           out, n, m.nk, sh.lchunk, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sh.nz == 1) return e;
  const size_t count = (size_t)(n + 1) * 2 * m.nb * m.nb * m.nk;
  reduce_partials_kernel<<<grid_for(count), 256, 0, st>>>(part, I, count, sh.nz, skip);
  return cudaGetLastError();
}

template <int NB>
cudaError_t sweep_blocked(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, double2 *part,
                          cudaStream_t st, const int *skip, int quad) {
  const Mesh m1{1, m.L0, m.L1, m.nk};   // one thread per k
  SweepShape sh = sweep_shape(m1, n, 1, tuned_target(KBE_PREC_C64, quad, m, n, kTargetPerSm),
                              KBE_BLOCKED_THREADS);
  double2 *out = sh.nz > 1 ? part : I;
  if (quad == kQuadGregory)
    sweep_blocked_kernel<ArithC64, NB, kQuadGregory><<<sh.grid, sh.threads, 0, st>>>(
        (const float2 *)H, (const float2 *)Cf, out, n, m.nk, sh.lchunk, skip);
  else
    sweep_blocked_kernel<ArithC64, NB, kQuadTrapezoid><<<sh.grid, sh.threads, 0, st>>>(
        (const float2 *)H, (const float2 *)Cf, out, n, m.nk, sh.lchunk, skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sh.nz == 1) return e;
  const size_t count = (size_t)(n + 1) * 2 * m.nb * m.nb * m.nk;
  reduce_partials_kernel<<<grid_for(count), 256, 0, st>>>(part, I, count, sh.nz, skip);
  return cudaGetLastError();
}

template <int NB>
cudaError_t sweep_staged(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, double2 *part,
                         cudaStream_t st, const int *skip, int quad, int *status, int inject) {
  cudaError_t e = staged_prepare<NB>();
  if (e != cudaSuccess) return e;
  const SweepShape sh = staged_shape(m, n, tuned_target(KBE_PREC_C64, quad, m, n, KBE_STAGED_TARGET));
  double2 *out = sh.nz > 1 ? part : I;
  const size_t smem = kStages * staged_stage_elems(NB) * sizeof(float2);
  CUtensorMap tmC, tmH;
  if (KBE_SWEEP_C64_TMA && staged_tensor_maps<NB>(Cf, H, n, m.nk, &tmC, &tmH)) {
    if (quad == kQuadGregory)
      sweep_c64_tma_kernel<NB, kQuadGregory><<<sh.grid, sh.threads, smem, st>>>(tmC, tmH, out, n, m.nk, sh.lchunk,
                                                                               skip, status, inject);
    else
      sweep_c64_tma_kernel<NB, kQuadTrapezoid><<<sh.grid, sh.threads, smem, st>>>(tmC, tmH, out, n, m.nk,
                                                                                 sh.lchunk, skip, status, inject);
  } else if (quad == kQuadGregory)
    sweep_c64_staged_kernel<NB, kQuadGregory><<<sh.grid, sh.threads, smem, st>>>(
        (const float2 *)H, (const float2 *)Cf, out, n, m.nk, sh.lchunk, skip);
  else
    sweep_c64_staged_kernel<NB, kQuadTrapezoid><<<sh.grid, sh.threads, smem, st>>>(
        (const float2 *)H, (const float2 *)Cf, out, n, m.nk, sh.lchunk, skip);
  e = cudaGetLastError();
  if (e != cudaSuccess || sh.nz == 1) return e;
  const size_t count = (size_t)(n + 1) * 2 * m.nb * m.nb * m.nk;
  reduce_partials_kernel<<<grid_for(count), 256, 0, st>>>(part, I, count, sh.nz, skip);
  return cudaGetLastError();
}

// The complex64 sweep's form per row: a negative tuned choice -TI selects the
// single-read tile kernel with TI rows per work item (kbe_sweep_tile.cu);
// untuned rows take it from n = 255 on (TI = 32), where its work items fill
// the GPU. Fault injection always takes the staged kernel.
constexpr int kTileMinTI = 32;
int tile_default(const Mesh &m, int prec, int n) {
  return tile_supported(m, prec) && n >= 255 ? -32 : 0;
}

// the tensor-core sweep of the split-FP16 form: TI = -choice rows per panel
constexpr int kTcDefaultTI = 64;
// (odd: TI - 1 rows per panel, the row segments copied by loader warps)
int tc_choice(const Mesh &m, int prec, int quad, int n) {
  const int t = tuned_target(prec, quad, m, n, -kTcDefaultTI);
  return t < 0 ? -t : kTcDefaultTI;
}

template <int NB>
cudaError_t sweep_prec(const Mesh &m, int n, int prec, const void *H, const void *Cf, double2 *I,
                       double2 *part, cudaStream_t st, const int *skip, int quad, int *status, int inject,
                       int cap) {
  if (prec == KBE_PREC_F16X2) {
    if (!tc_supported(m, prec)) return cudaErrorInvalidValue;
    return launch_sweep_tc(m, n, H, Cf, I, part, st, skip, quad, status, tc_choice(m, prec, quad, n), cap);
  }
  if constexpr (NB == 2 || NB == 4 || NB == 8) {
    if (tile_supported(m, prec) && !inject) {
      const int t = tuned_target(prec, quad, m, n, tile_default(m, prec, n));
      if (t < 0) return launch_sweep_tile(m, n, H, Cf, I, part, st, skip, quad, status, -t);
    }
  }
  if constexpr (NB == 1 || NB == 2 || NB == 4 || NB == 8 || NB == 16) {
    if (use_staged(m, prec)) return sweep_staged<NB>(m, n, H, Cf, I, part, st, skip, quad, status, inject);
  }
  if constexpr (NB <= 2) {
    if (use_blocked(m, prec)) return sweep_blocked<NB>(m, n, H, Cf, I, part, st, skip, quad);
  }
  if constexpr (NB <= 8) {
    if (use_f64m(m, prec)) {
      const size_t cn = (size_t)(n + 1) * 3 * NB * NB * m.nk;   // Cs follows the coefficient rows
      return sweep_f64m<NB>(m, n, H, Cf, (const double *)((const double2 *)Cf + cn), I, part, st, skip, quad);
    }
  }
  if (prec == KBE_PREC_FP64) return sweep_nb<ArithF64, NB>(m, n, H, Cf, I, part, st, skip, quad);
  if (prec == KBE_PREC_DF64) return sweep_nb<ArithDF64, NB>(m, n, H, Cf, I, part, st, skip, quad);
  if (sweep_width(m, prec) == 2) return sweep_nb<ArithC64x2, NB>(m, n, H, Cf, I, part, st, skip, quad);
  return sweep_nb<ArithC64, NB>(m, n, H, Cf, I, part, st, skip, quad);
}

// ---- the FP64 sweeps of many systems in one persistent launch (kbe_batch) --
// Every system contributes the blocks of its own sweep shape (k tiles x output
// columns x l-splits, the split chosen per shape by the autotuner); a CTA
// walks the concatenated block list with a grid stride and runs each block
// with its system's operands. One launch per (N_b, quadrature, kernel form).
constexpr int kMaxBatchJobs = 48;
struct BatchTable {
  SweepJob job[kMaxBatchJobs];
  long first[kMaxBatchJobs + 1];   // first[q]: the first block of job q; first[njobs]: all blocks
  int njobs;
};

__device__ __forceinline__ int batch_job_of(const BatchTable &t, long w) {
  int q = 0;
  while (q + 1 < t.njobs && w >= t.first[q + 1]) ++q;
  return q;
}

template <int NB, int QUAD>
__global__ void __launch_bounds__(kF64mThreads, f64m_minb(NB)) batch_f64m_kernel(const __grid_constant__ BatchTable t) {
  for (long w = blockIdx.x; w < t.first[t.njobs]; w += gridDim.x) {
    const SweepJob &jb = t.job[batch_job_of(t, w)];
    if (jb.skip && *jb.skip) continue;   // a converged corrector pass of that system
    const long loc = w - t.first[&jb - t.job];
    const int bx = (int)(loc % jb.tx);
    const long r = loc / jb.tx;
    f64m_block<NB, QUAD>(jb.H, jb.Cf, jb.Cs, jb.out, jb.n, jb.nk, jb.lchunk, bx, (int)(r % (jb.n + 1)),
                         (int)(r / (jb.n + 1)));
  }
}

template <int NB, int QUAD>
__global__ void __launch_bounds__(256, ArithF64::kMinBlocks) batch_plain_kernel(const __grid_constant__ BatchTable t) {
  for (long w = blockIdx.x; w < t.first[t.njobs]; w += gridDim.x) {
    const SweepJob &jb = t.job[batch_job_of(t, w)];
    if (jb.skip && *jb.skip) continue;
    const long loc = w - t.first[&jb - t.job];
    const int bx = (int)(loc % jb.tx);
    const long r = loc / jb.tx;
    sweep_block<ArithF64, NB, QUAD>(jb.H, jb.Cf, jb.out, jb.n, jb.nk, jb.lchunk, bx, (int)(r % (jb.n + 1)),
                                    (int)(r / (jb.n + 1)), jb.threads);
  }
}

template <int NB, int QUAD>
cudaError_t batch_launch_nb(const BatchTable &t, bool f64m, cudaStream_t st) {
  const long total = t.first[t.njobs];
  if (total == 0) return cudaSuccess;
  if (f64m) {
    if constexpr (NB <= 8) {
      const long slots = (long)device_sms() * f64m_minb(NB);
      batch_f64m_kernel<NB, QUAD><<<(unsigned)(total < slots ? total : slots), kF64mThreads, 0, st>>>(t);
    }
  } else {
    const long slots = (long)device_sms() * ArithF64::kMinBlocks;
    batch_plain_kernel<NB, QUAD><<<(unsigned)(total < slots ? total : slots), 256, 0, st>>>(t);
  }
  return cudaGetLastError();
}

template <int QUAD>
cudaError_t batch_launch(const BatchTable &t, int nb, bool f64m, cudaStream_t st) {
  switch (nb) {
    case 1: return batch_launch_nb<1, QUAD>(t, f64m, st);
    case 2: return batch_launch_nb<2, QUAD>(t, f64m, st);
    case 3: return batch_launch_nb<3, QUAD>(t, f64m, st);
    case 4: return batch_launch_nb<4, QUAD>(t, f64m, st);
    case 6: return batch_launch_nb<6, QUAD>(t, f64m, st);
    case 8: return batch_launch_nb<8, QUAD>(t, f64m, st);
    case 12: return batch_launch_nb<12, QUAD>(t, f64m, st);
    case 16: return batch_launch_nb<16, QUAD>(t, f64m, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool use_f64m(const Mesh &m, int prec) { return prec == KBE_PREC_FP64 && m.nb <= 8; }

double sweep_tc_flops(const Mesh &m, int prec, int quad, int n) {
  return tc_supported(m, prec) ? tc_tensor_flops(m, n, tc_choice(m, prec, quad, n)) : 0.0;
}

// cuTensorMapEncodeTiled from the driver (no link against libcuda); resolved
// once per process (a thread-safe static: the entry point is not per device)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PFN_cuTensorMapEncodeTiled_v12000 r = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
    return r;
  }();
  return fn;
}

int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = -1;
  }
  if (dev >= 0 && dev < kMaxDev) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 1;
  }
  if (dev < kMaxDev) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

bool sweep_supported(int nb) {
  switch (nb) {
    case 1: case 2: case 3: case 4: case 6: case 8: case 12: case 16: return true;
    default: return false;
  }
}

bool precision_supported(int prec) {
  return prec == KBE_PREC_FP64 || prec == KBE_PREC_DF64 || prec == KBE_PREC_C64 || prec == KBE_PREC_F16X2;
}

// bytes per stored complex number (F16X2: four halves)
size_t history_elem_bytes(int prec) {
  return prec == KBE_PREC_C64 || prec == KBE_PREC_F16X2 ? sizeof(float2) : 16;
}

// coefficient rows (n+1) x 3 blocks in the storage format, then the partial
// sums of the l split (FP64) or of the tile form (complex64)
// coefficient rows in the storage format (FP64: followed by their re + im sums)
size_t coef_region_bytes(const Mesh &m, int n, int prec) {
  const size_t cn = (size_t)(n + 1) * 3 * m.nb * m.nb * m.nk;
  size_t coef = cn * history_elem_bytes(prec) + (prec == KBE_PREC_FP64 ? cn * sizeof(double) : 0);
  return (coef + 255) / 256 * 256;
}

size_t sweep_workspace_bytes(const Mesh &m, int n, int prec) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const size_t coef = coef_region_bytes(m, n, prec);
  size_t part = 0;
  (void)prec;
  for (int r = 0; r <= n; ++r) {   // the largest partial buffer over rows 0..n, any split
    if (nz_cap(r) > 1) {
      const size_t b = (size_t)nz_cap(r) * (r + 1) * 2 * blk * sizeof(double2);
      if (b > part) part = b;
    }
  }
  if (tile_supported(m, prec)) {   // the tile form's partials at its smallest TI (grows with n)
    const size_t b = tile_part_bytes(m, n, kTileMinTI);
    if (b > part) part = b;
  }
  if (tc_supported(m, prec)) {     // the tensor-core form's operands and partials at its smallest TI
    const size_t b = tc_part_bytes(m, n, kTileMinTI);
    if (b > part) part = b;
  }
  return coef + part;
}

int sweep_splits(const Mesh &m, int n, int prec, int quad) {
  if (tc_supported(m, prec)) return 2;   // operand preparation, the MMA kernel, the reduction
  if ((m.nb == 2 || m.nb == 4 || m.nb == 8) && tile_supported(m, prec) &&
      tuned_target(prec, quad, m, n, tile_default(m, prec, n)) < 0)
    return 2;   // the tile kernel and its reduction
  if (use_staged(m, prec)) return staged_shape(m, n, tuned_target(prec, quad, m, n, KBE_STAGED_TARGET)).nz;
  return sweep_shape(m, n, sweep_width(m, prec), tuned_target(prec, quad, m, n, kTargetPerSm)).nz;
}

// Times launch_sweep at one row per power-of-two bucket of n (up to nmax)
// for each candidate target and keeps the fastest per bucket. H, Sig, I and
// work are the caller's buffers for row nmax (contents are not used for
// timing; I and work are overwritten). out[b] = the choice for bucket b.
cudaError_t tune_sweep(const Mesh &m, int prec, int quad, int nmax, double dt, const void *H, const double2 *Sig,
                       double2 *I, void *work, cudaStream_t st, int *out, int nout, int cap) {
  const bool staged = use_staged(m, prec);
  std::vector<int> cands = staged ? std::vector<int>{3, 6, 12, 24} : std::vector<int>{2, 4, 8, 16, 32};
  if (tile_supported(m, prec))   // the single-read tile form, TI rows per work item (odd: one CTA per unit)
    for (int ti : {kTileMinTI, 64, 128}) {
      cands.push_back(-ti);
      cands.push_back(-(ti + 1));
    }
  if (tc_supported(m, prec)) {   // the tensor-core form: TI rows per panel, bulk or loader-warp copies
    cands.clear();
    for (int ti : {kTileMinTI, 64, 128})
      if (ti <= tc_max_ti(m.nb)) {
        cands.push_back(-ti);
        cands.push_back(-(ti + 1));
      }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cudaErrorUnknown;
  cudaError_t err = cudaSuccess;
  for (int b = 0; b < nout; ++b) out[b] = 0;
  for (int b = 0; err == cudaSuccess && b <= row_bucket(nmax) && b < nout; ++b) {
    const int n = min(nmax, (3 << b) / 2 - 1 > 0 ? (3 << b) / 2 - 1 : 0);   // mid-bucket row
    const TuneKey key(prec, quad, m.nb, m.nk, b);
    float best = 1e30f;
    int best_t = cands[0];
    for (int t : cands) {
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = t;
      }
      for (int w = 0; w < 2 && err == cudaSuccess; ++w)
        err = launch_sweep(m, n, dt, prec, H, Sig, I, work, st, nullptr, quad, nullptr, 0, cap);
      if (err == cudaSuccess) err = cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && err == cudaSuccess; ++r)
        err = launch_sweep(m, n, dt, prec, H, Sig, I, work, st, nullptr, quad, nullptr, 0, cap);
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && ms < best) {
        best = ms;
        best_t = t;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_t;
    out[b] = best_t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

// manual form of the autotuner's table (kbe_set_sweep_choice): bucket -1 sets
// every bucket; choice 0 removes the entry (the default applies again)
bool set_sweep_choice(const Mesh &m, int prec, int quad, int bucket, int choice) {
  if (tc_supported(m, prec)) {   // the tensor-core form takes only TI = -choice (a multiple of 16; + 1: loader warps)
    const int ti = (-choice) & ~1;
    if (choice > 0 || (choice < 0 && (ti < 16 || ti % 16 != 0 || ti > tc_max_ti(m.nb)))) return false;
  } else if (choice < 0 && (!tile_supported(m, prec) || -choice < kTileMinTI || -choice > 4096)) {
    return false;
  }
  if (choice > 64 || bucket < -1 || bucket >= 31) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int b = bucket < 0 ? 0 : bucket; b <= (bucket < 0 ? 30 : bucket); ++b) {
    const TuneKey key(prec, quad, m.nb, m.nk, b);
    if (choice == 0) g_tune.erase(key);
    else g_tune[key] = choice;
  }
  return true;
}

// shared-memory limits of the staged kernels (host side, before any capture)
cudaError_t sweep_prepare(int nb) {
  cudaError_t e = tile_prepare(nb);
  if (e == cudaSuccess) e = tc_prepare(nb);
  if (e != cudaSuccess) return e;
  switch (nb) {
    case 1: return staged_prepare<1>();
    case 2: return staged_prepare<2>();
    case 4: return staged_prepare<4>();
    case 8: return staged_prepare<8>();
    case 16: return staged_prepare<16>();
    default: return cudaSuccess;
  }
}

cudaError_t launch_pack(int prec, const double2 *src, void *dst, size_t nblocks, size_t blk,
                        cudaStream_t st, const int *skip, int nb, int row, int cap) {
  if (nblocks == 0 || blk == 0) return cudaSuccess;
  if (prec == KBE_PREC_F16X2 && (!(nb == 4 || nb == 8) || blk % ((size_t)nb * nb) != 0 || cap <= 0))
    return cudaErrorInvalidValue;
  const int nk = nb > 0 ? (int)(blk / ((size_t)nb * nb)) : 0;
  pack_kernel<<<grid_for(nblocks * blk), 256, 0, st>>>(prec, src, dst, nblocks, blk, skip, nb, nk, row, cap);
  return cudaGetLastError();
}

size_t history_row_offset(const Mesh &m, int prec, int i) {
  if (prec == KBE_PREC_F16X2) return 0;
  return tri(i, 0) * 2 * (size_t)m.nb * m.nb * m.nk * history_elem_bytes(prec);
}

size_t history_bytes(const Mesh &m, int prec, int n) {
  if (prec == KBE_PREC_F16X2) return f16x2_history_bytes(n + 1, m.nb, m.nk);
  return (tri(n, n) + 1) * 2 * (size_t)m.nb * m.nb * m.nk * history_elem_bytes(prec);
}

cudaError_t launch_row_out(int prec, const double2 *fp64, const void *packed, size_t nblk, const Mesh &m,
                           int which, double2 *out, cudaStream_t st, int row, int cap) {
  const size_t count = nblk * (size_t)m.nb * m.nb * m.nk;
  if (count == 0) return cudaSuccess;
  if (prec == KBE_PREC_F16X2 && !fp64 && (row < 0 || cap <= row)) return cudaErrorInvalidValue;
  row_out_kernel<<<grid_for(count), 256, 0, st>>>(prec, fp64, packed, nblk, m.nb, m.nk, which, out, row, cap);
  return cudaGetLastError();
}

cudaError_t prepare_sweep_job(const Mesh &m, int n, double dt, const void *H, const double2 *Sig, double2 *I,
                              void *work, cudaStream_t st, const int *skip, int quad, SweepJob *job) {
  if (!sweep_supported(m.nb)) return cudaErrorInvalidValue;
  const size_t blk = (size_t)m.nb * m.nb * m.nk, total = (size_t)(n + 1) * blk;
  double *Cs = (double *)((double2 *)work + (size_t)(n + 1) * 3 * blk);
  coef_kernel<<<grid_for(total), 256, 0, st>>>(KBE_PREC_FP64, Sig, work, n, m.nk, m.nb * m.nb, dt, skip, quad, Cs,
                                              nullptr);   // as launch_sweep
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SweepJob &jb = *job;
  jb.H = (const double2 *)H;
  jb.Cf = (const double2 *)work;
  jb.Cs = Cs;
  jb.I = I;
  jb.skip = skip;
  jb.n = n;
  jb.nk = m.nk;
  jb.nb = m.nb;
  jb.quad = quad;
  jb.f64m = use_f64m(m, KBE_PREC_FP64) ? 1 : 0;
  const int target = tuned_target(KBE_PREC_FP64, quad, m, n, kTargetPerSm);
  if (jb.f64m) {   // as sweep_f64m
    const int KT = kF64mThreads / m.nb;
    jb.tx = (m.nk + KT - 1) / KT;
    jb.threads = kF64mThreads;
    const long nz = split_count((long)(n + 1) * jb.tx, n, target);
    jb.lchunk = (int)((n + 1 + nz - 1) / nz);
  } else {         // as sweep_nb<ArithF64>
    const SweepShape sh = sweep_shape(m, n, 1, target);
    jb.tx = (int)sh.grid.x;
    jb.threads = sh.threads;
    jb.lchunk = sh.lchunk;
  }
  jb.nz = (n + 1 + jb.lchunk - 1) / jb.lchunk;
  jb.out = jb.nz > 1 ? (double2 *)((char *)work + coef_region_bytes(m, n, KBE_PREC_FP64)) : I;
  return cudaSuccess;
}

cudaError_t finish_sweep_job(const SweepJob &job, cudaStream_t st) {
  if (job.nz <= 1) return cudaSuccess;
  const size_t count = (size_t)(job.n + 1) * 2 * job.nb * job.nb * job.nk;
  reduce_partials_kernel<<<grid_for(count), 256, 0, st>>>(job.out, job.I, count, job.nz, job.skip);
  return cudaGetLastError();
}

cudaError_t launch_sweep_batch(const SweepJob *jobs, int njobs, cudaStream_t st, int *launches) {
  std::vector<bool> done((size_t)njobs, false);
  if (launches) *launches = 0;
  for (int q0 = 0; q0 < njobs; ++q0) {   // one launch per (N_b, quadrature, form), at most kMaxBatchJobs jobs
    if (done[q0]) continue;
    BatchTable t{};
    t.njobs = 0;
    t.first[0] = 0;
    for (int q = q0; q < njobs && t.njobs < kMaxBatchJobs; ++q) {
      const SweepJob &a = jobs[q0], &b = jobs[q];
      if (done[q] || b.nb != a.nb || b.quad != a.quad || b.f64m != a.f64m) continue;
      done[q] = true;
      t.job[t.njobs] = b;
      t.first[t.njobs + 1] = t.first[t.njobs] + (long)b.tx * (b.n + 1) * b.nz;
      ++t.njobs;
    }
    cudaError_t e = jobs[q0].quad == kQuadGregory ? batch_launch<kQuadGregory>(t, jobs[q0].nb, jobs[q0].f64m != 0, st)
                                                  : batch_launch<kQuadTrapezoid>(t, jobs[q0].nb, jobs[q0].f64m != 0, st);
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
  }
  return cudaSuccess;
}

cudaError_t launch_sweep(const Mesh &m, int n, double dt, int precision, const void *H,
                         const double2 *Sig, double2 *I, void *work, cudaStream_t st, const int *skip,
                         int quad, int *status, int inject, int cap, bool sig32) {
  if (!precision_supported(precision)) return cudaErrorInvalidValue;
  if (sig32 && precision != KBE_PREC_C64 && precision != KBE_PREC_F16X2) return cudaErrorInvalidValue;
  if (cap <= 0) cap = n + 1;
  if (cap < n + 1) return cudaErrorInvalidValue;
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const size_t total = (size_t)(n + 1) * blk;
  double *Cs = precision == KBE_PREC_FP64 ? (double *)((double2 *)work + (size_t)(n + 1) * 3 * blk) : nullptr;
  double2 *part = (double2 *)((char *)work + coef_region_bytes(m, n, precision));
  unsigned *cmax = nullptr;   // the tensor-core form's coefficient scale
  cudaError_t e = cudaSuccess;
  if (tc_supported(m, precision)) {
    cmax = tc_cmax_word(part);
    e = cudaMemsetAsync(cmax, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  coef_kernel<<<grid_for(total), 256, 0, st>>>(precision, Sig, work, n, m.nk, m.nb * m.nb, dt, skip, quad, Cs, cmax,
                                              sig32 ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (m.nb) {
    case 1: return sweep_prec<1>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 2: return sweep_prec<2>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 3: return sweep_prec<3>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 4: return sweep_prec<4>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 6: return sweep_prec<6>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 8: return sweep_prec<8>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 12: return sweep_prec<12>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    case 16: return sweep_prec<16>(m, n, precision, H, work, I, part, st, skip, quad, status, inject, cap);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kbe

// build and device facts for diagnostics (include/kbe.h)
extern "C" kbe_status kbe_device_info(int *binary_version, int *sm_count) {
  if (binary_version) {
    cudaFuncAttributes fa{};
    const cudaError_t e = cudaFuncGetAttributes(&fa, kbe::reduce_partials_kernel);
    if (e != cudaSuccess) {
      kbe::set_last_error(std::string("device_info: ") + cudaGetErrorString(e));
      return KBE_ERR_CUDA;
    }
    *binary_version = fa.binaryVersion;
  }
  if (sm_count) *sm_count = kbe::device_sms();
  return KBE_OK;
}
