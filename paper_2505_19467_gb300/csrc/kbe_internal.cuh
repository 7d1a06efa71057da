// Internal declarations of libkbe (CUDA, sm_103a). Not part of the C ABI.
//
// Device layout (all c128 interleaved as double2):
//   history   H[tri(i,j)][x][a][b][k]   i >= j, tri(i,j) = i(i+1)/2 + j
//   rows      R[l][x][a][b][k]          (self-energy row, collision row)
//   per-k     M[a][b][k]                (h, U, V, W), lam[a][k]
// k is the fastest index so that consecutive threads (consecutive k) read
// consecutive 16-byte elements.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>

#include "kbe.h"

namespace kbe {

constexpr int kMaxNb = 16;
constexpr int kMaxNk = 4096;

struct Mesh {
  int nb, L0, L1, nk;
};

__host__ __device__ __forceinline__ size_t tri(int i, int j) {
  return (size_t)i * (size_t)(i + 1) / 2 + (size_t)j;
}

// composite trapezoid weight of node l on [0, t_m]; zero for m = 0
__host__ __device__ __forceinline__ double trap_weight(int m, int l, double dt) {
  if (m == 0) return 0.0;
  double w = dt;
  if (l == 0) w -= 0.5 * dt;
  if (l == m) w -= 0.5 * dt;
  return w;
}

enum : int { kQuadTrapezoid = 0, kQuadGregory = 1 };

// quadrature weight of node l on [0, t_m] in units of dt (zero for m = 0):
// trapezoid (the paper's second-order rule), or fourth-order Gregory: end
// corrections 3/8, 7/6, 23/24 at both ends for m >= 5, and for m <= 4 the
// closed Newton-Cotes rule of the whole interval (m = 1 trapezoid, 2 Simpson,
// 3 Simpson 3/8, 4 Boole); every m >= 2 integrates cubics exactly
__host__ __device__ __forceinline__ double quad_omega(int quad, int m, int l) {
  if (m <= 0) return 0.0;
  if (quad == kQuadTrapezoid || m == 1) return (l == 0 || l == m) ? 0.5 : 1.0;
  if (m == 2) return l == 1 ? 4.0 / 3.0 : 1.0 / 3.0;
  if (m == 3) return (l == 0 || l == 3) ? 0.375 : 1.125;
  if (m == 4) return (l == 0 || l == 4) ? 14.0 / 45.0 : (l == 2 ? 24.0 / 45.0 : 64.0 / 45.0);
  const int e = l < m - l ? l : m - l;
  return e == 0 ? 0.375 : (e == 1 ? 7.0 / 6.0 : (e == 2 ? 23.0 / 24.0 : 1.0));
}

// ---- double2 complex helpers -------------------------------------------
__device__ __forceinline__ double2 c_make(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_scale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 c_neg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ double2 c_mulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc + a * b
__device__ __forceinline__ double2 c_fma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// i * a
__device__ __forceinline__ double2 c_i(double2 a) { return make_double2(-a.y, a.x); }
// fused forms, four FMAs each (signs and conjugates folded into the FMAs):
// acc + a * conj(b)
__device__ __forceinline__ double2 c_fmac(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.y, b.x, fma(-a.x, b.y, acc.y)));
}
// acc - a * b
__device__ __forceinline__ double2 c_fnma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// acc - a * conj(b)
__device__ __forceinline__ double2 c_fnmac(double2 a, double2 b, double2 acc) {
  return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.y, b.x, fma(a.x, b.y, acc.y)));
}

// Instantiated CUDA graphs keyed by the call shape they replay. At most kCap
// are kept; to make room the least recently used one is destroyed (a graph
// that is still running is freed by the runtime once it completes).
template <class Key>
struct GraphCache {
  static constexpr size_t kCap = 64;
  struct Entry {
    cudaGraphExec_t exec;
    unsigned long long used;
  };
  std::map<Key, Entry> m;
  unsigned long long clock = 0;
  cudaGraphExec_t find(const Key &k) {
    auto it = m.find(k);
    if (it == m.end()) return nullptr;
    it->second.used = ++clock;
    return it->second.exec;
  }
  void put(const Key &k, cudaGraphExec_t e) {
    if (m.size() >= kCap) {
      auto lru = m.begin();
      for (auto it = m.begin(); it != m.end(); ++it)
        if (it->second.used < lru->second.used) lru = it;
      cudaGraphExecDestroy(lru->second.exec);
      m.erase(lru);
    }
    m[k] = Entry{e, ++clock};
  }
  template <class Pred>
  void drop_if(Pred stale) {
    for (auto it = m.begin(); it != m.end();) {
      if (stale(it->first)) {
        cudaGraphExecDestroy(it->second.exec);
        it = m.erase(it);
      } else {
        ++it;
      }
    }
  }
  void clear() {
    for (auto &kv : m) cudaGraphExecDestroy(kv.second.exec);
    m.clear();
  }
  size_t size() const { return m.size(); }
};

// streaming multiprocessors of the current device (queried once per device,
// cached; grids are sized in multiples of it)
int device_sms();

// ---- float2 complex helpers (the complex64 form's FP32 arithmetic) --------
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_scale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 c_fma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
// conversions between the two complex types
template <class C>
__device__ __forceinline__ C c_from(double2 z);
template <>
__device__ __forceinline__ double2 c_from<double2>(double2 z) { return z; }
template <>
__device__ __forceinline__ float2 c_from<float2>(double2 z) { return make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ double2 c_widen(double2 z) { return z; }
__device__ __forceinline__ double2 c_widen(float2 z) { return make_double2(z.x, z.y); }

// A running sum of FP32 terms kept as an unevaluated pair hi + lo on the FP32
// pipe: every addition is Knuth's TwoSum (s = hi + x and its exact rounding
// error), the errors summed in lo. For the few tens of terms of a partial-sum
// reduction the pair carries the sum to about 2^-44 of its largest term, as an
// FP64 running sum would for FP32 terms, at FP32 rate (GB300 issues FP64 at
// 1/64 of it).
struct FSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---- history storage of one (G^<, dG) pair (see kbe_op_pack) --------------
// dG = G^< - G^> is formed in FP64 by the caller; o0 / o1 index the stored
// complex numbers of component 0 and 1
__device__ __forceinline__ float4 split_df(double2 x) {
  const float rh = __double2float_rn(x.x), ih = __double2float_rn(x.y);
  return make_float4(rh, __double2float_rn(x.x - (double)rh), ih, __double2float_rn(x.y - (double)ih));
}
// Split-FP16 pair history (KBE_PREC_F16X2): every stored complex number z is
// kept as hi = fp16(S z), lo = fp16(S z - hi) per real part, S =
// kF16HistScale (|G| <= 1 and |dG| <= 2, so S z stays far inside the FP16
// range; below 2^-16 the pair keeps an absolute error of 2^-25 / S). The
// layout is the tensor-core sweep's operand layout (kbe_sweep_tc.cu). Column
// blocks come in strips of TM = f16x2_tm(N_b); block (i, j) at k belongs to
// strip s = j / TM, and one "slot" of 16 N_b^2 TM bytes holds the strip's
// blocks of row i:
//   [r / 4][h][x][j % TM][s][r % 4][re/im]  halves
// (h: hi / lo part, x: G^< / dG, element (r, s) of the N_b x N_b matrix).
// Per k, the strips follow each other and each strip holds its rows
// s TM .. cap - 1 as consecutive slots, cap = the rows the storage holds. A
// group of consecutive rows of one strip is therefore one contiguous range:
// one bulk copy lands it in shared memory as core matrices of 8 rows x 16
// bytes. Padding slots (blocks beyond a row's end) are never written.
constexpr double kF16HistScale = 4096.0;
__host__ __device__ constexpr int f16x2_tm(int nb) { return nb == 4 ? 16 : 8; }
__host__ __device__ constexpr size_t f16x2_slot_halves(int nb) { return (size_t)8 * nb * nb * f16x2_tm(nb); }
// first slot of strip s within one k (strips hold rows s TM .. cap - 1)
__host__ __device__ inline size_t f16x2_colstart(int s, int cap, int nb) {
  return (size_t)s * cap - (size_t)f16x2_tm(nb) * s * (s - 1) / 2;
}
__host__ __device__ inline size_t f16x2_kslots(int cap, int nb) {
  return f16x2_colstart((cap - 1) / f16x2_tm(nb) + 1, cap, nb);
}
// slot of row i in strip s at k
__host__ __device__ inline size_t f16x2_slot(int i, int s, int k, int cap, int nb) {
  return (size_t)k * f16x2_kslots(cap, nb) + f16x2_colstart(s, cap, nb) + (size_t)(i - s * f16x2_tm(nb));
}
// halves from the storage start to element (h, x, r, s) of block (i, j) at k
__host__ __device__ inline size_t f16x2_index(int i, int j, int k, int h, int x, int r, int s, int nb, int cap) {
  const int tm = f16x2_tm(nb);
  return f16x2_slot(i, j / tm, k, cap, nb) * f16x2_slot_halves(nb) +
         ((((size_t)(r / 4) * 4 + (size_t)(h * 2 + x)) * tm + (size_t)(j % tm)) * nb + (size_t)s) * 8 +
         (size_t)(r % 4) * 2;
}
// bytes of a storage holding rows 0 .. cap - 1
__host__ __device__ inline size_t f16x2_history_bytes(int cap, int nb, int nk) {
  return (size_t)nk * f16x2_kslots(cap, nb) * f16x2_slot_halves(nb) * 2;
}
// (hi, lo) of S z as two half2 values (re, im)
__device__ __forceinline__ void f16x2_split(double2 z, __half2 &hi, __half2 &lo) {
  const double sr = z.x * kF16HistScale, si = z.y * kF16HistScale;
  const __half hr = __double2half(sr), hm = __double2half(si);
  hi = __halves2half2(hr, hm);
  lo = __halves2half2(__double2half(sr - (double)__half2float(hr)), __double2half(si - (double)__half2float(hm)));
}
__device__ __forceinline__ double2 f16x2_value(__half2 hi, __half2 lo) {
  return make_double2(((double)__low2float(hi) + (double)__low2float(lo)) / kF16HistScale,
                      ((double)__high2float(hi) + (double)__high2float(lo)) / kF16HistScale);
}
// element (r, s) of component x of block (i, j) at k, as complex128
// halves between the x planes of a slot (the h planes are twice as far apart)
__host__ __device__ constexpr size_t f16x2_xplane(int nb) { return (size_t)8 * nb * f16x2_tm(nb); }
__device__ __forceinline__ double2 f16x2_get(const __half *H, int i, int j, int k, int x, int r, int s, int nb,
                                             int cap) {
  const size_t o = f16x2_index(i, j, k, 0, x, r, s, nb, cap), lo = 2 * f16x2_xplane(nb);   // the h = 1 plane
  return f16x2_value(*reinterpret_cast<const __half2 *>(H + o), *reinterpret_cast<const __half2 *>(H + o + lo));
}
// the same in FP32 (hi + lo is exact in FP32: the pair spans 22 bits)
__device__ __forceinline__ float2 f16x2_getf(const __half *H, int i, int j, int k, int x, int r, int s, int nb, int cap) {
  const size_t o = f16x2_index(i, j, k, 0, x, r, s, nb, cap), lo = 2 * f16x2_xplane(nb);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(H + o));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(H + o + lo));
  constexpr float inv = (float)(1.0 / kF16HistScale);
  return make_float2((a.x + b.x) * inv, (a.y + b.y) * inv);
}
// block index bq of a triangle counted from row 0 -> (row, column)
__device__ __forceinline__ void tri_decode(size_t bq, int &i, int &j) {
  int ii = (int)((sqrt(8.0 * (double)bq + 1.0) - 1.0) / 2.0);
  while ((size_t)ii * (ii + 1) / 2 > bq) --ii;
  while ((size_t)(ii + 1) * (ii + 2) / 2 <= bq) ++ii;
  i = ii;
  j = (int)(bq - (size_t)ii * (ii + 1) / 2);
}
// o0 indexes component 0 of a block in the [block][x][r][s][k] numbering of the
// other forms (block bq = o0 / (2 blk)); dst is the storage start; row >= 0:
// the blocks are row `row` and bq its column, row < 0: bq counts from row 0
__device__ __forceinline__ void pack_store_f16x2(void *dst, size_t o0, int nb, int nk, int row, int cap, double2 gl,
                                                 double2 dg) {
  const size_t blk = (size_t)nb * nb * nk, bq = o0 / (2 * blk), rem = o0 - bq * 2 * blk;
  const int rs = (int)(rem / nk), k = (int)(rem - (size_t)rs * nk), r = rs / nb, s = rs - r * nb;
  int i = row, j = (int)bq;
  if (row < 0) tri_decode(bq, i, j);
  __half *H = (__half *)dst;
  const size_t o = f16x2_index(i, j, k, 0, 0, r, s, nb, cap), dx = f16x2_xplane(nb), lo = 2 * dx;
  __half2 hi, lw;
  f16x2_split(gl, hi, lw);
  *reinterpret_cast<__half2 *>(H + o) = hi;
  *reinterpret_cast<__half2 *>(H + o + lo) = lw;
  f16x2_split(dg, hi, lw);
  *reinterpret_cast<__half2 *>(H + o + dx) = hi;
  *reinterpret_cast<__half2 *>(H + o + dx + lo) = lw;
}
// nb, nk, row, cap: the mesh, the row of the blocks (< 0: a triangle from row
// 0) and the rows the storage holds (KBE_PREC_F16X2 only; dst is then the
// storage start)
__device__ __forceinline__ void pack_store(int prec, void *dst, size_t o0, size_t o1, double2 gl, double2 dg,
                                           int nb = 0, int nk = 0, int row = -1, int cap = 0) {
  if (prec == KBE_PREC_F16X2) {
    pack_store_f16x2(dst, o0, nb, nk, row, cap, gl, dg);
  } else if (prec == KBE_PREC_DF64) {
    ((float4 *)dst)[o0] = split_df(gl);
    ((float4 *)dst)[o1] = split_df(dg);
  } else if (prec == KBE_PREC_C64) {
    ((float2 *)dst)[o0] = make_float2((float)gl.x, (float)gl.y);
    ((float2 *)dst)[o1] = make_float2((float)dg.x, (float)dg.y);
  } else {
    ((double2 *)dst)[o0] = gl;
    ((double2 *)dst)[o1] = dg;
  }
}

// ---- status word written by kernels (sticky, read by the host) -----------
// kDevTimeoutDrain: after a timeout, the wait for a CTA's own copies in
// flight also ran out, so a copy may still land in shared memory that a later
// CTA owns: the handle's results can no longer be trusted, even after a reset
enum : int {
  kDevOk = 0,
  kDevNonFinite = 1,
  kDevEigNoConv = 2,
  kDevAdjUnsupported = 4,
  kDevTimeout = 8,
  kDevTimeoutDrain = 16
};

// ---- kernels launch wrappers (return cudaGetLastError()) ------------------
// a1 self-energy row
// raises the DFT kernel's shared-memory limit for an L0 x L1 mesh (host side)
cudaError_t dft_prepare(int L0, int L1);
// out[arr] = scale * DFT_sign(in[arr]) for narr arrays of n_k points (added
// to out when accumulate)
cudaError_t launch_dft_rows(const double2 *in, double2 *out, long narr, int L0, int L1, int sign,
                            double scale, cudaStream_t st, bool accumulate = false,
                            const int *skip = nullptr);
// skip (device int, may be NULL): when it holds non-zero the launch does
// nothing (the corrector passes of a converged step, Algorithm 1's break).
cudaError_t launch_sigma_products(const Mesh &m, const double *v, int n, double Un,
                                  const double *Ul_dev, const double2 *GR, double2 *SR,
                                  cudaStream_t st, const int *skip = nullptr);
size_t sigma_workspace_bytes(const Mesh &m, int n);
// fp32: the transforms and products in complex FP32 (the complex64 history
// form, whose coefficient rows round Sigma to complex64 anyway); Sig is FP64
// fp32: complex64 transforms and products. Hrow32 (fp32 only, may be NULL):
// row n as complex64 (G^<, dG) pairs, read instead of Grow. sig32: Sig is
// written as complex64 (the coefficient rows of the complex64 and split-FP16
// sweeps read it so: launch_sweep's sig32)
cudaError_t sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                      const double2 *Grow, double2 *Sig, double2 *work, cudaStream_t st,
                      const int *skip = nullptr, bool fp32 = false, const float2 *Hrow32 = nullptr,
                      bool sig32 = false);

// a2 collision row. H is the history triangle in the precision's storage
// (double2 / float4 hi-lo pairs / float2), each block holding G^< and
// dG = G^< - G^>; work holds the coefficient rows and the l-split partial
// sums (sweep_workspace_bytes).
bool sweep_supported(int nb);
bool use_f64m(const Mesh &m, int prec);   // the FP64 sweep takes the three-multiplication kernel
bool precision_supported(int prec);
size_t history_elem_bytes(int prec);
size_t sweep_workspace_bytes(const Mesh &m, int n, int prec);
int sweep_splits(const Mesh &m, int n, int prec, int quad);   // CTAs sharing one output's l range
// autotuner of the l-split (see kbe_sweep.cu); out[b] per row bucket b
cudaError_t tune_sweep(const Mesh &m, int prec, int quad, int nmax, double dt, const void *H, const double2 *Sig,
                       double2 *I, void *work, cudaStream_t st, int *out, int nout, int cap = 0);
cudaError_t sweep_prepare(int nb);   // kernel attributes, host side (before stream capture)
// set (choice != 0) or clear (0) the tuned launch choice of a sweep shape for
// row bucket `bucket` (-1: all); false if the choice does not apply
bool set_sweep_choice(const Mesh &m, int prec, int quad, int bucket, int choice);
// the single-read complex64 sweep (kbe_sweep_tile.cu): N_b in {2, 4, 8}, n_k
// even; TI rows per work item; part holds its partial sums (tile_part_bytes)
bool tile_supported(const Mesh &m, int prec);
size_t tile_part_bytes(const Mesh &m, int n, int TI);
cudaError_t tile_prepare(int nb);
cudaError_t launch_sweep_tile(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part,
                              cudaStream_t st, const int *skip, int quad, int *status, int TI);
// the tensor-core sweep of the split-FP16 form (kbe_sweep_tc.cu): N_b in {4, 8};
// TI rows per panel (a multiple of 16, at most tc_max_ti); part holds its
// coefficient operands and partial sums (tc_part_bytes), headed by the word
// that receives coef_kernel's largest |coefficient| (tc_cmax_word)
bool tc_supported(const Mesh &m, int prec);
int tc_max_ti(int nb);
size_t tc_part_bytes(const Mesh &m, int n, int TI);
unsigned *tc_cmax_word(void *part);
double tc_tensor_flops(const Mesh &m, int n, int TI);   // tensor-core flops of one launch at row n
// the tensor-core flops one sweep launch executes at row n with the panel
// height the sweep will use (0 unless the form is the tensor-core one)
double sweep_tc_flops(const Mesh &m, int prec, int quad, int n);
cudaError_t tc_prepare(int nb);
cudaError_t launch_sweep_tc(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part,
                            cudaStream_t st, const int *skip, int quad, int *status, int TI, int cap);
// nb: the mesh's N_b (required by KBE_PREC_F16X2, whose layout needs it);
// row >= 0: the blocks are row `row` and dst is that row's start
// (history_row_offset), row < 0: a triangle from row 0 and dst its start;
// cap: the rows the storage holds (F16X2)
cudaError_t launch_pack(int prec, const double2 *src, void *dst, size_t nblocks, size_t blk,
                        cudaStream_t st, const int *skip = nullptr, int nb = 0, int row = -1, int cap = 0);
// byte offset of row i in the history (0 for F16X2, whose rows are spread
// over the strips: its kernels address the whole storage), and the bytes of
// a storage for rows 0 .. n
size_t history_row_offset(const Mesh &m, int prec, int i);
size_t history_bytes(const Mesh &m, int prec, int n);
// component `which` of nblk blocks into [j][k][a][b]: from the FP64 working
// row when fp64 != NULL, else from the history storage of precision prec
cudaError_t launch_row_out(int prec, const double2 *fp64, const void *packed, size_t nblk, const Mesh &m,
                           int which, double2 *out, cudaStream_t st, int row = -1, int cap = 0);
// status (may be NULL): device word that receives kDevTimeout if a staged
// copy never completes (bounded waits)
// inject (test only): 1 makes the staged C64 sweep's first CTA omit its first
// node's copies, so that its bounded waits run out (kDevTimeout), no fault
// One system's FP64 collision sweep, prepared (coefficient rows enqueued) for a
// batched launch with other systems' sweeps (kbe_batch): its operands, its
// launch shape (k tiles x columns x l-splits) and where its partials go.
struct SweepJob {
  const double2 *H, *Cf;
  const double *Cs;
  double2 *out, *I;
  const int *skip;
  int n, nk, nb, quad, lchunk, nz, tx, threads, f64m;
};
cudaError_t prepare_sweep_job(const Mesh &m, int n, double dt, const void *H, const double2 *Sig, double2 *I,
                              void *work, cudaStream_t st, const int *skip, int quad, SweepJob *job);
// the sweeps of many jobs: one persistent launch per (N_b, quadrature, form)
cudaError_t launch_sweep_batch(const SweepJob *jobs, int njobs, cudaStream_t st, int *launches);
// the job's partial sums into its I row (when its l range was split)
cudaError_t finish_sweep_job(const SweepJob &job, cudaStream_t st);
}  // namespace kbe
// a step of a handle in segments that stop at each collision sweep (kbe_api.cu;
// used by kbe_batch.cu): segment 0 .. step_segment_count - 1; a segment with
// *has_job hands back its sweep, which must run before the next segment
struct kbe_handle;
int step_segment_count(const kbe_handle *h);
kbe_status step_segment(kbe_handle *h, int seg, kbe::SweepJob *job, bool *has_job);
kbe_status step_segment_check(kbe_handle *h);
namespace kbe {
// cap: the rows H holds (the F16X2 layout depends on it; <= 0: n + 1)
cudaError_t launch_sweep(const Mesh &m, int n, double dt, int precision, const void *H,
                         const double2 *Sig, double2 *I, void *work, cudaStream_t st,
                         const int *skip = nullptr, int quad = kQuadTrapezoid, int *status = nullptr,
                         int inject = 0, int cap = 0, bool sig32 = false);

// a3 propagators / initial state / density
struct HopTable {
  int nhop;
  const int *R;        // device [nhop][2]
  const double2 *T;    // device [nhop][nb][nb]
  double d0, d1;       // drive direction
};
cudaError_t launch_init_state(const Mesh &m, const HopTable &hop, double beta, double mu,
                              double2 *H00, int *status, cudaStream_t st);
cudaError_t launch_local_density(const Mesh &m, const double2 *Gdiag, double2 *rho_out,
                                 cudaStream_t st, const int *skip = nullptr);
struct PropParams {
  double A;                     // Peierls sample for this step
  const double2 *rho_a;         // device nb*nb, mid density = ca*rho_a + cb*rho_b
  const double2 *rho_b;
  double ca, cb;
  double Umid;
  int hf, paper_shift;
  double v[kMaxNb * kMaxNb];
  const double2 *dipM;          // device nb*nb dipole coupling (Eq. 4), or NULL
  double dipE;                  // its field sample for the step
};
// h for the step (from the hopping table, mean field and shift; or h_in when
// not NULL, then hop / p are unused), U = e^{-i dt h}, V = (U - 1) h^{-1};
// h_out (may be NULL) receives h. All per-k [a][b][k].
cudaError_t launch_build_props(const Mesh &m, const HopTable &hop, const PropParams &p, double dt,
                               const double2 *h_in, double2 *h_out, double2 *U, double2 *V,
                               cudaStream_t st, const int *skip = nullptr);

// a4 update: rows j < n and the time diagonal (h, U, V of the step).
// maxdiff (may be NULL): max over the new row of |G^< - its previous value in
// out| is folded in (atomicMax on the bits of a non-negative double).
// packed (may be NULL): the history's row n in the storage of precision prec,
// written with the row ((G^<, dG) per block, as kbe_op_pack would); for
// KBE_PREC_F16X2 the storage start, holding cap rows.
cudaError_t launch_update_row(const Mesh &m, int n, double dt, double theta, const double2 *h,
                              const double2 *U, const double2 *V, const double2 *Gprev,
                              const double2 *Iprev, const double2 *Icur, double2 *out,
                              cudaStream_t st, const int *skip = nullptr,
                              unsigned long long *maxdiff = nullptr, void *packed = nullptr, int prec = 0,
                              int cap = 0);
// Algorithm 1's convergence test after a corrector pass (one thread): unless
// skip is set, count the pass in *iters, set skip when *maxdiff <= tol, and
// clear *maxdiff for the next pass.
cudaError_t launch_corr_check(unsigned long long *maxdiff, double tol, int *skip, int *iters,
                              cudaStream_t st);

// a5 observables
struct ObsParams {
  double Abar, Un;
  int hf, paper_shift;
  double v[kMaxNb * kMaxNb];
};
// part: 3 doubles per CTA (at most n_k CTAs); ticket: one zeroed word
cudaError_t launch_observables(const Mesh &m, const HopTable &hop, const ObsParams &p,
                               const double2 *Gdiag, const double2 *Idiag, const double2 *rho_n,
                               double *obs_out, double *nkb_out, int *status, double *part, unsigned *ticket,
                               cudaStream_t st);

// reverse mode (FP64 history; see kbe_adjoint.cu). Rows are [l][x][a][b][k]
// with x = (G^<, G^>) or their adjoints.
// (G^<, dG) history blocks -> (G^<, G^>)
cudaError_t launch_unpack_fp64(const double2 *packed, double2 *out, size_t nblocks, size_t blk,
                               cudaStream_t st);
// transpose of the collision row at n: lamSig = lambda of the Sigma row;
// lamH (blocks of rows < n) and lamRowN (row n) += lambda of the history
// blocks the sweep read (H holds row n as that sweep saw it). c1_work holds
// (n+1) blocks (the C1 coefficients).
size_t adj_coef_workspace_bytes(const Mesh &m, int nmax);
cudaError_t launch_adj_sweep(const Mesh &m, int n, double dt, const double2 *H, const double2 *Sig,
                             const double2 *lamI, double2 *lamSig, double2 *lamH, double2 *lamRowN,
                             double2 *coef_work, double2 *c1_work, cudaStream_t st,
                             int quad = kQuadTrapezoid);
// transpose of the Sigma row (factor -U_n U_l, Ul_dev NULL: U_l = U_n): lamRow
// += lambda of the G row; gU[i] += dL/dU_i (gU[n] only when Ul_dev is NULL)
size_t adj_sigma_workspace_bytes(const Mesh &m, int n);
cudaError_t adj_sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                          const double2 *Grow, const double2 *lamSig, double2 *lamRow, double *gU,
                          double2 *work, cudaStream_t st);
// transpose of the row and diagonal update: lamGprev, lamIp, lamIc +=;
// lamh (per k) = lambda of the step's h through U, V and the diagonal
size_t adj_update_workspace_bytes(const Mesh &m);
cudaError_t launch_adj_update(const Mesh &m, int n, double dt, double theta, const double2 *h,
                              const double2 *U, const double2 *V, const double2 *Gprev, const double2 *Ip,
                              const double2 *Ic, const double2 *lam, double2 *lamGprev, double2 *lamIp,
                              double2 *lamIc, double2 *lamh, double2 *work, int *status, cudaStream_t st);
// transpose of h = h0(k - A d) + U hf(mid) + shift: dL/dA, dL/dU and the
// lambda of the mid density (to rho_a, rho_b or a G^<(n,n) block)
struct AdjHvecArgs {
  double A, U;
  int hf, paper_shift;
  const double2 *rho_a, *rho_b;
  double ca, cb;
  double2 *lam_rho_a, *lam_rho_b, *lam_cur;
  double cur_scale;
  double *gA, *gU_a, *gU_b;   // dL/dU_mid is split evenly between U_{n-1} and U_n
};
cudaError_t launch_adj_hvec(const Mesh &m, const HopTable &hop, const AdjHvecArgs &a, const double *v_host,
                            const double2 *lamh, cudaStream_t st);
// lamDiag[e][k] += i scale lamRho[e]
cudaError_t launch_adj_density(const Mesh &m, const double2 *lamRho, double scale, double2 *lamDiag,
                               cudaStream_t st);
// message returned by kbe_last_error(NULL) on this thread
void set_last_error(const std::string &msg);
// kbe_step in pieces, for a graph that spans the steps of several handles
kbe_status step_check(kbe_handle *h, int nsteps);
bool step_capturable(const kbe_handle *h);
kbe_status step_prepare(kbe_handle *h);
kbe_status step_record(kbe_handle *h, int nsteps);
void step_advance(kbe_handle *h, int nsteps);
void step_key(const kbe_handle *h, int *ring, unsigned *gen);
// the host-side step state (row, I-ring order), saved before a capture that
// records steps and put back after it
struct StepMark {
  int n;
  void *Ip, *Ic;
};
StepMark step_mark(const kbe_handle *h);
void step_rewind(kbe_handle *h, const StepMark &mk);
cudaStream_t handle_stream(const kbe_handle *h);
int handle_precision(const kbe_handle *h);

}  // namespace kbe
