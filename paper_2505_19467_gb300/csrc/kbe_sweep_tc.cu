// (a2) Collision-integral sweep on the fifth-generation tensor cores
// (tcgen05.mma), for the split-FP16 pair history (KBE_PREC_F16X2), Eq. 6 in
// left form.
//
// Per k the sweep is a chain of N_b x N_b complex products over the stored
// triangle. Every stored block B = (G^<, dG)(t_i, t_m), i > m, has two uses:
//   column use (output column m, node i):  X(m) += C1(i) B^<,  Y(m) -= C1(i) dB
//   row use (output column i, node m):     X(i) -= C1(m) conj(B^<)^T + f C2^<(m) conj(dB)^T
// with X = I^<, Y = I^> - I^<, C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<, f =
// w^(i)_m / dt (1 in the interior). Both become MMAs with the history as the
// A operand (M = 128 rows) and the coefficients as the B operand (N = 4 N_b):
//   column use: rows (x, m, s) of a strip of TM columns (x = G^< / dG),
//     K = (r, re/im) of row i; the complex product is expanded on the B side
//     (N = (part, a, re/im), with the signs of C1 placed in B);
//   row use: rows (i, r, re/im) of a group of RG rows, K = (x, m, s) of the
//     strip; expanded on the A side, the epilogue combining the four real
//     products of conj(B) C.
// The history is stored in this operand layout (kbe_internal.cuh, F16X2): for
// each row and k, the blocks of a strip of TM columns form one contiguous
// slot, [r / 4][h][x][block][s][r % 4][re/im], so one bulk copy
// (cp.async.bulk) lands a row segment in shared memory as core matrices of 8
// rows x 16 bytes that are K-major for the column use and MN-major for the
// row use (canonical no-swizzle layouts: LBO = K-direction, SBO =
// MN-direction core-matrix stride).
// Each value is split in two FP16 parts (hi, lo), the history under the fixed
// scale 2^12, the coefficients under a power-of-two scale from the row's
// largest |C1|, |C2^<| (coef_kernel); the two A parts are two MMAs into the
// same accumulator, the two B parts two halves of N, so the accumulator holds
// (A_hi + A_lo)(C_hi + C_lo) in FP32: a ~22-bit product at FP16 tensor rate.
//
// Work unit: a panel of TI rows [R0, R1) and one k. A persistent CTA walks
// the panel strip by strip (columns [M0, M0 + TM), M0 <= R1 - 1), each strip
// in groups of RG rows through a two-set ring of row segments:
//   warp 0     copy producer: the strip's coefficient tiles (B of the row
//              use), each row's segment and its coefficient tile (B of the
//              column use), all by bulk copies completing on mbarriers;
//   warp 1     MMA issuer: zeroes the blocks on and above the diagonal in
//              the strips that reach it, issues the column-use MMAs (into a
//              per-strip accumulator, double-buffered) and the row-use MMAs
//              (into one accumulator per row group, kept across the whole
//              panel), and frees ring slots with tcgen05.commit;
//   warps 2-5  epilogue: tensor memory -> registers -> complex64 partial
//              sums: one column partial per (panel, column, k), one row
//              partial per (row, k).
// tc_reduce_kernel then sums the partials (hi + lo FP32 pairs) and adds what the MMAs leave
// out: the diagonal block (the end node of column j), the row use's weights
// f != 1 (trapezoid: node 0; Gregory: its end nodes) and the Gregory Y terms.
//
// Every wait is bounded (one second of %globaltimer): a copy or MMA that never
// completes marks kDevTimeout in the status word and the CTA winds down.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "kbe_internal.cuh"
#include "kbe_tma.cuh"

namespace kbe {

namespace {

// TM columns per strip (x-stacked column-use M = 2 TM N_b = 128), RG rows per
// group (row-use M = 2 RG N_b = 128)
template <int NB>
struct TcCfg;
// NC independent column-use accumulators per strip buffer: back-to-back MMAs
// into one accumulator wait on each other (~57 ns each at N <= 128 on
// GB300), so consecutive MMAs alternate between accumulators (and between the
// column and row uses), which the epilogue sums
// SETS row groups in flight in the shared-memory ring (three fit at N_b = 4)
template <>
struct TcCfg<4> {
  static constexpr int TM = 16, RG = 16, NC = 4, SETS = 3;
};
template <>
struct TcCfg<8> {
  static constexpr int TM = 8, RG = 8, NC = 2, SETS = 2;
};

// warp 0 bulk copies, warp 1 MMA, warps 2-5 epilogue; with WC, warps 6-9 copy
// the row segments with 16-byte cp.async (many small requests in flight)
// instead of one bulk copy per row group
constexpr int kTcLoaders = 128;
// the row-use accumulators are drained every tc_sd strips (complex64 partial
// per (strip group, row, k)), which bounds their FP32 chains: 4 strips of 128
// K-terms at N_b = 8, 16 strips of 128 at N_b = 4 (whose full-panel chains
// were already within the mixed bar; every drain is a wait of the MMA warp)
__host__ __device__ constexpr int tc_sd(int nb) { return nb == 8 ? 4 : 16; }
__host__ __device__ constexpr int tc_threads(bool wc) { return wc ? 192 + kTcLoaders : 192; }

// the row use reads the slot ring as an MN-major A operand: core matrices
// 4096 bytes apart along M (rows, or r halves at N_b = 8), 128 apart along K
#ifndef KBE_TC_MN_LBO
#define KBE_TC_MN_LBO 128u
#endif
#ifndef KBE_TC_MN_SBO
#define KBE_TC_MN_SBO 4096u
#endif

template <int NB>
__host__ __device__ constexpr int tc_n() { return 4 * NB; }   // MMA N: (part, a, re/im)
template <int NB>
__host__ __device__ constexpr unsigned tc_slot() { return 16u * NB * NB * TcCfg<NB>::TM; }   // A bytes per row
template <int NB>
__host__ __device__ constexpr unsigned tc_bcol() { return 16u * NB * NB; }   // column-use B bytes per row
template <int NB>
__host__ __device__ constexpr unsigned tc_brow() { return 16u * NB * NB * TcCfg<NB>::TM; }   // row-use B per strip
template <int NB>
__host__ __device__ constexpr unsigned tc_btile() { return 64u * NB; }   // one row-use B tile (column or column pair)
// ring of A slots and column-use B tiles, two row-use B buffers, one zero
// column-use B tile (the operand of the MMAs that clear unused accumulators)
template <int NB>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return (size_t)TcCfg<NB>::SETS * TcCfg<NB>::RG * (tc_slot<NB>() + tc_bcol<NB>()) + 2 * (size_t)tc_brow<NB>() +
         tc_bcol<NB>();
}
static_assert(tc_smem_bytes<4>() + 1024 <= 227 * 1024 && tc_smem_bytes<8>() + 1024 <= 227 * 1024, "tc smem");

// byte offsets inside one row slot: the h (hi / lo) planes are 2048 bytes
// apart; column-use K-direction (next row at N_b = 4, next r half at 8) and
// row-use M-direction core matrices are 4096 apart; consecutive (x, m)
// core-matrix groups are 128 apart
constexpr unsigned kTcPlane = 2048, kTcFar = 4096, kTcCore = 128;

// ---- tcgen05 helpers ---------------------------------------------------
// shared-memory matrix descriptor, no swizzle: start, LBO, SBO (bytes)
__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16 with FP16 A and B, FP32 accumulator,
// M = 128, N; A K-major (0) or MN-major (1), B K-major
__host__ __device__ constexpr uint32_t tc_idesc(int N, int amn) {
  return (1u << 4) | ((uint32_t)amn << 15) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// power-of-two scale of the coefficient parts: max |C| * S < 2^14
__device__ __forceinline__ float tc_coef_scale(const unsigned *cmax) {
  const float big = __uint_as_float(*cmax);
  if (!(big > 0.f) || !(big < 3.0e38f)) return 1.f;
  int e = 0;
  frexpf(big, &e);   // big < 2^e
  return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ void split16(float v, __half &hi, __half &lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// ---- coefficient operands ---------------------------------------------
// Bc [k][l][tile]: the column-use B of row l (K-major, core matrices of 8
// N-rows x 8 K-halves): K = (r, re/im) (N_b = 8: two K halves r < 4, r >= 4),
// N-row nr = (part, a, re/im out); value (C1 of row l expanded):
//   out re: C1r[a][r] (in re), -C1i[a][r] (in im); out im: C1i (in re), C1r (in im).
// Br [x][k][t][tile]: the row-use B for column l (N_b = 8, t = l) or the
// column pair l = 2t, 2t + 1 (N_b = 4): K = s (N_b = 8) or (l - 2t, s);
// value C1 (x = 0) or C2^< (x = 1) at [a][s], part re/im; zero for l > n.
template <int NB>
__global__ void tc_coef_kernel(const float2 *__restrict__ Cf, const unsigned *__restrict__ cmax, __half *__restrict__ Bc,
                               __half *__restrict__ Br, int n, int nk, int lt, const int *__restrict__ skip) {
  if (skip && *skip) return;
  constexpr int N = tc_n<NB>(), KH = 2 * NB / 8;   // K chunks of 8 halves per column-use row
  const size_t blk = (size_t)NB * NB * nk;
  const float sc = tc_coef_scale(cmax);
  const size_t ncol = (size_t)nk * (n + 1) * N * KH, nrow = (size_t)2 * nk * lt * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < ncol + nrow;
       idx += (size_t)gridDim.x * blockDim.x) {
    __half out[8];
    __half *dst;
    if (idx < ncol) {   // (k, l, kh, nr): one 16-byte row of a core matrix
      const int nr = (int)(idx % N);
      size_t q = idx / N;
      const int kh = (int)(q % KH);
      q /= KH;
      const int l = (int)(q % (n + 1)), k = (int)(q / (n + 1));
      const int part = nr / (2 * NB), a = (nr % (2 * NB)) / 2, ro = nr & 1;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = kh * 4 + e / 2, ri = e & 1;
        const float2 c = Cf[(size_t)l * 3 * blk + (size_t)(a * NB + r) * nk + k];
        const float v = ro == 0 ? (ri == 0 ? c.x : -c.y) : (ri == 0 ? c.y : c.x);
        __half hi, lo;
        split16(v * sc, hi, lo);
        out[e] = part ? lo : hi;
      }
      dst = Bc + (((size_t)k * (n + 1) + l) * (tc_bcol<NB>() / 2)) + (size_t)kh * (N * 8) + (size_t)nr * 8;
    } else {            // (x, k, t, nr)
      size_t q = idx - ncol;
      const int nr = (int)(q % N);
      q /= N;
      const int t = (int)(q % lt);
      q /= lt;
      const int k = (int)(q % nk), x = (int)(q / nk);
      const int part = nr / (2 * NB), a = (nr % (2 * NB)) / 2, rc = nr & 1;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int l = NB == 8 ? t : 2 * t + e / 4, sidx = NB == 8 ? e : e % 4;
        float v = 0.f;
        if (l <= n) {
          const float2 c = Cf[((size_t)l * 3 + x) * blk + (size_t)(a * NB + sidx) * nk + k];
          v = rc ? c.y : c.x;
        }
        __half hi, lo;
        split16(v * sc, hi, lo);
        out[e] = part ? lo : hi;
      }
      dst = Br + (((size_t)x * nk + k) * lt + t) * (tc_btile<NB>() / 2) + (size_t)nr * 8;
    }
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(out);
  }
}

// ---- the sweep -----------------------------------------------------------
// CP [panel][j][k][x][a][b], RP [j][k][a][b] (complex64)
template <int NB, bool WC>
__global__ void __launch_bounds__(tc_threads(WC), 1)
    sweep_tc_kernel(const __half *__restrict__ Hh, const __half *__restrict__ Bcg,
                    const __half *__restrict__ Brg, const unsigned *__restrict__ cmax, float2 *__restrict__ CP,
                    float2 *__restrict__ RP, int n, int nk, int TI, int lt, uint32_t tcols, int NR, int cap,
                    const int *__restrict__ skip, int *status) {
  if (skip && *skip) return;
  constexpr int TM = TcCfg<NB>::TM, RG = TcCfg<NB>::RG, N = tc_n<NB>(), NG = NB / 2, NC = TcCfg<NB>::NC;
  constexpr int SETS = TcCfg<NB>::SETS, SD = tc_sd(NB);
  constexpr unsigned SLOT = tc_slot<NB>(), BCOL = tc_bcol<NB>(), BROW = tc_brow<NB>();
  constexpr int CSTEP = 8 / NB;   // row slots per column-use MMA (K = 16 halves)
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char *sA = tc_smem;
  unsigned char *sBc = sA + (size_t)SETS * RG * SLOT;
  unsigned char *sBr = sBc + (size_t)SETS * RG * BCOL;
  unsigned char *sZero = sBr + 2 * (size_t)BROW;   // a zero column-use B tile
  __shared__ __align__(8) uint64_t full[SETS], empty[SETS], brf[2], bre[2], dcf[2], dce[2], drf, dre, done;
  static_assert(SETS <= 3, "slot sets");
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = (n + TI) / TI;   // panels of TI rows
  const int units = P * nk;

  // zero the ring (stale slots then always hold finite values), barriers, TMEM
  for (size_t o = (size_t)threadIdx.x * 16; o < (size_t)SETS * RG * (SLOT + BCOL); o += (size_t)blockDim.x * 16)
    *reinterpret_cast<uint4 *>(sA + o) = make_uint4(0, 0, 0, 0);
  for (unsigned o = threadIdx.x * 16; o < BCOL; o += blockDim.x * 16)
    *reinterpret_cast<uint4 *>(sZero + o) = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (threadIdx.x == 0) {
    for (int q = 0; q < SETS; ++q) {
      mbar_init(&full[q], WC ? 1 + kTcLoaders : 1);   // (WC: the loaders' cp.async arrivals too)
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&brf[q], 1);
      mbar_init(&bre[q], 1);
      mbar_init(&dcf[q], 1);
      mbar_init(&dce[q], 4);
    }
    mbar_init(&drf, 1);
    mbar_init(&dre, 4);
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tbase)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  auto fail = [&](int code) {
    abort_flag = 1;
    if (status) atomicOr(status, code);
  };
  auto wait = [&](uint64_t *bar, unsigned parity) -> bool {
    if (abort_flag) return false;
    if (mbar_wait(bar, parity, kMbarWaitLimit)) return true;
    fail(kDevTimeout);
    return false;
  };

  if (warp == 0) {
    // ------------------------------------------------------------- copies
    if (lane == 0) {
      int gcount = 0, scount = 0;
      for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
        const int p = P - 1 - u / nk, k = u % nk;
        const int R0 = p * TI, R1 = min(R0 + TI, n + 1);
        const int S = (R1 - 1) / TM + 1;
        for (int s = 0; s < S && !abort_flag; ++s, ++scount) {
          const int M0 = s * TM, b = scount & 1, use = scount >> 1;
          if (use >= 1 && !wait(&bre[b], (unsigned)((use - 1) & 1))) break;
          mbar_expect_tx(&brf[b], BROW);
          for (int x = 0; x < 2; ++x)
            bulk_load(sBr + (size_t)b * BROW + (size_t)x * (BROW / 2),
                      Brg + (((size_t)x * nk + k) * lt + (size_t)M0 * NB / 8) * (tc_btile<NB>() / 2), BROW / 2,
                      &brf[b]);
          for (int G0 = max(R0, M0); G0 < R1 && !abort_flag; G0 += RG, ++gcount) {
            const int set = gcount % SETS, use2 = gcount / SETS;
            if (use2 >= 1 && !wait(&empty[set], (unsigned)((use2 - 1) & 1))) break;
            const int rows = min(RG, R1 - G0);
            // the group's row segments of strip s are consecutive slots of the history,
            // and its column-use coefficient tiles consecutive tiles: two bulk copies
            mbar_expect_tx(&full[set], (unsigned)rows * ((WC ? 0 : SLOT) + BCOL));
            if (!WC)
              bulk_load(sA + (size_t)set * RG * SLOT, Hh + f16x2_slot(G0, s, k, cap, NB) * (SLOT / 2),
                        (unsigned)rows * SLOT, &full[set]);
            bulk_load(sBc + (size_t)set * RG * BCOL, Bcg + ((size_t)k * (n + 1) + G0) * (BCOL / 2),
                      (unsigned)rows * BCOL, &full[set]);
          }
        }
      }
      // let the copies in flight land before the CTA can exit (the last group of each set)
      for (int last = gcount - 1; last >= 0 && last >= gcount - SETS; --last)
        if (!mbar_wait(&full[last % SETS], (unsigned)((last / SETS) & 1), kMbarWaitLimit) && status)
          atomicOr(status, kDevTimeout | kDevTimeoutDrain);
      if (scount > 0) {
        const int last = scount - 1;
        if (!mbar_wait(&brf[last & 1], (unsigned)((last >> 1) & 1), kMbarWaitLimit) && status)
          atomicOr(status, kDevTimeout | kDevTimeoutDrain);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    const uint32_t id_col = tc_idesc(N, 0), id_row = tc_idesc(N, 1);
    const unsigned aBase = smem_addr(sA);
    const uint64_t descA_col = tc_desc(aBase, kTcFar, kTcCore);
    const uint64_t descB_col = tc_desc(smem_addr(sBc), (unsigned)NG * kTcCore, kTcCore);
    const uint64_t descA_row = tc_desc(aBase, KBE_TC_MN_LBO, KBE_TC_MN_SBO);
    const uint64_t descB_row = tc_desc(smem_addr(sBr), (unsigned)NG * kTcCore, kTcCore);
    int gcount = 0, scount = 0, dcount = 0;   // dcount: row-use drains so far
    for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
      const int p = P - 1 - u / nk;
      const int R0 = p * TI, R1 = min(R0 + TI, n + 1);
      const int S = (R1 - 1) / TM + 1;
      for (int s = 0; s < S && !abort_flag; ++s, ++scount) {
        const int M0 = s * TM, b = scount & 1, use = scount >> 1;
        // a strip group starts: its row-use accumulators are overwritten once drained
        if (s % SD == 0 && dcount >= 1 && !wait(&dre, (unsigned)((dcount - 1) & 1))) break;
        if (!wait(&brf[b], (unsigned)(use & 1))) break;
        if (use >= 1 && !wait(&dce[b], (unsigned)((use - 1) & 1))) break;
        tc_fence_after();
        unsigned colinit = 0;   // column-use accumulators written in this strip
        for (int G0 = max(R0, M0); G0 < R1 && !abort_flag; G0 += RG, ++gcount) {
          const int set = gcount % SETS, use2 = gcount / SETS, gi = (G0 - R0) / RG;
          const int rows = min(RG, R1 - G0);
          if (!wait(&full[set], (unsigned)(use2 & 1))) break;
          // blocks on and above the diagonal (m >= i) of rows i < M0 + TM take no part
          for (int r = 0; r < rows; ++r) {
            const int i = G0 + r;
            if (i >= M0 + TM) break;
            unsigned char *dA = sA + (size_t)(set * RG + r) * SLOT;
            const int m0 = i - M0;   // first local column to clear
            if (NB == 4) {           // [h][x][m/2][(m%2, s) rows][16 B]: 64 bytes per (plane, column)
              const int pieces = 4 * (TM - m0) * 4;   // 16-byte pieces
              for (int q = lane; q < pieces; q += 32) {
                const int pl = q / ((TM - m0) * 4), rem = q % ((TM - m0) * 4);
                const int ml = m0 + rem / 4, row = rem % 4;
                *reinterpret_cast<uint4 *>(dA + pl * 1024 + (ml / 2) * 128 + (ml % 2) * 64 + row * 16) =
                    make_uint4(0, 0, 0, 0);
              }
            } else {   // [ch][hx][m][s][16 B]: 128 bytes per (plane, column)
              const int pieces = 8 * (TM - m0) * 8;
              for (int q = lane; q < pieces; q += 32) {
                const int pl = q / ((TM - m0) * 8), rem = q % ((TM - m0) * 8);
                const int ml = m0 + rem / 8, row = rem % 8;
                *reinterpret_cast<uint4 *>(dA + (pl >> 2) * kTcFar + (pl & 3) * 1024 + ml * 128 + row * 16) =
                    make_uint4(0, 0, 0, 0);
              }
            }
          }
          if (NB == 4 && (rows & 1)) {   // the column-use MMA of the last row pairs it with a zero coefficient tile
            unsigned char *dB = sBc + (size_t)(set * RG + rows) * BCOL;
            for (int q = lane; q < (int)BCOL / 16; q += 32) *reinterpret_cast<uint4 *>(dB + q * 16) = make_uint4(0, 0, 0, 0);
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            tc_fence_after();
            const uint32_t dcol = tmem + (uint32_t)(b * NC * N), drow = tmem + (uint32_t)((2 * NC + gi * NR) * N);
            const int ncm = (rows + CSTEP - 1) / CSTEP;
            // descriptors advance by (byte offset >> 4) in their start-address field
            const uint64_t dAc = descA_col + ((unsigned)(set * RG) * SLOT >> 4);
            const uint64_t dBc = descB_col + ((unsigned)(set * RG) * BCOL >> 4);
            const uint64_t dAr = descA_row + ((unsigned)(set * RG) * SLOT >> 4);
            const uint64_t dBr = descB_row + ((unsigned)b * BROW >> 4);
            // column use: (h, cm) -> accumulator (h * ncm + cm) % NC; row use: (h, t) ->
            // accumulator t % NR; the two uses alternate so that independent MMAs follow
            // each other
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                if (q < ncm) {
                  const int c = (h * ncm + q) % NC;
                  tc_mma(dcol + (uint32_t)(c * N), dAc + ((unsigned)(q * CSTEP) * SLOT + h * kTcPlane >> 4),
                         dBc + ((unsigned)(q * CSTEP) * BCOL >> 4), id_col, (colinit >> c) & 1);
                  colinit |= 1u << c;
                }
                tc_mma(drow + (uint32_t)((q % NR) * N), dAr + (h * kTcPlane + 2u * q * kTcCore >> 4),
                       dBr + (2u * q * NG * kTcCore >> 4), id_row, (s % SD == 0 && h == 0 && q < NR) ? 0 : 1);
              }
            tc_commit(&empty[set]);
          }
          __syncwarp();
        }
        if (lane == 0) {
          // accumulators no MMA of this strip reached: clear them with the zero
          // tile as both operands (every core matrix read from the same 128 zero bytes)
          for (int c = 0; c < NC; ++c)
            if (!((colinit >> c) & 1))
              tc_mma(tmem + (uint32_t)((b * NC + c) * N), tc_desc(smem_addr(sZero), 0, 0),
                     tc_desc(smem_addr(sZero), 0, 0), id_col, 0);
          tc_commit(&dcf[b]);
          tc_commit(&bre[b]);
          if (s % SD == SD - 1 || s == S - 1) tc_commit(&drf);   // the strip group's row use
        }
        if (s % SD == SD - 1 || s == S - 1) ++dcount;
        __syncwarp();
      }
    }
    if (lane == 0) {   // every MMA done before the columns are released
      tc_commit(&done);
      if (!mbar_wait(&done, 0, kMbarWaitLimit) && status) atomicOr(status, kDevTimeout | kDevTimeoutDrain);
    }
    __syncwarp();
  } else if (WC && warp >= 6) {
    // ------------------------------------------------- row-segment loaders
    const int lt_id = threadIdx.x - 192;
    int gcount = 0;
    for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
      const int p = P - 1 - u / nk, k = u % nk;
      const int R0 = p * TI, R1 = min(R0 + TI, n + 1);
      const int S = (R1 - 1) / TM + 1;
      for (int s = 0; s < S && !abort_flag; ++s)
        for (int G0 = max(R0, s * TM); G0 < R1 && !abort_flag; G0 += RG, ++gcount) {
          const int set = gcount % SETS, use2 = gcount / SETS;
          if (use2 >= 1 && !wait(&empty[set], (unsigned)((use2 - 1) & 1))) break;
          const int rows = min(RG, R1 - G0);
          const char *src = (const char *)(Hh + f16x2_slot(G0, s, k, cap, NB) * (SLOT / 2));
          const unsigned dst = smem_addr(sA + (size_t)set * RG * SLOT);
          for (unsigned c = lt_id; c < (unsigned)rows * (SLOT / 16); c += kTcLoaders)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + c * 16), "l"(src + (size_t)c * 16)
                         : "memory");
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_addr(&full[set]))
                       : "memory");
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy outlives the CTA
  } else {
    // ----------------------------------------------------------- epilogue
    const int ew = warp & 3;                  // tensor-memory lane quarter of this warp
    const int L = ew * 32 + lane;             // accumulator row
    const uint32_t lane_addr = tmem + ((uint32_t)(ew * 32) << 16);
    const float inv = 1.f / ((float)kF16HistScale * tc_coef_scale(cmax));
    const size_t nb2 = (size_t)NB * NB;
    int scount = 0, dcount = 0;
    for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
      const int p = P - 1 - u / nk, k = u % nk;
      const int R0 = p * TI, R1 = min(R0 + TI, n + 1);
      const int S = (R1 - 1) / TM + 1;
      for (int s = 0; s < S && !abort_flag; ++s, ++scount) {
        const int M0 = s * TM, b = scount & 1, use = scount >> 1;
        if (!wait(&dcf[b], (unsigned)(use & 1))) break;
        tc_fence_after();
        {
          float v[N];
#pragma unroll
          for (int c = 0; c < N; c += 16) tc_ld16(lane_addr + (uint32_t)(b * NC * N + c), v + c);
#pragma unroll
          for (int acc = 1; acc < NC; ++acc) {
            float w[N];
#pragma unroll
            for (int c = 0; c < N; c += 16) tc_ld16(lane_addr + (uint32_t)((b * NC + acc) * N + c), w + c);
            tc_wait_ld();
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] += w[c];
          }
          tc_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&dce[b]);
          // row L = (x, m, s): value (a, re/im) = part hi + part lo
          const int x = L / 64, ml = (L % 64) / NB, sc = L % NB, m = M0 + ml;
          if (ml < TM && m <= n) {
            const float sg = x ? -inv : inv;   // Y -= C1 dB
            float2 *dst = CP + ((((size_t)p * (n + 1) + m) * nk + k) * 2 + x) * nb2 + sc;
#pragma unroll
            for (int a = 0; a < NB; ++a)
              dst[(size_t)a * NB] =
                  make_float2(sg * (v[2 * a] + v[2 * NB + 2 * a]), sg * (v[2 * a + 1] + v[2 * NB + 2 * a + 1]));
          }
        }
        if (!(s % SD == SD - 1 || s == S - 1)) continue;
        // end of a strip group: drain the row-use accumulators of the groups its
        // first strip reached (every later strip of the group reaches a subset)
        if (abort_flag || !wait(&drf, (unsigned)(dcount & 1))) break;
        ++dcount;
        tc_fence_after();
        const int s0 = s - s % SD, sg = s0 / SD;
        const int groups = (R1 - R0 + RG - 1) / RG, g0 = (max(R0, s0 * TM) - R0) / RG;
        for (int gi = g0; gi < groups; ++gi) {
          float v[N];
#pragma unroll
          for (int c = 0; c < N; c += 16) tc_ld16(lane_addr + (uint32_t)((2 * NC + gi * NR) * N + c), v + c);
          tc_wait_ld();
          for (int acc = 1; acc < NR; ++acc) {
            float w[N];
#pragma unroll
            for (int c = 0; c < N; c += 16) tc_ld16(lane_addr + (uint32_t)((2 * NC + gi * NR + acc) * N + c), w + c);
            tc_wait_ld();
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] += w[c];
          }
          // row L = (i, r, re/im of B); value (a, re/im of C) = part hi + part lo
          float pr[NB], pi[NB];   // P[mine][re][a], P[mine][im][a]
#pragma unroll
          for (int a = 0; a < NB; ++a) {
            pr[a] = v[2 * a] + v[2 * NB + 2 * a];
            pi[a] = v[2 * a + 1] + v[2 * NB + 2 * a + 1];
          }
          const int il = L / (2 * NB), r = (L % (2 * NB)) / 2, riA = L & 1, i = R0 + gi * RG + il;
          // conj(B) C = (P[re][re] + P[im][im]) + i (P[re][im] - P[im][re]); the re lane
          // writes a < NB/2, the im lane a >= NB/2
#pragma unroll
          for (int a = 0; a < NB; ++a) {
            const float or_ = __shfl_xor_sync(0xffffffffu, pr[a], 1), oi = __shfl_xor_sync(0xffffffffu, pi[a], 1);
            const float prr = riA ? or_ : pr[a], pii = riA ? pi[a] : oi;    // P[re][re], P[im][im]
            const float pri = riA ? oi : pi[a], pir = riA ? pr[a] : or_;    // P[re][im], P[im][re]
            if ((a < NB / 2) == (riA == 0) && il < RG && i < R1)
              RP[((((size_t)sg * (n + 1) + i) * nk + k) * NB + a) * NB + r] =
                  make_float2(-inv * (prr + pii), -inv * (pri - pir));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dre);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

// I(j) in FP64 from the partials, plus what the MMAs leave out: the diagonal
// block (end node l = j of column j; for j = 0 an ordinary node above the
// output), the row use at nodes m < j whose weight f = w^(j)_m / dt is not 1
// (X -= (f - 1) C2^<(m) conj(dB(j, m))^T), and the Gregory Y terms of the
// row use (the nodes where the weights of [0, t_j] and [0, t_n] differ).
// A CTA owns column j and KTR consecutive k: it reads the k-outer partials
// and stages the coefficient rows of node j coalesced, sums in FP64, and
// writes I (k fastest) through shared memory.
template <int NB>
__host__ __device__ constexpr int tc_red_kt() { return NB == 4 ? 32 : 8; }

template <int NB, int QUAD>
__global__ void __launch_bounds__(256)
    tc_reduce_kernel(const float2 *__restrict__ CP, const float2 *__restrict__ RP, const float2 *__restrict__ Cf,
                     const __half *__restrict__ H, double2 *__restrict__ I, int n, int nk, int TI, int cap,
                     const int *__restrict__ skip) {
  if (skip && *skip) return;
  constexpr int TM = TcCfg<NB>::TM, NB2 = NB * NB, KTR = tc_red_kt<NB>(), ITEMS = KTR * NB2, SD = tc_sd(NB);
  __shared__ double2 sI[2][NB2][KTR];      // [x][ab][kk]
  __shared__ float2 sC[3][NB2][KTR];       // C1, C2^<, C3 of node j: [q][a c][kk]
  const size_t blk = (size_t)NB2 * nk;
  const int P = (n + TI) / TI;
  const int ktiles = (nk + KTR - 1) / KTR;
  const int j = blockIdx.x / ktiles, k0 = (blockIdx.x % ktiles) * KTR;
  if (j > n) return;
  for (int t = threadIdx.x; t < 3 * ITEMS; t += blockDim.x) {   // coalesced along k
    const int kk = t % KTR, ac = (t / KTR) % NB2, q = t / ITEMS;
    sC[q][ac][kk] = k0 + kk < nk ? Cf[((size_t)j * 3 + q) * blk + (size_t)ac * nk + k0 + kk] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int pmin = (j / TM) * TM / TI;
  for (int t = threadIdx.x; t < ITEMS; t += blockDim.x) {   // ab fastest: the partials are [k][x][a b]
    const int ab = t % NB2, kk = t / NB2, k = k0 + kk;
    if (k >= nk) continue;
    const int a = ab / NB, b = ab % NB;
    FSum sxr, sxi, syr, syi;   // the complex64 partials, summed on the FP32 pipe
    for (int sg = 0; sg * SD * TM <= j; ++sg) {   // the row use's partial of each strip group reaching row j
      const float2 rp = RP[(((size_t)sg * (n + 1) + j) * nk + k) * NB2 + ab];
      sxr.add(rp.x);
      sxi.add(rp.y);
    }
    for (int p = pmin; p < P; ++p) {
      const size_t o = ((((size_t)p * (n + 1) + j) * nk + k) * 2) * NB2 + ab;
      const float2 x = CP[o], y = CP[o + NB2];
      sxr.add(x.x);
      sxi.add(x.y);
      syr.add(y.x);
      syi.add(y.y);
    }
    double xr = sxr.value(), xi = sxi.value(), yr = syr.value(), yi = syi.value();
    // the diagonal block and the end-node terms in FP32 (their operands are
    // complex64 coefficients and 22-bit history values), added to the FP64 sums
    float2 tx = make_float2(0.f, 0.f), ty = make_float2(0.f, 0.f);
    const float f = (float)quad_omega(QUAD, j, j);
    for (int c = 0; c < NB; ++c) {   // diagonal block (j, j)
      const float2 gl = f16x2_getf(H, j, j, k, 0, c, b, NB, cap), dg = f16x2_getf(H, j, j, k, 1, c, b, NB, cap);
      const float2 k1 = sC[0][a * NB + c][kk];
      tx = c_fma(k1, gl, tx);
      if (j == 0) {
        ty = c_fma(make_float2(-k1.x, -k1.y), dg, ty);
      } else {
        const float2 k2 = sC[1][a * NB + c][kk], k3 = sC[2][a * NB + c][kk];
        tx = c_fma(make_float2(f * k2.x, f * k2.y), dg, tx);
        ty = c_fma(make_float2(f * (k3.x - k2.x) + (f - 1.f) * k1.x, f * (k3.y - k2.y) + (f - 1.f) * k1.y), dg, ty);
      }
    }
    // nodes m < j with a weight on [0, t_j] other than dt: trapezoid node 0;
    // Gregory nodes 0, 1, 2, j-2, j-1 (every m < j for j <= 4)
    if (j > 0) {
      const int ns = QUAD == kQuadTrapezoid ? 1 : (j >= 5 ? 5 : j);
      for (int t2 = 0; t2 < ns; ++t2) {
        const int mnode = (QUAD != kQuadTrapezoid && j >= 5 && t2 >= 3) ? j - 5 + t2 : t2;
        const float fm = (float)quad_omega(QUAD, j, mnode);
        for (int c = 0; c < NB; ++c) {
          // the row use pairs output (a, b) with conj(dB(j, m)[b, c])
          const float2 dg = f16x2_getf(H, j, mnode, k, 1, b, c, NB, cap);
          const float2 cd = make_float2(dg.x, -dg.y);
          const size_t o = (size_t)(a * NB + c) * nk + k;
          const float2 k2 = Cf[((size_t)mnode * 3 + 1) * blk + o];
          tx = c_fma(make_float2(-(fm - 1.f) * k2.x, -(fm - 1.f) * k2.y), cd, tx);
          if (QUAD != kQuadTrapezoid) {
            const float2 k1 = Cf[(size_t)mnode * 3 * blk + o], k3 = Cf[((size_t)mnode * 3 + 2) * blk + o];
            ty = c_fma(make_float2(-(fm * (k3.x - k2.x) + (fm - 1.f) * k1.x), -(fm * (k3.y - k2.y) + (fm - 1.f) * k1.y)),
                       cd, ty);
          }
        }
      }
    }
    xr += tx.x;
    xi += tx.y;
    yr += ty.x;
    yi += ty.y;
    sI[0][ab][kk] = make_double2(xr, xi);
    sI[1][ab][kk] = make_double2(xr + yr, xi + yi);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * ITEMS; t += blockDim.x) {   // k fastest: I is [j][x][a b][k]
    const int kk = t % KTR, ab = (t / KTR) % NB2, x = t / ITEMS;
    if (k0 + kk < nk) I[((size_t)j * 2 + x) * blk + (size_t)ab * nk + k0 + kk] = sI[x][ab][kk];
  }
}

template <int NB>
cudaError_t tc_prepare_nb() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  tensor_map_encoder();
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(sweep_tc_kernel<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes<NB>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_tc_kernel<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes<NB>());
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

int tc_tm_of(int nb) { return nb == 4 ? TcCfg<4>::TM : TcCfg<8>::TM; }
int tc_lt(int nb, int n) {   // row-use coefficient tiles per (x, k): strips x TM columns (pairs at N_b = 4)
  const int tm = tc_tm_of(nb);
  return (n / tm + 1) * tm * nb / 8;
}

// strip groups of a row: strips of TM columns, SD at a time
int tc_strip_groups(int nb, int n) { return (n / tc_tm_of(nb) + tc_sd(nb)) / tc_sd(nb); }

// part: [256-byte header (cmax)][Bc][Br][CP][RP per strip group]
struct TcParts {
  unsigned *cmax;
  __half *Bc, *Br;
  float2 *CP, *RP;
};
TcParts tc_parts(const Mesh &m, int n, int TI, void *part) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  char *p = (char *)part;
  TcParts t;
  t.cmax = (unsigned *)p;
  p += 256;
  t.Bc = (__half *)p;
  p += ((size_t)m.nk * (n + 1) * 16 * m.nb * m.nb + 255) / 256 * 256;
  t.Br = (__half *)p;
  p += ((size_t)2 * m.nk * tc_lt(m.nb, n) * 64 * m.nb + 255) / 256 * 256;
  t.CP = (float2 *)p;
  p += (((size_t)((n + TI) / TI) * (n + 1) * 2 * blk) * sizeof(float2) + 255) / 256 * 256;
  t.RP = (float2 *)p;
  return t;
}

template <int NB>
cudaError_t tc_launch(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part, cudaStream_t st,
                      const int *skip, int quad, int *status, int TI, int cap, bool wc) {
  cudaError_t e = tc_prepare_nb<NB>();
  if (e != cudaSuccess) return e;
  const TcParts t = tc_parts(m, n, TI, part);
  const int lt = tc_lt(NB, n);
  {
    const size_t items = (size_t)m.nk * (n + 1) * tc_n<NB>() * (2 * NB / 8) + (size_t)2 * m.nk * lt * tc_n<NB>();
    size_t cb = (items + 255) / 256;
    if (cb > (size_t)device_sms() * 16) cb = (size_t)device_sms() * 16;
    tc_coef_kernel<NB><<<(unsigned)cb, 256, 0, st>>>((const float2 *)Cf, t.cmax, t.Bc, t.Br, n, m.nk, lt, skip);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // tensor-memory columns: NC column-use accumulators per strip buffer (two
  // buffers) and NR per row group of a panel (2 where they fit, else 1)
  const int N = tc_n<NB>(), NC = TcCfg<NB>::NC, groups = TI / TcCfg<NB>::RG;
  int NR = 2;
  if (2 * NC * N + groups * NR * N > 512) NR = 1;
  const int need = 2 * NC * N + groups * NR * N;
  uint32_t tcols = 32;
  while ((int)tcols < need) tcols <<= 1;
  if (tcols > 512) return cudaErrorInvalidValue;
  const long units = (long)((n + TI) / TI) * m.nk;
  const long slots = device_sms();
  const unsigned grid = (unsigned)(units < slots ? units : slots);
  if (wc)
    sweep_tc_kernel<NB, true><<<grid, tc_threads(true), tc_smem_bytes<NB>(), st>>>(
        (const __half *)H, t.Bc, t.Br, t.cmax, t.CP, t.RP, n, m.nk, TI, lt, tcols, NR, cap, skip, status);
  else
    sweep_tc_kernel<NB, false><<<grid, tc_threads(false), tc_smem_bytes<NB>(), st>>>(
        (const __half *)H, t.Bc, t.Br, t.cmax, t.CP, t.RP, n, m.nk, TI, lt, tcols, NR, cap, skip, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned rblocks = (unsigned)((n + 1) * ((m.nk + tc_red_kt<NB>() - 1) / tc_red_kt<NB>()));
  if (quad == kQuadGregory)
    tc_reduce_kernel<NB, kQuadGregory><<<rblocks, 256, 0, st>>>(t.CP, t.RP, (const float2 *)Cf, (const __half *)H, I, n,
                                                               m.nk, TI, cap, skip);
  else
    tc_reduce_kernel<NB, kQuadTrapezoid><<<rblocks, 256, 0, st>>>(t.CP, t.RP, (const float2 *)Cf, (const __half *)H, I,
                                                                 n, m.nk, TI, cap, skip);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Mesh &m, int prec) { return prec == KBE_PREC_F16X2 && (m.nb == 4 || m.nb == 8); }

// the largest TI whose accumulators fit the 512 tensor-memory columns (one
// row-use accumulator per group at the largest heights)
int tc_max_ti(int nb) { return nb == 4 ? 256 : 96; }

size_t tc_part_bytes(const Mesh &m, int n, int TI) {
  if (!(m.nb == 4 || m.nb == 8)) return 0;
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  size_t b = 256;
  b += ((size_t)m.nk * (n + 1) * 16 * m.nb * m.nb + 255) / 256 * 256;
  b += ((size_t)2 * m.nk * tc_lt(m.nb, n) * 64 * m.nb + 255) / 256 * 256;
  b += (((size_t)((n + TI) / TI) * (n + 1) * 2 * blk) * sizeof(float2) + 255) / 256 * 256;
  b += (size_t)tc_strip_groups(m.nb, n) * (n + 1) * blk * sizeof(float2);
  return b;
}

unsigned *tc_cmax_word(void *part) { return (unsigned *)part; }

// tensor-core flops one launch executes at row n (2 x 128 x N x 16 per MMA):
// per panel, strip and row group, 2 x ceil(rows / (8 / N_b)) column-use and
// 16 row-use MMAs, for every k
double tc_tensor_flops(const Mesh &m, int n, int TI) {
  if (!(m.nb == 4 || m.nb == 8) || TI <= 0) return 0.0;
  const int TM = tc_tm_of(m.nb), RG = TM, cstep = 8 / m.nb;
  double mmas = 0.0;
  for (int R0 = 0; R0 <= n; R0 += TI) {
    const int R1 = std::min(R0 + TI, n + 1);
    for (int M0 = 0; M0 <= R1 - 1; M0 += TM)
      for (int G0 = std::max(R0, M0); G0 < R1; G0 += RG) {
        const int rows = std::min(RG, R1 - G0);
        mmas += 2.0 * ((rows + cstep - 1) / cstep) + 16.0;
      }
  }
  return mmas * m.nk * 2.0 * 128.0 * (4.0 * m.nb) * 16.0;
}

cudaError_t tc_prepare(int nb) {
  switch (nb) {
    case 4: return tc_prepare_nb<4>();
    case 8: return tc_prepare_nb<8>();
    default: return cudaSuccess;
  }
}

// TI odd: TI - 1 rows per panel with the row segments copied by loader warps
cudaError_t launch_sweep_tc(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part,
                            cudaStream_t st, const int *skip, int quad, int *status, int TI, int cap) {
  const bool wc = (TI & 1) != 0;
  TI &= ~1;
  if (TI < 16 || TI % 16 != 0 || TI > tc_max_ti(m.nb) || cap < n + 1) return cudaErrorInvalidValue;
  switch (m.nb) {
    case 4: return tc_launch<4>(m, n, H, Cf, I, part, st, skip, quad, status, TI, cap, wc);
    case 8: return tc_launch<8>(m, n, H, Cf, I, part, st, skip, quad, status, TI, cap, wc);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kbe
