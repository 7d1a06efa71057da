// (a2) Collision-integral sweep of the complex64 history that reads every
// stored block from HBM once per evaluation (Eq. 6, left form).
//
// The sweep needs each stored block B = (G^<, dG)(t_i, t_m), i > m, twice:
//   column use (output column m, memory-time node i > m):
//       X(m) += C1(i) B^<,        Y(m) -= C1(i) dB,
//   row use (output column i, node m < i, through G(t_m, t_i) = -B^+):
//       X(i) += C1(m) G^<(m,i) + f C2^<(m) dG(m,i),
// with X = I^<, Y = I^> - I^<, C1 = w^(n)_l (S^> - S^<), C2^< = dt S^<,
// C3 = dt S^> - C1, and f = w^(i)_m / dt the weight of node m on [0, t_i]
// (1 in the interior). The diagonal block (j, j) is the end node l = j of
// column j: X(j) += C1 B^< + f C2^< dB, Y(j) += (f (C3 - C2^<) + (f - 1) C1) dB
// (for j = 0 it is an ordinary node above the output, X += C1 B^<,
// Y -= C1 dB). The per-column sweep (kbe_sweep.cu) serves the two uses from
// different CTAs, so every block crosses HBM twice.
//
// Here a CTA owns a strip of TM output columns [M0, M0 + TM), a chunk of at
// most TI rows [R0, R1) below the strip's top, and KT consecutive k. It walks
// the chunk one row i at a time: the row segment, blocks (i, M0 .. M0+TM-1),
// is contiguous in the triangle, so one 4-D TMA box brings it (with the C1(i)
// coefficient row) into a 3-stage shared-memory ring, and every block of it
// feeds both uses from shared memory:
//   - warp g handles the TMW columns M0 + g TMW + q; a lane is one (k, a)
//     pair, so a lane owns the output row a of X(m), Y(m) for its columns and
//     keeps them in registers over the whole chunk (column use);
//   - the same lane adds the row use of its columns to X(i)_{a, .}; the warps'
//     shares are summed through shared memory once per row.
// Every lane of a warp reads the same block (lanes differ in k and a), so a
// load is KT consecutive complex64 values, conflict-free.
//
// Partial sums are complex64: the column partials of one chunk (X, Y of each
// column, summed over <= TI rows) and the row partials of one strip (X of each
// row, summed over the strip's TM columns). tile_reduce_kernel adds them as
// hi + lo FP32 pairs (FSum) in a fixed order (the result is deterministic) and adds the row use's
// Y terms at the few nodes where the weights of [0, t_j] and [0, t_n] differ
// (none for the trapezoid rule; the Gregory end nodes). The extra traffic is
// ~(1/TI + 1/(2 TM)) of the triangle's bytes, written once and read once.
//
// Every wait on an mbarrier is bounded (kbe_tma.cuh): a copy that never lands
// marks kDevTimeout (and kDevTimeoutDrain if the copies in flight cannot be
// drained) in the status word and the CTA stops.
#include <mutex>

#include "kbe_internal.cuh"
#include "kbe_tma.cuh"

namespace kbe {

namespace {

// per N_b: KG warps share one column group, each on 32 / N_b of the CTA's
// KT = KG 32 / N_b consecutive k (a lane is one (k, a)); TMW columns per
// column group, W warps (TM = TMW W / KG columns per strip), S stages of the
// ring, RB row-reduction buffers (2: one barrier per row), MINB CTAs per SM.
// Four columns per warp amortise the per-row work (the C1(i) row, the
// reduction of the row use over the column groups, the barrier) over four
// blocks. (Timed at row 511 of c2, against one CTA of 8 warps of four
// columns: 16 warps of two columns at <= 128 registers 20 % slower; 128-byte
// TMA rows (two warps per column group) no faster; two CTAs of 4 warps per
// SM 3 % slower.)
template <int NB>
struct TileCfg;
template <>
struct TileCfg<2> {
  static constexpr int KG = 1, KT = 16, TMW = 4, W = 8, S = 3, RB = 2, MINB = 1;
};
template <>
struct TileCfg<4> {
  static constexpr int KG = 1, KT = 8, TMW = 4, W = 8, S = 3, RB = 2, MINB = 1;
};
template <>
struct TileCfg<8> {
  static constexpr int KG = 1, KT = 4, TMW = 2, W = 8, S = 3, RB = 1, MINB = 1;
};

constexpr size_t kTileCounterBytes = 256;   // the work-unit counter ahead of the partial sums

template <int NB>
__host__ __device__ constexpr int tile_tm() {
  return TileCfg<NB>::TMW * TileCfg<NB>::W / TileCfg<NB>::KG;
}
template <int NB>
__host__ __device__ constexpr int tile_threads() {
  return 32 * TileCfg<NB>::W;
}
// complex64 values of one stage: the TM blocks [q][x][a b][kk], then C1(i) [a c][kk]
template <int NB>
__host__ __device__ constexpr int tile_block_elems() {
  return tile_tm<NB>() * 2 * NB * NB * TileCfg<NB>::KT;
}
template <int NB>
__host__ __device__ constexpr int tile_stage_elems() {
  return tile_block_elems<NB>() + NB * NB * TileCfg<NB>::KT;
}
template <int NB>
__host__ __device__ constexpr int tile_red_elems() {
  return TileCfg<NB>::W / TileCfg<NB>::KG * NB * NB * TileCfg<NB>::KT;   // [column group][cc][a][kk]
}
template <int NB>
constexpr size_t tile_smem_bytes() {
  return sizeof(float2) * ((size_t)TileCfg<NB>::S * tile_stage_elems<NB>() +
                           (size_t)TileCfg<NB>::RB * tile_red_elems<NB>());
}
static_assert(tile_smem_bytes<2>() + 256 <= 227 * 1024 && tile_smem_bytes<4>() + 256 <= 227 * 1024 &&
                  tile_smem_bytes<8>() + 256 <= 227 * 1024,
              "tile sweep shared memory");
static_assert((tile_block_elems<4>() * sizeof(float2)) % 128 == 0 && (tile_stage_elems<4>() * sizeof(float2)) % 128 == 0 &&
                  (tile_stage_elems<2>() * sizeof(float2)) % 128 == 0 && (tile_stage_elems<8>() * sizeof(float2)) % 128 == 0,
              "stage alignment");

// acc + x * y, acc - x * y, acc + x * conj(y) on complex64 (FP32 FMAs)
__device__ __forceinline__ float2 f_fma(float2 x, float2 y, float2 acc) {
  return make_float2(fmaf(x.x, y.x, fmaf(-x.y, y.y, acc.x)), fmaf(x.x, y.y, fmaf(x.y, y.x, acc.y)));
}
__device__ __forceinline__ float2 f_fnma(float2 x, float2 y, float2 acc) {
  return make_float2(fmaf(-x.x, y.x, fmaf(x.y, y.y, acc.x)), fmaf(-x.x, y.y, fmaf(-x.y, y.x, acc.y)));
}
__device__ __forceinline__ float2 f_fmac(float2 x, float2 y, float2 acc) {
  return make_float2(fmaf(x.x, y.x, fmaf(x.y, y.y, acc.x)), fmaf(x.y, y.x, fmaf(-x.x, y.y, acc.y)));
}

// (strip, chunk) of work item p: strip s covers columns [s TM, (s+1) TM) and
// rows [s TM, n], split into chunks of TI rows; false past the last item
__device__ __forceinline__ bool tile_item(int p, int n, int TM, int TI, int *s_out, int *c_out) {
  const int strips = (n + TM) / TM;
  for (int s = 0; s < strips; ++s) {
    const int cs = (n + 1 - s * TM + TI - 1) / TI;
    if (p < cs) {
      *s_out = s;
      *c_out = p;
      return true;
    }
    p -= cs;
  }
  return false;
}

// Work unit u: k-tile u % ktiles of work item u / ktiles (the k-tiles of one
// item adjacent, so that their DRAM pages are read together); items come strip
// by strip, so the last units are the short strips near the diagonal's end.
// persistent != 0: one CTA per SM claims units from a counter; the
// shared-memory ring and its mbarrier phases run on over the units (g = rows
// consumed so far). Otherwise one CTA per unit.
// CP: column partials [chunk][j][x][a][b][k], RP: row partials [strip][j][a][b][k]
// (complex64). counter: zeroed before the launch.
template <int NB, int QUAD>
__global__ void __launch_bounds__(tile_threads<NB>(), TileCfg<NB>::MINB)
    sweep_tile_kernel(const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmH,
                      const float2 *__restrict__ Cf, float2 *__restrict__ CP, float2 *__restrict__ RP, int n,
                      int nk, int TI, int units, int *counter, int persistent, const int *__restrict__ skip,
                      int *status) {
  if (skip && *skip) return;
  constexpr int KT = TileCfg<NB>::KT, TMW = TileCfg<NB>::TMW, TM = tile_tm<NB>(), NB2 = NB * NB;
  constexpr int SE = tile_stage_elems<NB>(), BE = tile_block_elems<NB>(), RB = TileCfg<NB>::RB;
  constexpr int kStg = TileCfg<NB>::S, kW = TileCfg<NB>::W;
  constexpr unsigned kBytesH = (unsigned)BE * sizeof(float2), kBytesC = (unsigned)NB2 * KT * sizeof(float2);
  extern __shared__ __align__(128) float4 tile_smem4[];
  __shared__ __align__(8) uint64_t bar[kStg];
  __shared__ int failed, s_unit;
  float2 *smem = reinterpret_cast<float2 *>(tile_smem4);
  float2 *redbase = smem + (size_t)kStg * SE;
  constexpr int KG = TileCfg<NB>::KG, KW = KT / KG, NCG = kW / KG;   // k per warp, column groups
  const int ktiles = (nk + KT - 1) / KT;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warp = wid / KG;                              // column group
  const int kk = (wid % KG) * KW + lane % KW, a = lane / KW;   // k within the tile, row a
  const size_t blk = (size_t)NB2 * nk;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStg; ++st) mbar_init(&bar[st], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int g0 = 0;   // rows this CTA consumed in earlier units
  for (int pass = 0;; ++pass) {
    if (persistent) {
      if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
      __syncthreads();
    } else if (threadIdx.x == 0) {
      s_unit = pass == 0 ? (int)blockIdx.x : units;   // one unit per CTA
    }
    if (!persistent) __syncthreads();
    const int unit = s_unit;
    if (unit >= units) break;
    int s = 0, c = 0;
    if (!tile_item(unit / ktiles, n, TM, TI, &s, &c)) break;   // cannot happen: units = ktiles x items
    const int M0 = s * TM, R0 = M0 + c * TI, R1 = min(M0 + (c + 1) * TI, n + 1);
    const int rows = R1 - R0;
    const int k0 = (unit % ktiles) * KT;
    const int k = k0 + kk;
    const bool kvalid = k < nk;

    // C1(m), C2^<(m) of this lane's columns (row a, this k), kept for the unit
    float2 C1m[TMW][NB], C2m[TMW][NB];
#pragma unroll
    for (int q = 0; q < TMW; ++q) {
      const int m = M0 + warp * TMW + q;
#pragma unroll
      for (int cc = 0; cc < NB; ++cc) {
        const bool ok = m <= n && kvalid;
        const size_t o = (size_t)(a * NB + cc) * nk + k;
        C1m[q][cc] = ok ? Cf[(size_t)m * 3 * blk + o] : make_float2(0.f, 0.f);
        C2m[q][cc] = ok ? Cf[((size_t)m * 3 + 1) * blk + o] : make_float2(0.f, 0.f);
      }
    }
    float2 X[TMW][NB], Y[TMW][NB];   // column use: X(m)_{a,b}, Y(m)_{a,b}
#pragma unroll
    for (int q = 0; q < TMW; ++q)
#pragma unroll
      for (int b = 0; b < NB; ++b) X[q][b] = Y[q][b] = make_float2(0.f, 0.f);

    auto issue = [&](int r) {   // row R0 + r (the CTA's row g0 + r) into stage (g0 + r) % kStg
      const int i = R0 + r, st = (g0 + r) % kStg;
      float2 *dst = smem + (size_t)st * SE;
      mbar_expect_tx(&bar[st], kBytesH + kBytesC);
      tma_load_4d(dst, &tmH, 2 * k0, 0, 0, (int)tri(i, M0), &bar[st]);
      tma_load_3d(dst + BE, &tmC, 2 * k0, 0, 3 * i, &bar[st]);
    };
    if (threadIdx.x == 0)
      for (int r = 0; r < kStg - 1 && r < rows; ++r) issue(r);
    int issued = min(kStg - 1, rows);

    for (int r = 0; r < rows; ++r) {
      const int g = g0 + r;   // the ring's stage and phase
      if (threadIdx.x == 0 && issued < rows && issued == r + kStg - 1) issue(issued);
      issued = min(r + kStg, rows);
      const int st = g % kStg;
      if (!mbar_wait(&bar[st], (unsigned)((g / kStg) & 1), kMbarWaitLimit)) failed = 1;
      __syncthreads();
      if (failed) {   // a copy did not arrive: flag it, let the in-flight ones land, stop
        if (threadIdx.x == 0) {
          int code = kDevTimeout;
          for (int q = r; q < issued; ++q) {
            const int gq = g0 + q;
            if (!mbar_wait(&bar[gq % kStg], (unsigned)((gq / kStg) & 1), kMbarWaitLimit))
              code |= kDevTimeoutDrain;
          }
          if (status) atomicOr(status, code);
        }
        __syncthreads();
        return;
      }
      const int i = R0 + r;
      const float2 *stg = smem + (size_t)st * SE;
      float2 C1i[NB];
#pragma unroll
      for (int cc = 0; cc < NB; ++cc) C1i[cc] = stg[BE + (a * NB + cc) * KT + kk];
      float2 T[NB];   // row use, summed over this warp's columns: X(i)_{a,cc} = -T[cc]
#pragma unroll
      for (int cc = 0; cc < NB; ++cc) T[cc] = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < TMW; ++q) {
        const int m = M0 + warp * TMW + q;
        if (m > i) continue;   // past the diagonal (warp-uniform)
        const float2 *B = stg + (size_t)(warp * TMW + q) * 2 * NB2 * KT + kk;   // [x][r s][kk]
        if (m < i) {
          const float f = (float)quad_omega(QUAD, i, m);
          float2 K2[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) K2[b] = f == 1.0f ? C2m[q][b] : make_float2(f * C2m[q][b].x, f * C2m[q][b].y);
#pragma unroll
          for (int cc = 0; cc < NB; ++cc)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 x = B[(cc * NB + b) * KT], d = B[(NB2 + cc * NB + b) * KT];
              X[q][b] = f_fma(C1i[cc], x, X[q][b]);
              Y[q][b] = f_fnma(C1i[cc], d, Y[q][b]);
              T[cc] = f_fmac(C1m[q][b], x, T[cc]);
              T[cc] = f_fmac(K2[b], d, T[cc]);
            }
        } else if (i == 0) {   // the only node of column 0 on the diagonal: above the output
#pragma unroll
          for (int cc = 0; cc < NB; ++cc)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 x = B[(cc * NB + b) * KT], d = B[(NB2 + cc * NB + b) * KT];
              X[q][b] = f_fma(C1i[cc], x, X[q][b]);
              Y[q][b] = f_fnma(C1i[cc], d, Y[q][b]);
            }
        } else {   // end node l = j of column j = i: weight f, Y coefficient f (C3 - C2^<) + (f - 1) C1
          const float f = (float)quad_omega(QUAD, i, i);
#pragma unroll
          for (int cc = 0; cc < NB; ++cc) {
            const float2 k3 = kvalid ? Cf[((size_t)i * 3 + 2) * blk + (size_t)(a * NB + cc) * nk + k]
                                     : make_float2(0.f, 0.f);
            const float2 k2 = C2m[q][cc], k1 = C1i[cc];
            const float2 K2 = make_float2(f * k2.x, f * k2.y);
            const float2 KY = make_float2(f * (k3.x - k2.x) + (f - 1.0f) * k1.x, f * (k3.y - k2.y) + (f - 1.0f) * k1.y);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 x = B[(cc * NB + b) * KT], d = B[(NB2 + cc * NB + b) * KT];
              X[q][b] = f_fma(k1, x, X[q][b]);
              X[q][b] = f_fma(K2, d, X[q][b]);
              Y[q][b] = f_fma(KY, d, Y[q][b]);
            }
          }
        }
      }
      // the column groups' row-use shares: red[cg][cc][a][kk], summed by the first NB NB KT threads
      float2 *red = redbase + (size_t)(g % RB) * tile_red_elems<NB>();
#pragma unroll
      for (int cc = 0; cc < NB; ++cc) red[((warp * NB + cc) * NB + a) * KT + kk] = T[cc];
      __syncthreads();   // the stage is consumed and the shares are written
      if (threadIdx.x < NB * NB * KT) {
        const int t = threadIdx.x;   // (a', cc', kk') with kk' fastest: coalesced writes
        const int kk2 = t % KT, ac = t / KT, cc2 = ac % NB, a2 = ac / NB;
        float2 sum = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NCG; ++w) {
          const float2 v = red[((w * NB + cc2) * NB + a2) * KT + kk2];
          sum.x += v.x;
          sum.y += v.y;
        }
        const int k2 = k0 + kk2;
        if (k2 < nk)
          RP[(((size_t)s * (n + 1) + i) * NB2 + a2 * NB + cc2) * nk + k2] = make_float2(-sum.x, -sum.y);
      }
      if (RB == 1) __syncthreads();   // single buffer: its sums are read before the next row writes it
    }
    g0 += rows;
    // column partials of this unit's chunk
#pragma unroll
    for (int q = 0; q < TMW; ++q) {
      const int m = M0 + warp * TMW + q;
      if (m > n || !kvalid) continue;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const size_t o = (size_t)(a * NB + b) * nk + k;
        CP[(((size_t)c * (n + 1) + m) * 2) * blk + o] = X[q][b];
        CP[(((size_t)c * (n + 1) + m) * 2 + 1) * blk + o] = Y[q][b];
      }
    }
  }
}

// I(j) from the partials (hi + lo FP32 pairs, FP64 result): X = sum of the column partials of column j
// (one per chunk of its strip) and of its row partials (one per strip left of
// it); Y = the column partials' Y plus the row use's Y at nodes m < j whose
// weight on [0, t_j] differs from the one on [0, t_n]: (f (C3 - C2^<) +
// (f - 1) C1)(m) dG(m, j), dG(m, j) = -dB(j, m)^+ (Gregory end nodes; the
// trapezoid has none: its only such node, l = 0, has f = w^(n)_0 / dt).
template <int NB, int QUAD>
__global__ void tile_reduce_kernel(const float2 *__restrict__ CP, const float2 *__restrict__ RP,
                                   const float2 *__restrict__ Cf, const float2 *__restrict__ H,
                                   double2 *__restrict__ I, int n, int nk, int TI, int TM,
                                   const int *__restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NB2 = NB * NB;
  const size_t blk = (size_t)NB2 * nk, count = (size_t)(n + 1) * blk;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / blk);
    const size_t r = idx - (size_t)j * blk;   // (a b) nk + k
    const int ab = (int)(r / nk), k = (int)(r - (size_t)ab * nk);
    const int a = ab / NB, b = ab - a * NB;
    const int M0 = (j / TM) * TM;
    const int chunks = (n + 1 - M0 + TI - 1) / TI, strips = j / TM + 1;
    FSum sxr, sxi, syr, syi;   // the complex64 partials, summed on the FP32 pipe
    for (int c = 0; c < chunks; ++c) {
      const float2 x = CP[(((size_t)c * (n + 1) + j) * 2) * blk + r];
      const float2 y = CP[(((size_t)c * (n + 1) + j) * 2 + 1) * blk + r];
      sxr.add(x.x);
      sxi.add(x.y);
      syr.add(y.x);
      syi.add(y.y);
    }
    for (int s = 0; s < strips; ++s) {
      const float2 x = RP[((size_t)s * (n + 1) + j) * blk + r];
      sxr.add(x.x);
      sxi.add(x.y);
    }
    double xr = sxr.value(), xi = sxi.value(), yr = syr.value(), yi = syi.value();
    if (QUAD != kQuadTrapezoid && j > 0 && n >= 1) {
      const int ns = j >= 5 ? 5 : j;   // nodes 0, 1, 2, j-2, j-1 (every m < j for j <= 4)
      for (int t = 0; t < ns; ++t) {
        const int m = (j >= 5 && t >= 3) ? j - 5 + t : t;
        const float f = (float)quad_omega(QUAD, j, m);
        const float2 *dB = H + (tri(j, m) * 2 + 1) * blk + k;   // dG(j, m), [r s] rows of n_k
        float2 acc = make_float2(0.f, 0.f);
        for (int cc = 0; cc < NB; ++cc) {
          const size_t o = (size_t)(a * NB + cc) * nk + k;
          const float2 k1 = Cf[(size_t)m * 3 * blk + o], k2 = Cf[((size_t)m * 3 + 1) * blk + o],
                       k3 = Cf[((size_t)m * 3 + 2) * blk + o];
          const float2 KY = make_float2(f * (k3.x - k2.x) + (f - 1.0f) * k1.x, f * (k3.y - k2.y) + (f - 1.0f) * k1.y);
          // dG(m, j)_{cc, b} = -conj(dB(j, m)_{b, cc})
          acc = f_fmac(KY, dB[(size_t)(b * NB + cc) * nk], acc);
        }
        yr -= acc.x;
        yi -= acc.y;
      }
    }
    I[((size_t)j * 2) * blk + r] = make_double2(xr, xi);
    I[((size_t)j * 2 + 1) * blk + r] = make_double2(xr + yr, xi + yi);
  }
}

template <int NB>
bool tile_maps(const void *Cf, const void *H, int n, int nk, CUtensorMap *tmC, CUtensorMap *tmH) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  constexpr int KT = TileCfg<NB>::KT, NB2 = NB * NB, TM = tile_tm<NB>();
  const cuuint64_t row = (cuuint64_t)2 * nk * sizeof(float);   // one (a, c) row of k, bytes
  {
    const cuuint64_t dim[3] = {(cuuint64_t)2 * nk, (cuuint64_t)NB2, (cuuint64_t)3 * (n + 1)};
    const cuuint64_t stride[2] = {row, row * NB2};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * KT), (cuuint32_t)NB2, 1};
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
    const cuuint32_t box[4] = {(cuuint32_t)(2 * KT), (cuuint32_t)NB2, 2, (cuuint32_t)TM};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(tmH, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(H), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// shared-memory limit of the tile kernels, raised once per device under a lock
template <int NB>
cudaError_t tile_prepare_nb() {
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
  const int bytes = (int)tile_smem_bytes<NB>();
  e = cudaFuncSetAttribute(sweep_tile_kernel<NB, kQuadTrapezoid>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_tile_kernel<NB, kQuadGregory>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

int tile_tm_of(int nb) { return nb == 2 ? tile_tm<2>() : nb == 4 ? tile_tm<4>() : tile_tm<8>(); }

long tile_items(int n, int TM, int TI) {
  long p = 0;
  for (int s = 0; s * TM <= n; ++s) p += (n + 1 - s * TM + TI - 1) / TI;
  return p;
}

template <int NB>
cudaError_t tile_launch(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part,
                        cudaStream_t st, const int *skip, int quad, int *status, int TI, bool persistent) {
  cudaError_t e = tile_prepare_nb<NB>();
  if (e != cudaSuccess) return e;
  CUtensorMap tmC, tmH;
  if (!tile_maps<NB>(Cf, H, n, m.nk, &tmC, &tmH)) return cudaErrorNotSupported;
  constexpr int TM = tile_tm<NB>(), KT = TileCfg<NB>::KT;
  const size_t blk = (size_t)NB * NB * m.nk;
  int *counter = (int *)part;   // the work-unit counter, then the partial sums
  float2 *CP = (float2 *)((char *)part + kTileCounterBytes);
  float2 *RP = CP + (size_t)((n + TI) / TI) * (n + 1) * 2 * blk;
  const long units = (long)((m.nk + KT - 1) / KT) * tile_items(n, TM, TI);
  const long slots = (long)device_sms() * TileCfg<NB>::MINB;   // resident CTAs
  const unsigned grid = persistent ? (unsigned)(units < slots ? units : slots) : (unsigned)units;
  const size_t smem = tile_smem_bytes<NB>();
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (quad == kQuadGregory)
    sweep_tile_kernel<NB, kQuadGregory><<<grid, tile_threads<NB>(), smem, st>>>(tmC, tmH, (const float2 *)Cf, CP, RP, n,
                                                                          m.nk, TI, (int)units, counter,
                                                                          persistent ? 1 : 0, skip, status);
  else
    sweep_tile_kernel<NB, kQuadTrapezoid><<<grid, tile_threads<NB>(), smem, st>>>(tmC, tmH, (const float2 *)Cf, CP, RP,
                                                                            n, m.nk, TI, (int)units, counter,
                                                                            persistent ? 1 : 0, skip, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t count = (size_t)(n + 1) * blk;
  size_t blocks = (count + 255) / 256;
  const size_t cap = (size_t)device_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (quad == kQuadGregory)
    tile_reduce_kernel<NB, kQuadGregory><<<(unsigned)blocks, 256, 0, st>>>(CP, RP, (const float2 *)Cf,
                                                                          (const float2 *)H, I, n, m.nk, TI, TM, skip);
  else
    tile_reduce_kernel<NB, kQuadTrapezoid><<<(unsigned)blocks, 256, 0, st>>>(CP, RP, (const float2 *)Cf,
                                                                            (const float2 *)H, I, n, m.nk, TI, TM, skip);
  return cudaGetLastError();
}

}  // namespace

bool tile_supported(const Mesh &m, int prec) {
  return prec == KBE_PREC_C64 && (m.nb == 2 || m.nb == 4 || m.nb == 8) && m.nk % 2 == 0;
}

size_t tile_part_bytes(const Mesh &m, int n, int TI) {
  if (!(m.nb == 2 || m.nb == 4 || m.nb == 8)) return 0;
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const int TM = tile_tm_of(m.nb);
  const size_t cp = (size_t)((n + TI) / TI) * (n + 1) * 2 * blk;
  const size_t rp = (size_t)((n + TM) / TM) * (n + 1) * blk;
  return kTileCounterBytes + (cp + rp) * sizeof(float2);
}

cudaError_t tile_prepare(int nb) {
  switch (nb) {
    case 2: return tile_prepare_nb<2>();
    case 4: return tile_prepare_nb<4>();
    case 8: return tile_prepare_nb<8>();
    default: return cudaSuccess;
  }
}

cudaError_t launch_sweep_tile(const Mesh &m, int n, const void *H, const void *Cf, double2 *I, void *part,
                              cudaStream_t st, const int *skip, int quad, int *status, int TI) {
  const bool persistent = (TI & 1) == 0;   // an odd TI asks for one CTA per work unit (TI - 1 rows)
  TI &= ~1;
  switch (m.nb) {
    case 2: return tile_launch<2>(m, n, H, Cf, I, part, st, skip, quad, status, TI, persistent);
    case 4: return tile_launch<4>(m, n, H, Cf, I, part, st, skip, quad, status, TI, persistent);
    case 8: return tile_launch<8>(m, n, H, Cf, I, part, st, skip, quad, status, TI, persistent);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kbe
