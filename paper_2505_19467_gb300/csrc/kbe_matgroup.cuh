// Per-k matrix groups shared by the propagator, update and adjoint kernels.
// Internal to libkbe (CUDA, sm_103a); included by the .cu files that need it.
#pragma once

#include "kbe_internal.cuh"

namespace kbe {

namespace {

// ------------------------------------------------ per-k matrix functions ----
// A CTA holds kpc k-points (chosen at launch so that the CTAs cover the SMs:
// the series are FP64-pipe bound); thread t works on element (a, b) of
// k-point t / N_b^2. Matrices live in dynamic shared memory, [kk][a][b].
extern __shared__ double2 kbe_dsm[];

template <int NB>
struct MatGroup {
  static constexpr int E = NB * NB;
  int kk, a, b, e;
  __device__ MatGroup() {
    kk = threadIdx.x / E;
    e = threadIdx.x - kk * E;
    a = e / NB;
    b = e - a * NB;
  }
  // (A B)_ab of this thread's k-point. The sum over c runs as two independent
  // chains (even and odd c) added at the end: the series kernels are chains of
  // these products on one warp per SM sub-partition, so the dependent FP64
  // latency, not the pipe, sets their time.
  __device__ __forceinline__ double2 mm(const double2 *A, const double2 *B) const {
    const double2 *Ar = A + kk * E + a * NB;
    const double2 *Bc = B + kk * E + b;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c + 1 < NB; c += 2) {
      s0 = c_fma(Ar[c], Bc[c * NB], s0);
      s1 = c_fma(Ar[c + 1], Bc[(c + 1) * NB], s1);
    }
    if (NB % 2) s0 = c_fma(Ar[NB - 1], Bc[(NB - 1) * NB], s0);
    return c_add(s0, s1);
  }
  // (A B^+)_ab, two chains as mm
  __device__ __forceinline__ double2 mm_adj(const double2 *A, const double2 *B) const {
    const double2 *Ar = A + kk * E + a * NB;
    const double2 *Br = B + kk * E + b * NB;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c + 1 < NB; c += 2) {
      s0 = c_add(s0, c_mulc(Ar[c], Br[c]));
      s1 = c_add(s1, c_mulc(Ar[c + 1], Br[c + 1]));
    }
    if (NB % 2) s0 = c_add(s0, c_mulc(Ar[NB - 1], Br[NB - 1]));
    return c_add(s0, s1);
  }
};

// 1/m for the series coefficients tau / m (m = 0 .. 23; entry 0 unused): a
// multiplication by a tabulated reciprocal in place of an FP64 division,
// which costs about ten FP64-pipe instructions, per term and element
static __constant__ double kSeriesInv[24] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,
    1.0 / 8,    1.0 / 9,    1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15,
    1.0 / 16,   1.0 / 17,   1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23};

// The series lengths: with nu = tau ||h|| <= 1/4 (rowsum norm, submultiplicative)
// the m-th term of U_tau (and of V_tau / tau) is bounded by nu^m / m! of the
// leading term, the m-th term of X_tau by (2 nu)^m / (m + 1)! of tau ||S||. Each
// series stops before its first term whose bound is below 2^-60 (1/128 of the
// FP64 unit roundoff; the terms after it decay faster still): at the worst
// nu = 1/4 that is 13 and 15 terms, at nu ~ 0.12 (dt = 0.02, ||h|| ~ 6) 11 and
// 12. At most 14 and 18 terms.
struct SeriesPlan {
  int s;      // doublings: tau = dt / 2^s
  int mexp;   // terms m = 1 .. mexp of U_tau (and V_tau)
  int mx;     // terms m = 1 .. mx of X_tau
};

__device__ __forceinline__ SeriesPlan series_lengths(double nu) {
  const double exp_tail = 0x1p-60, x_tail = 0x1p-60;
  SeriesPlan p{0, 14, 18};
  double t = 1.0;                    // nu^m / m!
  for (int m = 1; m <= 14; ++m) {
    t *= nu * kSeriesInv[m];
    if (t <= exp_tail) {             // term m is already below the bound: m - 1 terms suffice
      p.mexp = m > 1 ? m - 1 : 1;
      break;
    }
  }
  double q = 1.0;                    // (2 nu)^m / m!
  for (int m = 1; m <= 18; ++m) {
    q *= 2.0 * nu * kSeriesInv[m];
    if (q * kSeriesInv[m + 1] <= x_tail) {   // (2 nu)^m / (m + 1)!
      p.mx = m > 1 ? m - 1 : 1;
      break;
    }
  }
  return p;
}

// number of doublings s with (dt / 2^s) * max_k ||h_k||_rowsum <= 1/4, for
// all k-points of the CTA (uniform across the CTA), and the series lengths
// for tau = dt / 2^s; h in shared memory
template <int NB>
__device__ SeriesPlan series_plan(const MatGroup<NB> &g, const double2 *h, int kpc, int nvalid, double dt,
                                  double *red) {
  if (g.b == 0) {
    double r = 0.0;
    for (int c = 0; c < NB; ++c) {
      const double2 z = h[g.kk * g.E + g.a * NB + c];
      r += hypot(z.x, z.y);
    }
    red[g.kk * NB + g.a] = (g.kk < nvalid) ? r : 0.0;
  }
  __syncthreads();
  __shared__ SeriesPlan plan_sh;
  if (threadIdx.x == 0) {
    double nu = 0.0;
    for (int i = 0; i < kpc * NB; ++i) nu = fmax(nu, red[i]);
    nu *= dt;
    int sc = 0;
    while (nu > 0.25 && sc < 40) {   // bounded: nu <= 2^40 / 4 covers any finite h
      nu *= 0.5;
      ++sc;
    }
    SeriesPlan p = series_lengths(nu);
    p.s = sc;
    plan_sh = p;
  }
  __syncthreads();
  return plan_sh;
}

// U_dt and V_dt of h (shared memory), element (a, b) returned in u, v;
// P, Q, W are shared scratch of KPC * N_b^2 each; mt terms of the series
// (series_plan).
template <int NB>
__device__ void exp_and_phi(const MatGroup<NB> &g, const double2 *h, double tau, int s, double2 *P,
                            double2 *Q, double2 *W, double2 &u, double2 &v, int mt = 14) {
  const int o = g.kk * g.E + g.e;
  const double2 one = make_double2(g.a == g.b ? 1.0 : 0.0, 0.0);
  P[o] = one;
  u = one;
  v = make_double2(0.0, -tau * one.x);   // -i tau P_0 / 1
  __syncthreads();
  for (int m = 1; m <= mt; ++m) {
    const double cm = tau * kSeriesInv[m], cv = tau * kSeriesInv[m + 1];
    double2 t = g.mm(P, h);
    t = make_double2(cm * t.y, -cm * t.x);   // (-i tau / m) (P h)
    __syncthreads();
    P[o] = t;
    u = c_add(u, t);
    v = c_add(v, make_double2(cv * t.y, -cv * t.x));
    __syncthreads();
  }
  for (int r = 0; r < s; ++r) {   // V <- (U + 1) V, U <- U U
    P[o] = u;
    Q[o] = v;
    W[o] = c_add(u, one);
    __syncthreads();
    const double2 un = g.mm(P, P), vn = g.mm(W, Q);
    __syncthreads();
    u = un;
    v = vn;
  }
}

// (A^+ B)_ab of this thread's k-point
template <int NB>
__device__ __forceinline__ double2 mm_hadj(const MatGroup<NB> &g, const double2 *A, const double2 *B) {
  const double2 *Ac = A + g.kk * g.E + g.a;
  const double2 *Bc = B + g.kk * g.E + g.b;
  double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
#pragma unroll
  for (int c = 0; c + 1 < NB; c += 2) {
    s0 = c_add(s0, c_mulc(Bc[c * NB], Ac[c * NB]));
    s1 = c_add(s1, c_mulc(Bc[(c + 1) * NB], Ac[(c + 1) * NB]));
  }
  if (NB % 2) s0 = c_add(s0, c_mulc(Bc[(NB - 1) * NB], Ac[(NB - 1) * NB]));
  return c_add(s0, s1);
}

#define KBE_NB_SWITCH(nb, CALL)          \
  switch (nb) {                          \
    case 1: { constexpr int NB = 1; CALL; } break;   \
    case 2: { constexpr int NB = 2; CALL; } break;   \
    case 3: { constexpr int NB = 3; CALL; } break;   \
    case 4: { constexpr int NB = 4; CALL; } break;   \
    case 6: { constexpr int NB = 6; CALL; } break;   \
    case 8: { constexpr int NB = 8; CALL; } break;   \
    case 12: { constexpr int NB = 12; CALL; } break; \
    case 16: { constexpr int NB = 16; CALL; } break; \
    default: return cudaErrorInvalidValue;           \
  }

// k-points per CTA: enough CTAs to cover the SMs, at most 256 threads
template <int NB>
int matgroup_kpc(int nk) {
  const int E = NB * NB, maxk = 256 / E > 0 ? 256 / E : 1;
  const int sms = device_sms();
  int kpc = (nk + sms - 1) / sms;
  return kpc < 1 ? 1 : (kpc > maxk ? maxk : kpc);
}
template <int NB>
unsigned matgroup_blocks(int nk) {
  const int kpc = matgroup_kpc<NB>(nk);
  return (unsigned)((nk + kpc - 1) / kpc);
}
template <int NB>
unsigned matgroup_threads(int nk) {
  return (unsigned)(matgroup_kpc<NB>(nk) * NB * NB);
}
template <int NB>
size_t matgroup_smem(int nk, int nmat) {
  const int kpc = matgroup_kpc<NB>(nk);
  return sizeof(double2) * (size_t)nmat * kpc * NB * NB + sizeof(double) * (size_t)kpc * NB;
}

}  // namespace

}  // namespace kbe
