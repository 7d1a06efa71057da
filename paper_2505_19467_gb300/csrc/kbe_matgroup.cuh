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
  // (A B)_ab of this thread's k-point
  __device__ __forceinline__ double2 mm(const double2 *A, const double2 *B) const {
    const double2 *Ar = A + kk * E + a * NB;
    const double2 *Bc = B + kk * E + b;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < NB; ++c) s = c_fma(Ar[c], Bc[c * NB], s);
    return s;
  }
  // (A B^+)_ab
  __device__ __forceinline__ double2 mm_adj(const double2 *A, const double2 *B) const {
    const double2 *Ar = A + kk * E + a * NB;
    const double2 *Br = B + kk * E + b * NB;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < NB; ++c) s = c_add(s, c_mulc(Ar[c], Br[c]));
    return s;
  }
};

// number of doublings s with (dt / 2^s) * max_k ||h_k||_rowsum <= 1/4, for
// all k-points of the CTA (uniform across the CTA); h in shared memory
template <int NB>
__device__ int doublings(const MatGroup<NB> &g, const double2 *h, int kpc, int nvalid, double dt,
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
  __shared__ int s_sh;
  if (threadIdx.x == 0) {
    double nu = 0.0;
    for (int i = 0; i < kpc * NB; ++i) nu = fmax(nu, red[i]);
    nu *= dt;
    int sc = 0;
    while (nu > 0.25 && sc < 40) {   // bounded: nu <= 2^40 / 4 covers any finite h
      nu *= 0.5;
      ++sc;
    }
    s_sh = sc;
  }
  __syncthreads();
  return s_sh;
}

// U_dt and V_dt of h (shared memory), element (a, b) returned in u, v;
// P, Q, W are shared scratch of KPC * N_b^2 each.
template <int NB>
__device__ void exp_and_phi(const MatGroup<NB> &g, const double2 *h, double tau, int s, double2 *P,
                            double2 *Q, double2 *W, double2 &u, double2 &v) {
  const int o = g.kk * g.E + g.e;
  const double2 one = make_double2(g.a == g.b ? 1.0 : 0.0, 0.0);
  P[o] = one;
  u = one;
  v = make_double2(0.0, -tau * one.x);   // -i tau P_0 / 1
  __syncthreads();
  for (int m = 1; m <= 14; ++m) {
    double2 t = g.mm(P, h);
    t = make_double2(tau * t.y / m, -tau * t.x / m);   // (-i tau / m) (P h)
    __syncthreads();
    P[o] = t;
    u = c_add(u, t);
    v = c_add(v, make_double2(tau * t.y / (m + 1), -tau * t.x / (m + 1)));
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
  double2 s = make_double2(0.0, 0.0);
#pragma unroll
  for (int c = 0; c < NB; ++c) s = c_add(s, c_mulc(Bc[c * NB], Ac[c * NB]));
  return s;
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
