// Internal declarations of libkbe (CUDA, sm_103a). Not part of the C ABI.
//
// Device layout (all c128 interleaved as double2):
//   history   H[tri(i,j)][x][a][b][k]   i >= j, tri(i,j) = i(i+1)/2 + j
//   rows      R[l][x][a][b][k]          (self-energy row, collision row)
//   per-k     M[a][b][k]                (h, U, V, W), lam[a][k]
// k is the fastest index so that consecutive threads (consecutive k) read
// consecutive 16-byte elements.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

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

// ---- status word written by kernels (sticky, read by the host) -----------
enum : int { kDevOk = 0, kDevNonFinite = 1, kDevEigNoConv = 2 };

// ---- kernels launch wrappers (return cudaGetLastError()) ------------------
// a1 self-energy row
cudaError_t launch_dft_rows(const double2 *in, double2 *out, long narr, int L0, int L1, int sign,
                            double scale, cudaStream_t st);
cudaError_t launch_sigma_products(const Mesh &m, const double *v, int n, double Un,
                                  const double *Ul_dev, const double2 *GR, double2 *SR,
                                  cudaStream_t st);
size_t sigma_workspace_bytes(const Mesh &m, int n);
cudaError_t sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                      const double2 *Grow, double2 *Sig, double2 *work, cudaStream_t st);

// a2 collision row. H is the history triangle in the precision's storage
// (double2 / float4 hi-lo pairs / float2), each block holding G^< and
// dG = G^< - G^>; work holds the coefficient rows and the l-split partial
// sums (sweep_workspace_bytes).
bool sweep_supported(int nb);
bool precision_supported(int prec);
size_t history_elem_bytes(int prec);
size_t sweep_workspace_bytes(const Mesh &m, int n, int prec);
int sweep_splits(const Mesh &m, int n);   // CTAs sharing one output's l range
cudaError_t launch_pack(int prec, const double2 *src, void *dst, size_t nblocks, size_t blk,
                        cudaStream_t st);
cudaError_t launch_sweep(const Mesh &m, int n, double dt, int precision, const void *H,
                         const double2 *Sig, double2 *I, void *work, cudaStream_t st);

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
                                 cudaStream_t st);
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
                               cudaStream_t st);

// a4 update: rows j < n and the time diagonal (h, U, V of the step)
cudaError_t launch_update_row(const Mesh &m, int n, double dt, double theta, const double2 *h,
                              const double2 *U, const double2 *V, const double2 *Gprev,
                              const double2 *Iprev, const double2 *Icur, double2 *out,
                              cudaStream_t st);

// a5 observables
struct ObsParams {
  double Abar, Un;
  int hf, paper_shift;
  double v[kMaxNb * kMaxNb];
};
cudaError_t launch_observables(const Mesh &m, const HopTable &hop, const ObsParams &p,
                               const double2 *Gdiag, const double2 *Idiag, const double2 *rho_n,
                               double *obs_out, double *nkb_out, int *status, cudaStream_t st);

// message returned by kbe_last_error(NULL) on this thread
void set_last_error(const std::string &msg);

}  // namespace kbe
