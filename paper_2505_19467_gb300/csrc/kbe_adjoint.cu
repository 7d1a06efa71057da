// Reverse mode (discrete adjoint) of one time step, FP64 history.
//
// kbe_backward differentiates a loss of the final-time occupations n_kb(t_N)
// with respect to the Peierls samples A_i and the interaction U by walking
// the steps n = N..1 backwards. Everything step n reads is the history
// triangle (rows < n are final once written) and I_{n-1}, itself a function
// of that history, so the step's intermediates (predictor and corrector
// rows, h, U, V, the Sigma and collision rows of every stage) are recomputed
// from the history, then the step's operations are transposed in reverse
// order. The transposes are those of the kernels' own arithmetic (the
// sweep in its (I^<, I^> - I^<) form, the DFT Sigma, the truncated power
// series of the propagators), so the gradient is that of the computed trajectory.
//
// Convention: for a complex variable z the adjoint lam_z is defined by
// dL = Re sum conj(lam_z) dz. A holomorphic use z = c w gives lam_w += conj(c)
// lam_z, an anti-holomorphic one z = c conj(w) gives lam_w += conj(lam_z) c;
// a matrix product Z = A B gives lam_A += lam_Z B^+ and lam_B += A^+ lam_Z.
//
// Pieces (forward operation -> kernel here):
//   collision row (a2), coefficients  -> adj_coef_kernel: lam of the Sigma row
//   collision row (a2), history       -> adj_hist_kernel: lam of every block
//   Sigma row (a1)                    -> DFT, sigma_adj_products_kernel, DFT
//   row / diagonal update (a4)        -> adj_rows_kernel, adj_uv_kernel,
//                                        adj_diag_kernel (series reversed)
//   h from A, mean field, shift (a3)  -> adj_hvec_kernel (dL/dA_i, dL/dU)
#include "kbe_adjoint_impl.cuh"
#include "kbe_adjoint_inst.cuh"

namespace kbe {

// compiled in kbe_adjoint_nb*.cu
KBE_ADJ_INSTANCES(extern, 1)
KBE_ADJ_INSTANCES(extern, 2)
KBE_ADJ_INSTANCES(extern, 3)
KBE_ADJ_INSTANCES(extern, 4)
KBE_ADJ_INSTANCES(extern, 6)
KBE_ADJ_INSTANCES(extern, 8)
KBE_ADJ_INSTANCES(extern, 12)
KBE_ADJ_INSTANCES(extern, 16)

// ---------------------------------------------------------- launchers ----

cudaError_t launch_unpack_fp64(const double2 *packed, double2 *out, size_t nblocks, size_t blk,
                               cudaStream_t st) {
  if (nblocks == 0 || blk == 0) return cudaSuccess;
  unpack_fp64_kernel<<<grid_for_count(nblocks * blk), 256, 0, st>>>(packed, out, nblocks, blk);
  return cudaGetLastError();
}

size_t adj_coef_workspace_bytes(const Mesh &m, int nmax) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  size_t part = 0;
  for (int r = 0; r <= nmax; ++r) {
    const CoefShape sh = coef_shape(m, r);
    if (sh.nz > 1) {
      const size_t b = (size_t)sh.nz * (r + 1) * 2 * blk * sizeof(double2);
      if (b > part) part = b;
    }
  }
  return part ? part : 256;
}

cudaError_t launch_adj_sweep(const Mesh &m, int n, double dt, const double2 *H, const double2 *Sig,
                             const double2 *lamI, double2 *lamSig, double2 *lamH, double2 *lamRowN,
                             double2 *coef_work, double2 *c1_work, cudaStream_t st, int quad) {
  KBE_NB_SWITCH(m.nb, return adj_sweep_nb<NB>(m, n, dt, H, Sig, lamI, lamSig, lamH, lamRowN, coef_work,
                                               c1_work, st, quad));
  return cudaErrorInvalidValue;
}

size_t adj_sigma_workspace_bytes(const Mesh &m, int n) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  return 3 * (size_t)(n + 1) * 2 * blk * sizeof(double2) + (size_t)(n + 1) * m.nb * m.nk * sizeof(double);
}

cudaError_t adj_sigma_row(const Mesh &m, const double *v_host, int n, double Un, const double *Ul_dev,
                          const double2 *Grow, const double2 *lamSig, double2 *lamRow, double *gU,
                          double2 *work, cudaStream_t st) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  const size_t row = (size_t)(n + 1) * 2 * blk;
  const long narr = (long)(n + 1) * 2 * m.nb * m.nb;
  double2 *GR = work, *LR = work + row, *GLR = work + 2 * row;
  // forward: G(R) = DFT_+(G(k)) / n_k; Sigma(k) = DFT_-(products(G(R)))
  cudaError_t e = launch_dft_rows(Grow, GR, narr, m.L0, m.L1, +1, 1.0 / m.nk, st);
  if (e != cudaSuccess) return e;
  // transpose of DFT_- is DFT_+, of DFT_+ / n_k is DFT_- / n_k
  e = launch_dft_rows(lamSig, LR, narr, m.L0, m.L1, +1, 1.0, st);
  if (e != cudaSuccess) return e;
  VMat vm;
  for (int i = 0; i < kMaxNb * kMaxNb; ++i) vm.v[i] = 0.0;
  for (int i = 0; i < m.nb * m.nb; ++i) vm.v[i] = v_host[i];
  double *gpart = (double *)(work + 3 * row);
  bool pair = m.nb >= 3;   // v = 1 - delta exactly: the closed form
  for (int a = 0; a < m.nb; ++a)
    for (int b = 0; b < m.nb; ++b) pair = pair && v_host[a * m.nb + b] == (a == b ? 0.0 : 1.0);
  KBE_NB_SWITCH(m.nb, e = adj_products_nb<NB>(pair, GR, LR, GLR, n, m.nk, Un, Ul_dev, vm, gpart, st));
  if (e != cudaSuccess) return e;
  adj_sigma_u_kernel<<<1, 256, 0, st>>>(gpart, n, m.nb * m.nk, Un, Ul_dev, gU);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dft_rows(GLR, lamRow, narr, m.L0, m.L1, -1, 1.0 / m.nk, st, true);
}

size_t adj_update_workspace_bytes(const Mesh &m) {
  const size_t blk = (size_t)m.nb * m.nb * m.nk;
  return ((size_t)kUvMaxSplit * 2 + 18) * blk * sizeof(double2);
}

cudaError_t launch_adj_update(const Mesh &m, int n, double dt, double theta, const double2 *h,
                              const double2 *U, const double2 *V, const double2 *Gprev, const double2 *Ip,
                              const double2 *Ic, const double2 *lam, double2 *lamGprev, double2 *lamIp,
                              double2 *lamIc, double2 *lamh, double2 *work, int *status, cudaStream_t st) {
  KBE_NB_SWITCH(m.nb, return adj_update_nb<NB>(m, n, dt, theta, h, U, V, Gprev, Ip, Ic, lam, lamGprev, lamIp,
                                                lamIc, lamh, work, status, st));
  return cudaErrorInvalidValue;
}

cudaError_t launch_adj_hvec(const Mesh &m, const HopTable &hop, const AdjHvecArgs &a, const double *v_host,
                            const double2 *lamh, cudaStream_t st) {
  HvecAdj p{};
  p.A = a.A;
  p.U = a.U;
  p.hf = a.hf;
  p.paper_shift = a.paper_shift;
  for (int i = 0; i < m.nb * m.nb; ++i) p.v[i] = v_host[i];
  p.rho_a = a.rho_a;
  p.rho_b = a.rho_b;
  p.ca = a.ca;
  p.cb = a.cb;
  p.lam_rho_a = a.lam_rho_a;
  p.lam_rho_b = a.lam_rho_b;
  p.lam_cur = a.lam_cur;
  p.cur_scale = a.cur_scale;
  p.gA = a.gA;
  p.gU_a = a.gU_a;
  p.gU_b = a.gU_b;
  KBE_NB_SWITCH(m.nb, return adj_hvec_nb<NB>(m, hop, p, lamh, st));
  return cudaErrorInvalidValue;
}

cudaError_t launch_adj_density(const Mesh &m, const double2 *lamRho, double scale, double2 *lamDiag,
                               cudaStream_t st) {
  const int total = m.nb * m.nb * m.nk;
  adj_density_kernel<<<(total + 255) / 256, 256, 0, st>>>(m.nb * m.nb, m.nk, lamRho, scale, lamDiag);
  return cudaGetLastError();
}

}  // namespace kbe
