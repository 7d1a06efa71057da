// C ABI of libkbe: handle life cycle, the Algorithm 1 step schedule on the
// device-resident history, and the stateless per-row operations.
//
// One step n (P(EC)^n_corr E, Algorithm 1 of the paper):
//   predictor : h from the extrapolated density, props, update with I_{n-1}
//   corrector : density of the current row -> h, props; Sigma row (a1);
//               collision row (a2); update with (I_{n-1} + I_n)/2 (a4)
//   final     : Sigma row + collision row -> I_n (kept for step n+1),
//               local density, observables (a5)
// Everything is enqueued on the handle's stream; nothing returns to the host
// inside a step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kbe_internal.cuh"

using kbe::Mesh;
using kbe::tri;

struct kbe_handle {
  kbe_config cfg{};
  Mesh mesh{};
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t blk = 0;   // complex numbers in one (component) block: nb*nb*nk
  int nb2 = 0;

  // host copies of the inputs
  int nhop = 0;
  std::vector<int> hopR;
  std::vector<double> hopT;
  std::vector<double> Useq{0.0};
  std::vector<double> v;
  std::vector<double> A;
  double dir[2] = {1.0, 0.0};
  std::vector<double> dipE;    // dipole field samples
  double2 *d_dipM = nullptr;   // dipole coupling (device)

  // device arena
  void *H = nullptr;           // history triangle (G^<, dG = G^< - G^>) in the precision's storage
  size_t esz = 16;             // bytes per stored complex number
  double2 *Wrow[2] = {nullptr, nullptr};   // FP64 (G^<, G^>) rows n-1 and n (ring)
  void *coef = nullptr;        // sweep workspace: coefficient rows + l-split partial sums
  double2 *Ip = nullptr;       // I row n-1
  double2 *Ic = nullptr;       // I row n
  double2 *Ip0 = nullptr, *Ic0 = nullptr;   // their order after kbe_reset
  double2 *Sig = nullptr;      // Sigma row
  double2 *work = nullptr;     // Sigma scratch
  double2 *U = nullptr, *V = nullptr, *hk = nullptr;   // step propagators and h, per k
  double2 *rho = nullptr;      // [(nt_max+2)][nb][nb]; slot nt_max+1 = current estimate
  double *obs = nullptr;       // [(nt_max+1)][6]
  double *nkb = nullptr;       // [(nt_max+1)][nk][nb]
  int *status = nullptr;
  double *obs_part = nullptr;            // per-CTA partial sums of the observables kernel
  unsigned *obs_ticket = nullptr;        // its last-CTA counter (kept at 0 between launches)
  int *d_skip = nullptr;                 // corrector passes skipped once converged (corr_tol > 0)
  unsigned long long *d_maxdiff = nullptr;   // max |G^< change| of the last corrector pass (bits)
  int *d_iters = nullptr;                // corrector passes run at each step [(nt_max+1)]
  int *d_hopR = nullptr;
  double2 *d_hopT = nullptr;
  double *d_U = nullptr;       // U(t_l) samples, nt_max+1
  size_t bytes = 0;

  int n = -1;                  // last completed row
  bool ham_set = false;
  kbe_status sticky = KBE_OK;
  bool poisoned = false;   // a timed-out copy may have landed after its CTA exited: recreate the handle
  std::string err;

  // graph replay of kbe_step (kbe_set_graphs): one instantiated graph per
  // (first row, step count, order of the I ring), valid for the current inputs
  bool graphs = false;
  kbe::GraphCache<std::tuple<int, int, int>> gcache;
  unsigned graph_gen = 0;   // bumped whenever captured kernels would carry stale inputs
  int inject = 0;   // one-shot fault injection for the timeout test (kbe_debug_inject)

  // reverse mode: one device arena, allocated by the first kbe_backward
  void *adj = nullptr;
  size_t adj_bytes = 0;

  // profiling
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<double> ev_flops, ev_flops_x, ev_bytes;
  size_t ev_used = 0;
  struct PhaseEv {
    cudaEvent_t a, b;
    int phase;
    double flops;
  };
  std::vector<PhaseEv> bev;    // backward phases
  size_t bev_used = 0;
  kbe_profile_stats stats{};
};

namespace {

// an NVTX range over one phase of a step, for timeline tools (nsys, ncu
// --nvtx); the calls cost next to nothing when no tool is attached. The range
// covers the host's enqueueing of the phase's kernels.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

thread_local std::string g_create_err;

kbe_status fail(kbe_handle *h, kbe_status s, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return s;
}

kbe_status cuda_fail(kbe_handle *h, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (h) h->sticky = KBE_ERR_CUDA;
  return fail(h, KBE_ERR_CUDA, m);
}

bool nb_ok(int nb) { return kbe::sweep_supported(nb); }

double U_at(const kbe_handle *h, int i) {
  return h->Useq.size() == 1 ? h->Useq[0] : h->Useq[(size_t)i];
}

double A_at(const kbe_handle *h, int i) {
  if (h->A.empty()) return 0.0;
  if (i < 0) i = 0;
  if (i >= (int)h->A.size()) i = (int)h->A.size() - 1;
  return h->A[(size_t)i];
}

kbe::HopTable hop_table(const kbe_handle *h) {
  kbe::HopTable t;
  t.nhop = h->nhop;
  t.R = h->d_hopR;
  t.T = h->d_hopT;
  t.d0 = h->dir[0];
  t.d1 = h->cfg.dim == 2 ? h->dir[1] : 0.0;
  return t;
}

template <typename T>
cudaError_t dalloc(kbe_handle *h, T **p, size_t count) {
  size_t b = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void **)p, b);
  if (e == cudaSuccess) h->bytes += b;
  return e;
}

void drop_graphs(kbe_handle *h) {
  h->gcache.clear();
  ++h->graph_gen;
}

void free_all(kbe_handle *h) {
  drop_graphs(h);
  void *ptrs[] = {h->H, h->Wrow[0], h->Wrow[1], h->coef, h->Ip, h->Ic, h->Sig, h->work, h->U, h->V,
                  h->hk, h->rho, h->obs, h->nkb, h->status, h->obs_part, h->obs_ticket, h->d_hopR, h->d_hopT, h->d_U,
                  h->d_dipM, h->adj, h->d_skip, h->d_maxdiff, h->d_iters};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto &pr : h->ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  h->ev.clear();
  for (auto &pe : h->bev) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  h->bev.clear();
}


// collision sweep flops of one launch at row n: the method's count with the
// G^> form of Eq. 6 (3 N_b^3 complex multiply-adds per stored block, ~24 n^2
// N_b^3 n_k flops) and the count the kernel executes with the (I^<, I^> - I^<)
// form (2 products per node, 3 at the two trapezoid end nodes of [0, t_j]).
// The three-multiplication FP64 kernel issues 3 DFMAs per complex multiply-add
// instead of 4, plus one DADD per history element and column (the element's
// re + im, shared by N_b products): its FP64-pipe operations, counted at 2
// flops each as the FMA probe counts them, are (3/4 + 1/(4 N_b)) of the count.
double sweep_flops(const kbe_handle *h, int n) {
  const double nb3 = (double)h->cfg.nb * h->cfg.nb * h->cfg.nb;
  const double cm = 2.0 * (n + 1.0) * (n + 1.0) + (double)n * (n + 3.0);
  return 8.0 * cm * nb3 * h->mesh.nk;
}
// (the tensor-core form: the flops its MMAs execute, hi and lo parts included)
double sweep_flops_executed(const kbe_handle *h, int n) {
  if (h->cfg.precision == KBE_PREC_F16X2) return kbe::sweep_tc_flops(h->mesh, h->cfg.precision, h->cfg.quadrature, n);
  const double nb3 = (double)h->cfg.nb * h->cfg.nb * h->cfg.nb;
  const double cm = 2.0 * n * (double)n + 6.0 * n + 2.0;
  const double f3m = kbe::use_f64m(h->mesh, h->cfg.precision) ? 0.75 + 0.25 / h->cfg.nb : 1.0;
  return 8.0 * cm * nb3 * h->mesh.nk * f3m;
}
double sweep_bytes(const kbe_handle *h, int n) {
  const double blk2 = 2.0 * (double)h->blk;
  const double tri_blocks = (n + 1.0) * (n + 2.0) / 2.0;
  // history triangle read once in its storage, Sigma row read, I row written (FP64)
  return blk2 * (tri_blocks * (double)h->esz + 2.0 * (n + 1.0) * 16.0);
}

// FP64 (G^<, G^>) copy of row i: the ring of the two newest rows (valid for
// i = n-1, n)
double2 *frow(kbe_handle *h, int i) { return h->Wrow[i & 1]; }

// store row i into the history triangle: (G^<, dG) in the storage format
kbe_status publish(kbe_handle *h, int i, const int *skip = nullptr) {
  char *dst = (char *)h->H + kbe::history_row_offset(h->mesh, h->cfg.precision, i);
  cudaError_t e = kbe::launch_pack(h->cfg.precision, frow(h, i), dst, (size_t)(i + 1), h->blk, h->stream, skip,
                                   h->cfg.nb, i, h->cfg.nt_max + 1);
  if (e != cudaSuccess) return cuda_fail(h, e, "publish row");
  if (h->prof) h->stats.launches += 1;
  return KBE_OK;
}

kbe_status evaluate_row(kbe_handle *h, int n, const int *skip = nullptr) {
  NvtxRange nv("kbe: Sigma row + collision sweep");
  const Mesh &m = h->mesh;
  double2 *Hrow = frow(h, n);
  const double *Ul = h->Useq.size() == 1 ? nullptr : h->d_U;
  // the complex64 and split-FP16 forms hold Sigma in complex FP32 (their coefficient rows round
  // it to complex64); the complex64 form transforms row n from its complex64 history copy
  const bool f32 = h->cfg.precision == KBE_PREC_C64 || h->cfg.precision == KBE_PREC_F16X2;
  const float2 *h32 = h->cfg.precision == KBE_PREC_C64
                          ? (const float2 *)((const char *)h->H + kbe::history_row_offset(m, KBE_PREC_C64, n))
                          : nullptr;
  cudaError_t e = kbe::sigma_row(m, h->v.data(), n, U_at(h, n), Ul, Hrow, h->Sig, h->work, h->stream, skip, f32,
                                 h32, f32);
  if (e != cudaSuccess) return cuda_fail(h, e, "sigma_row");
  const bool timed = h->prof;
  if (timed) {
    if (h->ev_used == h->ev.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      h->ev.push_back({a, b});
      h->ev_flops.push_back(0);
      h->ev_flops_x.push_back(0);
      h->ev_bytes.push_back(0);
    }
    cudaEventRecord(h->ev[h->ev_used].first, h->stream);
  }
  e = kbe::launch_sweep(m, n, h->cfg.dt, h->cfg.precision, h->H, h->Sig, h->Ic, h->coef, h->stream, skip,
                        h->cfg.quadrature, h->status, h->inject, h->cfg.nt_max + 1, f32);
  h->inject = 0;
  if (e != cudaSuccess) return cuda_fail(h, e, "collision sweep");
  if (timed) {
    cudaEventRecord(h->ev[h->ev_used].second, h->stream);
    h->ev_flops[h->ev_used] = sweep_flops(h, n);
    h->ev_flops_x[h->ev_used] = sweep_flops_executed(h, n);
    h->ev_bytes[h->ev_used] = sweep_bytes(h, n);
    h->ev_used++;
    h->stats.launches += 5 + (kbe::sweep_splits(h->mesh, n, h->cfg.precision, h->cfg.quadrature) > 1 ? 1 : 0);
  }
  return KBE_OK;
}

kbe_status build_props(kbe_handle *h, int n, const double2 *ra, const double2 *rb, double ca, double cb,
                       double2 *hk = nullptr, double2 *Uk = nullptr, double2 *Vk = nullptr,
                       const int *skip = nullptr) {
  NvtxRange nv("kbe: propagators");
  kbe::PropParams p{};
  p.A = A_at(h, n - 1);
  p.rho_a = ra;
  p.rho_b = rb;
  p.ca = ca;
  p.cb = cb;
  p.Umid = 0.5 * (U_at(h, n - 1) + U_at(h, n));
  p.hf = h->cfg.hf;
  p.paper_shift = h->cfg.paper_shift;
  for (int i = 0; i < h->nb2; ++i) p.v[i] = h->v[(size_t)i];
  p.dipM = h->dipE.empty() ? nullptr : h->d_dipM;
  p.dipE = (n - 1 < (int)h->dipE.size()) ? h->dipE[(size_t)(n - 1)] : 0.0;
  cudaError_t e = kbe::launch_build_props(h->mesh, hop_table(h), p, h->cfg.dt, nullptr, hk ? hk : h->hk,
                                          Uk ? Uk : h->U, Vk ? Vk : h->V, h->stream, skip);
  if (e != cudaSuccess) return cuda_fail(h, e, "build_props");
  if (h->prof) h->stats.launches += 1;
  return KBE_OK;
}

kbe_status update(kbe_handle *h, int n, double theta, const int *skip = nullptr,
                  unsigned long long *maxdiff = nullptr) {
  NvtxRange nv("kbe: row update");
  double2 *prev = frow(h, n - 1);
  double2 *row = frow(h, n);
  // the update kernels also store row n into the history triangle ("publish")
  char *hist = (char *)h->H + kbe::history_row_offset(h->mesh, h->cfg.precision, n);
  cudaError_t e = kbe::launch_update_row(h->mesh, n, h->cfg.dt, theta, h->hk, h->U, h->V, prev, h->Ip,
                                         h->Ic, row, h->stream, skip, maxdiff, hist, h->cfg.precision,
                                         h->cfg.nt_max + 1);
  if (e != cudaSuccess) return cuda_fail(h, e, "update_row");
  if (h->prof) h->stats.launches += 2;
  return KBE_OK;
}

kbe_status density(kbe_handle *h, int n, double2 *out, const int *skip = nullptr) {
  cudaError_t e = kbe::launch_local_density(h->mesh, frow(h, n) + (size_t)n * 2 * h->blk, out, h->stream, skip);
  if (e != cudaSuccess) return cuda_fail(h, e, "local_density");
  if (h->prof) h->stats.launches += 1;
  return KBE_OK;
}

kbe_status observables(kbe_handle *h, int n, const double2 *Irow) {
  kbe::ObsParams p{};
  p.Abar = 0.5 * (A_at(h, n - 1) + A_at(h, n));
  p.Un = U_at(h, n);
  p.hf = h->cfg.hf;
  p.paper_shift = h->cfg.paper_shift;
  for (int i = 0; i < h->nb2; ++i) p.v[i] = h->v[(size_t)i];
  cudaError_t e = kbe::launch_observables(h->mesh, hop_table(h), p, frow(h, n) + (size_t)n * 2 * h->blk,
                                          Irow + (size_t)n * 2 * h->blk, h->rho + (size_t)n * h->nb2,
                                          h->obs + (size_t)n * 6, h->nkb + (size_t)n * h->mesh.nk * h->cfg.nb,
                                          h->status, h->obs_part, h->obs_ticket, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "observables");
  if (h->prof) h->stats.launches += 1;
  return KBE_OK;
}

kbe_status one_step(kbe_handle *h) {
  NvtxRange nv("kbe: step");
  const int n = h->n + 1;
  const int nb2 = h->nb2;
  double2 *r1 = h->rho + (size_t)(n - 1) * nb2;
  double2 *r2 = h->rho + (size_t)(n >= 2 ? n - 2 : 0) * nb2;
  double2 *rcur = h->rho + (size_t)(h->cfg.nt_max + 1) * nb2;
  kbe_status s;
  // predictor: density extrapolated to the midpoint, Ibar = I_{n-1}
  if ((s = build_props(h, n, r1, r2, n >= 2 ? 1.5 : 1.0, n >= 2 ? -0.5 : 0.0)) != KBE_OK) return s;
  if ((s = update(h, n, 0.0)) != KBE_OK) return s;
  // correctors: a fixed count, or (corr_tol > 0) up to n_corr passes until the
  // largest change of the G^< row is <= corr_tol (Algorithm 1's break), decided
  // on the device: once converged, the remaining passes' kernels return at once
  const bool tol = h->cfg.corr_tol > 0.0;
  const int *skip = tol ? h->d_skip : nullptr;
  unsigned long long *md = tol ? h->d_maxdiff : nullptr;
  if (tol) {
    cudaError_t e = cudaMemsetAsync(h->d_skip, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_maxdiff, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_iters + n, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "corrector flags");
  }
  for (int c = 0; c < h->cfg.n_corr; ++c) {
    if ((s = density(h, n, rcur, skip)) != KBE_OK) return s;
    if ((s = build_props(h, n, r1, rcur, 0.5, 0.5, nullptr, nullptr, nullptr, skip)) != KBE_OK) return s;
    if ((s = evaluate_row(h, n, skip)) != KBE_OK) return s;
    if ((s = update(h, n, 0.5, skip, md)) != KBE_OK) return s;
    if (tol) {
      cudaError_t e = kbe::launch_corr_check(h->d_maxdiff, h->cfg.corr_tol, h->d_skip, h->d_iters + n, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "corrector check");
    }
  }
  if ((s = evaluate_row(h, n)) != KBE_OK) return s;
  if ((s = density(h, n, h->rho + (size_t)n * nb2)) != KBE_OK) return s;
  if ((s = observables(h, n, h->Ic)) != KBE_OK) return s;
  std::swap(h->Ip, h->Ic);
  h->n = n;
  return KBE_OK;
}

// ---- reverse mode ----------------------------------------------------------
// Pointers into the reverse-mode arena. Row slots hold (nt_max+1) blocks of
// (x, a, b, k) pairs; per-stage arrays are indexed by the stage c (0 =
// predictor, 1..n_corr = correctors, n_corr + 1 = the final evaluation).
struct AdjPtrs {
  double2 *lamH;          // adjoint of the history triangle, (G^<, G^>) per block
  double2 *rowp, *Ip, *sigp;   // recomputed row n-1 (G^<, G^>), I_{n-1}, Sigma_{n-1}
  double2 *rows;          // stage rows c = 0..n_corr
  double2 *sigs;          // Sigma rows of stages 1..n_corr and the final one
  double2 *Is;            // collision rows of stages 1..n_corr
  double2 *lst;           // adjoints of stage rows 0..n_corr-1
  double2 *hUV;           // (h, U, V) per k of every stage
  double2 *cur;           // current density of stages 1..n_corr
  double2 *lamIa, *lamIb, *lamIc, *lamSig;
  double2 *save;          // the stored row n while its stages are republished
  double2 *sigw, *coefw, *updw, *lamh, *lamRho, *c1w;
  double *gA, *gU;        // dL/dA_i; dL/dU_i per U sample (summed for a constant U)
  size_t row;             // complex numbers per row slot
};

size_t adj_carve(const kbe_config *cfg, const Mesh &m, char *base, AdjPtrs *p) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *r = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  const size_t T = (size_t)cfg->nt_max, nb2 = (size_t)cfg->nb * cfg->nb, blk = nb2 * m.nk;
  const size_t nc = (size_t)cfg->n_corr, c16 = sizeof(double2);
  p->row = (T + 1) * 2 * blk;
  const size_t R = p->row * c16;
  p->lamH = (double2 *)take((tri((int)T, (int)T) + 1) * 2 * blk * c16);
  p->rowp = (double2 *)take(R);
  p->Ip = (double2 *)take(R);
  p->sigp = (double2 *)take(R);
  p->rows = (double2 *)take((nc + 1) * R);
  p->sigs = (double2 *)take((nc + 1) * R);
  p->Is = (double2 *)take(nc * R);
  p->lst = (double2 *)take(nc * R);
  p->hUV = (double2 *)take((nc + 1) * 3 * blk * c16);
  p->cur = (double2 *)take((nc + 1) * nb2 * c16);
  p->lamIa = (double2 *)take(R);
  p->lamIb = (double2 *)take(R);
  p->lamIc = (double2 *)take(R);
  p->lamSig = (double2 *)take(R);
  p->save = (double2 *)take(R);
  p->sigw = (double2 *)take(kbe::adj_sigma_workspace_bytes(m, (int)T));
  p->coefw = (double2 *)take(kbe::adj_coef_workspace_bytes(m, (int)T));
  p->updw = (double2 *)take(kbe::adj_update_workspace_bytes(m));
  p->lamh = (double2 *)take(blk * c16);
  p->lamRho = (double2 *)take((T + 1) * nb2 * c16);
  p->c1w = (double2 *)take((T + 1) * blk * c16);
  p->gA = (double *)take(T * sizeof(double));
  p->gU = (double *)take((T + 1) * sizeof(double));
  return off;
}

// backward phase timing (profiling only): open() records the start event of
// a phase, close() its end; each phase is also an NVTX range (always, closed
// on every exit path)
constexpr const char *kBackwardPhase[4] = {"kbe_backward: recompute", "kbe_backward: collision transposes",
                                           "kbe_backward: sigma transposes", "kbe_backward: update and h transposes"};
struct PhaseTimer {
  kbe_handle *h;
  size_t cur = (size_t)-1;
  bool nvtx_open = false;
  explicit PhaseTimer(kbe_handle *hh) : h(hh) {}
  PhaseTimer(const PhaseTimer &) = delete;
  PhaseTimer &operator=(const PhaseTimer &) = delete;
  ~PhaseTimer() {
    if (nvtx_open) nvtxRangePop();
  }
  void open(int phase, double flops = 0.0) {
    if (nvtx_open) nvtxRangePop();
    nvtxRangePushA(kBackwardPhase[phase]);
    nvtx_open = true;
    if (!h->prof) return;
    if (h->bev_used == h->bev.size()) {
      kbe_handle::PhaseEv pe{};
      cudaEventCreate(&pe.a);
      cudaEventCreate(&pe.b);
      h->bev.push_back(pe);
    }
    cur = h->bev_used++;
    h->bev[cur].phase = phase;
    h->bev[cur].flops = flops;
    cudaEventRecord(h->bev[cur].a, h->stream);
  }
  void close() {
    if (nvtx_open) nvtxRangePop();
    nvtx_open = false;
    if (!h->prof || cur == (size_t)-1) return;
    cudaEventRecord(h->bev[cur].b, h->stream);
    cur = (size_t)-1;
  }
};

// flops of the collision-row transposes at row n, in complex multiply-adds per
// N_b^3 n_k: the coefficient transpose takes 2 per pair (l, j) off the diagonal
// and 3 on it; the history transpose 4 per block below the diagonal (2 per use)
// and 3 on it (the few Gregory end nodes with extra terms are not counted)
double adj_sweep_flops(const kbe_handle *h, int n) {
  const double nb3 = (double)h->cfg.nb * h->cfg.nb * h->cfg.nb, N = n;
  const double coef = 2.0 * N * (N + 1) + 3.0 * (N + 1);
  const double hist = 2.0 * N * (N + 1) + 3.0 * (N + 1);
  return 8.0 * (coef + hist) * nb3 * h->mesh.nk;
}

#define KBE_TRY(expr, where)                          \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// Step n in reverse: recompute the step from the history (rows < n) and
// I_{n-1}, then transpose its operations, last first. lamIcur is the adjoint
// of I_n (complete), lamIprev accumulates that of I_{n-1}.
kbe_status backward_step(kbe_handle *h, const AdjPtrs &P, int n, int nc, double2 *lamIcur, double2 *lamIprev) {
  const Mesh &m = h->mesh;
  const size_t blk = h->blk, nb2 = (size_t)h->nb2;
  const double dt = h->cfg.dt;
  const double *Ul = h->Useq.size() == 1 ? nullptr : h->d_U;   // as the forward's Sigma rows
  const double Un = U_at(h, n), Up = U_at(h, n - 1);
  cudaStream_t st = h->stream;   // nc: the corrector passes the forward ran at step n
  const double *v = h->v.data();
  double2 *Hd = (double2 *)h->H;
  double2 *histN = Hd + tri(n, 0) * 2 * blk;
  const size_t rowc = (size_t)(n + 1) * 2 * blk;
  auto row = [&](int c) { return P.rows + (size_t)c * P.row; };
  auto sig = [&](int c) { return P.sigs + (size_t)(c - 1) * P.row; };
  auto Ist = [&](int c) { return P.Is + (size_t)(c - 1) * P.row; };
  auto lst = [&](int c) { return P.lst + (size_t)c * P.row; };
  auto hk = [&](int c) { return P.hUV + (size_t)c * 3 * blk; };
  auto Uk = [&](int c) { return P.hUV + ((size_t)c * 3 + 1) * blk; };
  auto Vk = [&](int c) { return P.hUV + ((size_t)c * 3 + 2) * blk; };
  auto cur = [&](int c) { return P.cur + (size_t)c * nb2; };
  auto rho = [&](int i) { return h->rho + (size_t)i * nb2; };
  auto lrho = [&](int i) { return P.lamRho + (size_t)i * nb2; };
  const int n2 = n >= 2 ? n - 2 : 0;
  const double ca0 = n >= 2 ? 1.5 : 1.0, cb0 = n >= 2 ? -0.5 : 0.0;

  PhaseTimer tm(h);
  // ---- recompute step n (the forward's order and kernels) ----
  tm.open(0);
  KBE_TRY(cudaMemcpyAsync(P.save, histN, rowc * sizeof(double2), cudaMemcpyDeviceToDevice, st), "backward save");
  KBE_TRY(kbe::launch_unpack_fp64(Hd + tri(n - 1, 0) * 2 * blk, P.rowp, (size_t)n, blk, st), "backward unpack");
  KBE_TRY(kbe::sigma_row(m, v, n - 1, Up, Ul, P.rowp, P.sigp, h->work, st), "backward sigma");
  const int quad = h->cfg.quadrature;
  KBE_TRY(kbe::launch_sweep(m, n - 1, dt, KBE_PREC_FP64, h->H, P.sigp, P.Ip, h->coef, st, nullptr, quad),
          "backward sweep");
  kbe_status s = build_props(h, n, rho(n - 1), rho(n2), ca0, cb0, hk(0), Uk(0), Vk(0));
  if (s != KBE_OK) return s;
  KBE_TRY(kbe::launch_update_row(m, n, dt, 0.0, hk(0), Uk(0), Vk(0), P.rowp, P.Ip, nullptr, row(0), st),
          "backward update");
  KBE_TRY(kbe::launch_pack(KBE_PREC_FP64, row(0), histN, (size_t)(n + 1), blk, st), "backward pack");
  for (int c = 1; c <= nc; ++c) {
    KBE_TRY(kbe::launch_local_density(m, row(c - 1) + (size_t)n * 2 * blk, cur(c), st), "backward density");
    if ((s = build_props(h, n, rho(n - 1), cur(c), 0.5, 0.5, hk(c), Uk(c), Vk(c))) != KBE_OK) return s;
    KBE_TRY(kbe::sigma_row(m, v, n, Un, Ul, row(c - 1), sig(c), h->work, st), "backward sigma");
    KBE_TRY(kbe::launch_sweep(m, n, dt, KBE_PREC_FP64, h->H, sig(c), Ist(c), h->coef, st, nullptr, quad),
            "backward sweep");
    KBE_TRY(kbe::launch_update_row(m, n, dt, 0.5, hk(c), Uk(c), Vk(c), P.rowp, P.Ip, Ist(c), row(c), st),
            "backward update");
    KBE_TRY(kbe::launch_pack(KBE_PREC_FP64, row(c), histN, (size_t)(n + 1), blk, st), "backward pack");
  }
  KBE_TRY(kbe::sigma_row(m, v, n, Un, Ul, row(nc), sig(nc + 1), h->work, st), "backward sigma");
  tm.close();

  // ---- transpose ----
  double2 *lamN = P.lamH + tri(n, 0) * 2 * blk;       // row n (the final row's adjoint)
  double2 *lamP = P.lamH + tri(n - 1, 0) * 2 * blk;   // row n-1
  const kbe::HopTable hop = hop_table(h);
  // density rho_n of the final row, used by later steps
  KBE_TRY(kbe::launch_adj_density(m, lrho(n), 1.0 / m.nk, lamN + (size_t)n * 2 * blk, st), "backward density");
  // final evaluation: I_n = sweep(Sigma(row), history with row n)
  tm.open(1, adj_sweep_flops(h, n));
  KBE_TRY(kbe::launch_adj_sweep(m, n, dt, Hd, sig(nc + 1), lamIcur, P.lamSig, P.lamH, lamN, P.coefw, P.c1w, st, quad),
          "backward adj sweep");
  tm.close();
  tm.open(2);
  KBE_TRY(kbe::adj_sigma_row(m, v, n, Un, Ul, row(nc), P.lamSig, lamN, P.gU, P.sigw, st), "backward adj sigma");
  tm.close();
  kbe::AdjHvecArgs a{};
  a.U = 0.5 * (Up + Un);   // U_mid of the step
  a.hf = h->cfg.hf;
  a.paper_shift = h->cfg.paper_shift;
  a.A = A_at(h, n - 1);
  a.gA = P.gA + (n - 1);
  a.gU_a = P.gU + (n - 1);
  a.gU_b = P.gU + n;
  for (int c = nc; c >= 1; --c) {
    double2 *lamS = (c == nc) ? lamN : lst(c);
    double2 *lamPS = lst(c - 1);
    tm.open(3);
    KBE_TRY(cudaMemsetAsync(lamPS, 0, rowc * sizeof(double2), st), "backward memset");
    KBE_TRY(cudaMemsetAsync(P.lamIc, 0, rowc * sizeof(double2), st), "backward memset");
    KBE_TRY(kbe::launch_adj_update(m, n, dt, 0.5, hk(c), Uk(c), Vk(c), P.rowp, P.Ip, Ist(c), lamS, lamP,
                                   lamIprev, P.lamIc, P.lamh, P.updw, h->status, st),
            "backward adj update");
    a.rho_a = rho(n - 1);
    a.rho_b = cur(c);
    a.ca = a.cb = 0.5;
    a.lam_rho_a = lrho(n - 1);
    a.lam_rho_b = nullptr;
    a.lam_cur = lamPS + (size_t)n * 2 * blk;
    a.cur_scale = 0.5 / m.nk;
    KBE_TRY(kbe::launch_adj_hvec(m, hop, a, v, P.lamh, st), "backward adj h");
    // the stage's collision row saw the previous stage's row as row n
    KBE_TRY(kbe::launch_pack(KBE_PREC_FP64, row(c - 1), histN, (size_t)(n + 1), blk, st), "backward pack");
    tm.close();
    tm.open(1, adj_sweep_flops(h, n));
    KBE_TRY(kbe::launch_adj_sweep(m, n, dt, Hd, sig(c), P.lamIc, P.lamSig, P.lamH, lamPS, P.coefw, P.c1w, st, quad),
            "backward adj sweep");
    tm.close();
    tm.open(2);
    KBE_TRY(kbe::adj_sigma_row(m, v, n, Un, Ul, row(c - 1), P.lamSig, lamPS, P.gU, P.sigw, st),
            "backward adj sigma");
    tm.close();
  }
  double2 *lam0 = nc == 0 ? lamN : lst(0);
  tm.open(3);
  KBE_TRY(kbe::launch_adj_update(m, n, dt, 0.0, hk(0), Uk(0), Vk(0), P.rowp, P.Ip, nullptr, lam0, lamP,
                                 lamIprev, nullptr, P.lamh, P.updw, h->status, st),
          "backward adj update");
  a.rho_a = rho(n - 1);
  a.rho_b = rho(n2);
  a.ca = ca0;
  a.cb = cb0;
  a.lam_rho_a = lrho(n - 1);
  a.lam_rho_b = lrho(n2);
  a.lam_cur = nullptr;
  KBE_TRY(kbe::launch_adj_hvec(m, hop, a, v, P.lamh, st), "backward adj h");
  KBE_TRY(cudaMemcpyAsync(histN, P.save, rowc * sizeof(double2), cudaMemcpyDeviceToDevice, st),
          "backward restore");
  tm.close();
  return KBE_OK;
}

#undef KBE_TRY

// kbe_step through an instantiated graph: the first call for a given (row,
// count, I-ring order) captures the ordinary enqueue path on the handle's
// stream (nothing runs while capturing) and instantiates it; later calls with
// the same key replay it and only advance the host-side state.
kbe_status step_graph(kbe_handle *h, int nsteps) {
  const auto key = std::make_tuple(h->n, nsteps, h->Ip == h->Ip0 ? 0 : 1);
  cudaGraphExec_t exec = h->gcache.find(key);
  if (!exec) {
    cudaError_t e = kbe::dft_prepare(h->mesh.L0, h->mesh.L1);
    if (e == cudaSuccess) e = kbe::sweep_prepare(h->cfg.nb);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph prepare");
    const int n0 = h->n;
    double2 *ip = h->Ip, *ic = h->Ic;
    e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    kbe_status s = KBE_OK;
    for (int i = 0; i < nsteps && s == KBE_OK; ++i) s = one_step(h);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    // the capture only recorded: roll the host state back, then replay below
    h->n = n0;
    h->Ip = ip;
    h->Ic = ic;
    if (s != KBE_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      h->sticky = KBE_OK;
      return s != KBE_OK ? s : cuda_fail(h, e, "graph capture");
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    h->gcache.put(key, exec);
  }
  cudaError_t e = cudaGraphLaunch(exec, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
  for (int i = 0; i < nsteps; ++i) {   // the host-side state one_step keeps
    std::swap(h->Ip, h->Ic);
    h->n += 1;
  }
  return KBE_OK;
}

kbe_status check_device_status(kbe_handle *h) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  if (st & kbe::kDevNonFinite) {
    h->sticky = KBE_ERR_NONFINITE;
    return fail(h, KBE_ERR_NONFINITE, "non-finite value in the propagated state");
  }
  if (st & kbe::kDevEigNoConv) {
    h->sticky = KBE_ERR_NONFINITE;
    return fail(h, KBE_ERR_NONFINITE, "eigen-solver did not converge (non-finite or huge h)");
  }
  if (st & kbe::kDevTimeoutDrain) {
    h->sticky = KBE_ERR_TIMEOUT;
    h->poisoned = true;
    return fail(h, KBE_ERR_TIMEOUT,
                "a staged copy of the collision sweep did not complete and the copies in flight could not be "
                "drained: destroy and recreate the handle");
  }
  if (st & kbe::kDevTimeout) {
    h->sticky = KBE_ERR_TIMEOUT;
    return fail(h, KBE_ERR_TIMEOUT, "a staged copy of the collision sweep did not complete (bounded wait)");
  }
  return h->sticky;
}

bool mesh_ok(const kbe_mesh *m) {
  return m && nb_ok(m->nb) && m->L[0] >= 1 && m->L[1] >= 1 &&
         (long)m->L[0] * m->L[1] <= kbe::kMaxNk;
}

Mesh to_mesh(const kbe_mesh *m) { return Mesh{m->nb, m->L[0], m->L[1], m->L[0] * m->L[1]}; }

}  // namespace

// ---- one step in segments (batched systems) ---------------------------------
// The sequence of one_step cut at its n_corr + 1 collision sweeps: segment 0
// runs the predictor and stops before the first sweep, segments 1 .. n_corr
// finish the previous sweep and stop before the next, segment n_corr + 1
// finishes the last one and the step. A stopped segment has enqueued the Sigma
// row and the coefficient rows and hands back the sweep as a job, which the
// batch launches together with the other systems' (kbe_batch.cu); the
// arithmetic and the launch shapes are one_step's, so the results are bitwise
// one_step's. FP64 history only.
int step_segment_count(const kbe_handle *h) { return h->cfg.n_corr + 2; }

static kbe_status segment_eval_pre(kbe_handle *h, int n, const int *skip, kbe::SweepJob *job) {
  const double *Ul = h->Useq.size() == 1 ? nullptr : h->d_U;
  cudaError_t e = kbe::sigma_row(h->mesh, h->v.data(), n, U_at(h, n), Ul, frow(h, n), h->Sig, h->work, h->stream,
                                 skip, false);
  if (e == cudaSuccess)
    e = kbe::prepare_sweep_job(h->mesh, n, h->cfg.dt, h->H, h->Sig, h->Ic, h->coef, h->stream, skip,
                               h->cfg.quadrature, job);
  if (e != cudaSuccess) return cuda_fail(h, e, "sweep job");
  return KBE_OK;
}

kbe_status step_segment(kbe_handle *h, int seg, kbe::SweepJob *job, bool *has_job) {
  *has_job = false;
  if (h->cfg.precision != KBE_PREC_FP64) return fail(h, KBE_ERR_UNSUPPORTED, "step_segment: FP64 history only");
  const int nc = h->cfg.n_corr;
  const int n = h->n + 1;   // the row being computed (h->n advances at the last segment)
  const int nb2 = h->nb2;
  double2 *r1 = h->rho + (size_t)(n - 1) * nb2;
  double2 *r2 = h->rho + (size_t)(n >= 2 ? n - 2 : 0) * nb2;
  double2 *rcur = h->rho + (size_t)(h->cfg.nt_max + 1) * nb2;
  const bool tol = h->cfg.corr_tol > 0.0;
  const int *skip = tol ? h->d_skip : nullptr;
  unsigned long long *md = tol ? h->d_maxdiff : nullptr;
  kbe_status s;
  if (seg > 0) {   // the previous segment's sweep has run: its partial sums into I
    cudaError_t e = kbe::finish_sweep_job(*job, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sweep job finish");
  }
  if (seg == 0) {   // predictor: density extrapolated to the midpoint, Ibar = I_{n-1}
    if ((s = build_props(h, n, r1, r2, n >= 2 ? 1.5 : 1.0, n >= 2 ? -0.5 : 0.0)) != KBE_OK) return s;
    if ((s = update(h, n, 0.0)) != KBE_OK) return s;
    if (tol) {
      cudaError_t e = cudaMemsetAsync(h->d_skip, 0, sizeof(int), h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->d_maxdiff, 0, sizeof(unsigned long long), h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->d_iters + n, 0, sizeof(int), h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "corrector flags");
    }
  } else if (seg <= nc) {   // the corrector pass seg - 1 completes
    if ((s = update(h, n, 0.5, skip, md)) != KBE_OK) return s;
    if (tol) {
      cudaError_t e = kbe::launch_corr_check(h->d_maxdiff, h->cfg.corr_tol, h->d_skip, h->d_iters + n, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "corrector check");
    }
  }
  if (seg < nc) {   // corrector pass seg: its evaluation
    if ((s = density(h, n, rcur, skip)) != KBE_OK) return s;
    if ((s = build_props(h, n, r1, rcur, 0.5, 0.5, nullptr, nullptr, nullptr, skip)) != KBE_OK) return s;
    if ((s = segment_eval_pre(h, n, skip, job)) != KBE_OK) return s;
    *has_job = true;
    return KBE_OK;
  }
  if (seg == nc) {   // the final evaluation
    if ((s = segment_eval_pre(h, n, nullptr, job)) != KBE_OK) return s;
    *has_job = true;
    return KBE_OK;
  }
  if ((s = density(h, n, h->rho + (size_t)n * nb2)) != KBE_OK) return s;
  if ((s = observables(h, n, h->Ic)) != KBE_OK) return s;
  std::swap(h->Ip, h->Ic);
  h->n = n;
  return KBE_OK;
}

kbe_status step_segment_check(kbe_handle *h) {
  if (h->sticky != KBE_OK) return fail(h, h->sticky, "step: handle has a sticky error; reset it");
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "step: call kbe_reset first");
  if (h->n + 1 > h->cfg.nt_max) return fail(h, KBE_ERR_STATE, "step: past nt_max");
  if (h->cfg.precision != KBE_PREC_FP64 || h->prof || h->inject)
    return fail(h, KBE_ERR_UNSUPPORTED, "step: the batched sweep needs FP64 history, no profiling, no injection");
  return KBE_OK;
}

void kbe::set_last_error(const std::string &msg) { g_create_err = msg; }

// ---- pieces of kbe_step for a graph that spans several handles (kbe_batch) ----
kbe_status kbe::step_check(kbe_handle *h, int nsteps) {
  if (!h) return KBE_ERR_ARG;
  if (h->sticky != KBE_OK) return fail(h, h->sticky, "step: handle has a sticky error; reset it");
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "step: call kbe_reset first");
  if (nsteps < 0) return fail(h, KBE_ERR_ARG, "step: negative count");
  if (h->n + nsteps > h->cfg.nt_max) return fail(h, KBE_ERR_STATE, "step: past nt_max");
  return KBE_OK;
}

bool kbe::step_capturable(const kbe_handle *h) { return !h->prof && !h->inject && h->stream != nullptr; }

kbe_status kbe::step_prepare(kbe_handle *h) {
  cudaError_t e = kbe::dft_prepare(h->mesh.L0, h->mesh.L1);
  if (e == cudaSuccess) e = kbe::sweep_prepare(h->cfg.nb);
  return e == cudaSuccess ? KBE_OK : cuda_fail(h, e, "graph prepare");
}

// enqueue nsteps steps on the handle's stream (being captured by the caller)
// and roll the host-side state back: the steps run when the graph is replayed
kbe_status kbe::step_record(kbe_handle *h, int nsteps) {
  const int n0 = h->n;
  double2 *ip = h->Ip, *ic = h->Ic;
  kbe_status s = KBE_OK;
  for (int i = 0; i < nsteps && s == KBE_OK; ++i) s = one_step(h);
  h->n = n0;
  h->Ip = ip;
  h->Ic = ic;
  return s;
}

// the host-side state nsteps replayed steps leave (what one_step advances)
void kbe::step_advance(kbe_handle *h, int nsteps) {
  for (int i = 0; i < nsteps; ++i) {
    std::swap(h->Ip, h->Ic);
    h->n += 1;
  }
}

// what a captured step depends on besides its arguments: the I-ring order
// and the inputs' generation
void kbe::step_key(const kbe_handle *h, int *ring, unsigned *gen) {
  *ring = h->Ip == h->Ip0 ? 0 : 1;
  *gen = h->graph_gen;
}

kbe::StepMark kbe::step_mark(const kbe_handle *h) { return {h->n, h->Ip, h->Ic}; }

void kbe::step_rewind(kbe_handle *h, const kbe::StepMark &mk) {
  h->n = mk.n;
  h->Ip = (double2 *)mk.Ip;
  h->Ic = (double2 *)mk.Ic;
}

cudaStream_t kbe::handle_stream(const kbe_handle *h) { return h->stream; }
int kbe::handle_precision(const kbe_handle *h) { return h->cfg.precision; }

// device bytes of one handle (the allocations of kbe_create)
static size_t handle_bytes(const kbe_config *cfg) {
  const Mesh m{cfg->nb, cfg->L[0], cfg->L[1], cfg->L[0] * cfg->L[1]};
  const size_t T = (size_t)cfg->nt_max, nb2 = (size_t)cfg->nb * cfg->nb, blk = nb2 * m.nk;
  const size_t ntri = tri((int)T, (int)T) + 1, row = (T + 1) * 2 * blk * sizeof(double2);
  size_t b = kbe::history_bytes(m, cfg->precision, (int)T);
  (void)ntri;
  b += 2 * row;                                                   // FP64 working rows
  b += kbe::sweep_workspace_bytes(m, (int)T, cfg->precision);      // sweep coefficients, partials
  b += 3 * row;                                                   // I rows, Sigma row
  b += kbe::sigma_workspace_bytes(m, (int)T);                     // Sigma scratch
  b += 3 * blk * sizeof(double2);                                 // U, V, h
  b += (T + 2) * nb2 * sizeof(double2) + (T + 1) * (6 + (size_t)m.nk * cfg->nb) * sizeof(double);
  b += (T + 1) * sizeof(double) + 64;
  b += (T + 1) * sizeof(int) + 16;                                // corrector counts and flags
  b += 3 * (size_t)m.nk * sizeof(double) + sizeof(unsigned);       // observables partials, ticket
  return b;
}

extern "C" {

kbe_status kbe_create(const kbe_config *cfg, void *stream, kbe_handle **out) {
  if (!cfg || !out) return fail(nullptr, KBE_ERR_ARG, "kbe_create: null argument");
  *out = nullptr;
  if (!nb_ok(cfg->nb)) return fail(nullptr, KBE_ERR_UNSUPPORTED, "kbe_create: nb not in {1,2,3,4,6,8,12,16}");
  if (cfg->dim != 1 && cfg->dim != 2) return fail(nullptr, KBE_ERR_ARG, "kbe_create: dim must be 1 or 2");
  if (cfg->L[0] < 1 || cfg->L[1] < 1 || (cfg->dim == 1 && cfg->L[1] != 1))
    return fail(nullptr, KBE_ERR_ARG, "kbe_create: bad mesh extents");
  if ((long)cfg->L[0] * cfg->L[1] > kbe::kMaxNk) return fail(nullptr, KBE_ERR_ARG, "kbe_create: n_k > 4096");
  if (cfg->nt_max < 1 || cfg->nt_max > 65534) return fail(nullptr, KBE_ERR_ARG, "kbe_create: nt_max out of range");
  if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return fail(nullptr, KBE_ERR_ARG, "kbe_create: dt must be > 0");
  if (!std::isfinite(cfg->beta) || !std::isfinite(cfg->mu)) return fail(nullptr, KBE_ERR_ARG, "kbe_create: beta/mu not finite");
  if (!kbe::precision_supported(cfg->precision)) return fail(nullptr, KBE_ERR_UNSUPPORTED, "kbe_create: unknown precision");
  if (cfg->precision == KBE_PREC_F16X2 && cfg->nb != 4 && cfg->nb != 8)
    return fail(nullptr, KBE_ERR_UNSUPPORTED, "kbe_create: the split-FP16 (tensor-core) form needs nb 4 or 8");
  if (cfg->n_corr < 0 || cfg->n_corr > 64) return fail(nullptr, KBE_ERR_ARG, "kbe_create: n_corr out of range");
  if (!std::isfinite(cfg->corr_tol) || cfg->corr_tol < 0.0)
    return fail(nullptr, KBE_ERR_ARG, "kbe_create: corr_tol must be finite and >= 0");
  if (cfg->quadrature != KBE_QUAD_TRAPEZOID && cfg->quadrature != KBE_QUAD_GREGORY)
    return fail(nullptr, KBE_ERR_ARG, "kbe_create: unknown quadrature");

  kbe_handle *h = new kbe_handle();
  h->cfg = *cfg;
  h->mesh = Mesh{cfg->nb, cfg->L[0], cfg->L[1], cfg->L[0] * cfg->L[1]};
  h->stream = (cudaStream_t)stream;
  h->nb2 = cfg->nb * cfg->nb;
  h->blk = (size_t)h->nb2 * h->mesh.nk;
  h->v.assign((size_t)h->nb2, 0.0);
  for (int a = 0; a < cfg->nb; ++a)
    for (int b = 0; b < cfg->nb; ++b) h->v[(size_t)a * cfg->nb + b] = a == b ? 0.0 : 1.0;
  cudaGetDevice(&h->device);

  const size_t T = (size_t)cfg->nt_max;
  const size_t ntri = tri((int)T, (int)T) + 1;
  const size_t row = (T + 1) * 2 * h->blk;
  h->esz = kbe::history_elem_bytes(cfg->precision);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(h, (char **)&h->H, kbe::history_bytes(h->mesh, cfg->precision, (int)T));
  if (e == cudaSuccess) e = dalloc(h, &h->Wrow[0], row);
  if (e == cudaSuccess) e = dalloc(h, &h->Wrow[1], row);
  if (e == cudaSuccess) e = dalloc(h, (char **)&h->coef, kbe::sweep_workspace_bytes(h->mesh, (int)T, cfg->precision));
  if (e == cudaSuccess) e = dalloc(h, &h->Ip, row);
  if (e == cudaSuccess) e = dalloc(h, &h->Ic, row);
  if (e == cudaSuccess) e = dalloc(h, &h->Sig, row);
  if (e == cudaSuccess) e = dalloc(h, &h->work, kbe::sigma_workspace_bytes(h->mesh, (int)T) / sizeof(double2));
  if (e == cudaSuccess) e = dalloc(h, &h->U, h->blk);
  if (e == cudaSuccess) e = dalloc(h, &h->V, h->blk);
  if (e == cudaSuccess) e = dalloc(h, &h->hk, h->blk);
  if (e == cudaSuccess) e = dalloc(h, &h->rho, (T + 2) * h->nb2);
  if (e == cudaSuccess) e = dalloc(h, &h->obs, (T + 1) * 6);
  if (e == cudaSuccess) e = dalloc(h, &h->nkb, (T + 1) * h->mesh.nk * cfg->nb);
  if (e == cudaSuccess) e = dalloc(h, &h->status, 1);
  if (e == cudaSuccess) e = dalloc(h, &h->obs_part, 3 * (size_t)h->mesh.nk);
  if (e == cudaSuccess) e = dalloc(h, &h->obs_ticket, 1);
  if (e == cudaSuccess) e = dalloc(h, &h->d_U, T + 1);
  if (e == cudaSuccess) e = dalloc(h, &h->d_skip, 1);
  if (e == cudaSuccess) e = dalloc(h, &h->d_maxdiff, 1);
  if (e == cudaSuccess) e = dalloc(h, &h->d_iters, T + 1);
  if (e != cudaSuccess) {
    std::string msg = std::string("kbe_create: device allocation failed (") + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    free_all(h);
    delete h;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? KBE_ERR_OOM : KBE_ERR_CUDA, msg);
  }
  cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  cudaMemsetAsync(h->obs_ticket, 0, sizeof(unsigned), h->stream);
  cudaMemsetAsync(h->rho, 0, sizeof(double2) * (T + 2) * h->nb2, h->stream);
  cudaMemsetAsync(h->d_iters, 0, sizeof(int) * (T + 1), h->stream);
  h->Ip0 = h->Ip;
  h->Ic0 = h->Ic;
  *out = h;
  return KBE_OK;
}

kbe_status kbe_destroy(kbe_handle *h) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return KBE_OK;
}

kbe_status kbe_set_hamiltonian(kbe_handle *h, int nhop, const int *R, const double *t) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);   // captured kernels carry the old inputs
  if (nhop < 1 || nhop > 4096 || !R || !t) return fail(h, KBE_ERR_ARG, "set_hamiltonian: bad arguments");
  for (size_t i = 0; i < (size_t)nhop * h->nb2 * 2; ++i)
    if (!std::isfinite(t[i])) return fail(h, KBE_ERR_NONFINITE, "set_hamiltonian: non-finite hopping");
  h->hopR.assign(R, R + 2 * (size_t)nhop);
  if (h->cfg.dim == 1)
    for (int r = 0; r < nhop; ++r) h->hopR[2 * (size_t)r + 1] = 0;
  h->hopT.assign(t, t + (size_t)nhop * h->nb2 * 2);
  cudaStreamSynchronize(h->stream);
  if (h->d_hopR) cudaFree(h->d_hopR);
  if (h->d_hopT) cudaFree(h->d_hopT);
  h->d_hopR = nullptr;
  h->d_hopT = nullptr;
  cudaError_t e = cudaMalloc((void **)&h->d_hopR, sizeof(int) * 2 * nhop);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_hopT, sizeof(double2) * (size_t)nhop * h->nb2);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_hamiltonian alloc");
  e = cudaMemcpyAsync(h->d_hopR, h->hopR.data(), sizeof(int) * 2 * nhop, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_hopT, h->hopT.data(), sizeof(double2) * (size_t)nhop * h->nb2,
                        cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_hamiltonian copy");
  cudaStreamSynchronize(h->stream);
  h->nhop = nhop;
  h->ham_set = true;
  return KBE_OK;
}

kbe_status kbe_set_interaction(kbe_handle *h, int len, const double *U, const double *v) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);   // captured kernels carry the old inputs
  if (!U || (len != 1 && len < h->cfg.nt_max + 1))
    return fail(h, KBE_ERR_ARG, "set_interaction: need 1 or nt_max+1 samples of U");
  for (int i = 0; i < len; ++i)
    if (!std::isfinite(U[i])) return fail(h, KBE_ERR_NONFINITE, "set_interaction: non-finite U");
  if (v) {
    for (int i = 0; i < h->nb2; ++i)
      if (!std::isfinite(v[i])) return fail(h, KBE_ERR_NONFINITE, "set_interaction: non-finite v");
    const int nb = h->cfg.nb;
    for (int a = 0; a < nb; ++a)
      for (int b = a + 1; b < nb; ++b) {
        const double x = v[a * nb + b], y = v[b * nb + a];
        if (std::fabs(x - y) > 1e-12 * (std::fabs(x) + std::fabs(y)))
          return fail(h, KBE_ERR_ARG, "set_interaction: v must be symmetric (v_ab = v_ba)");
      }
    h->v.assign(v, v + h->nb2);
  }
  h->Useq.assign(U, U + (len == 1 ? 1 : h->cfg.nt_max + 1));
  std::vector<double> full((size_t)h->cfg.nt_max + 1);
  for (int i = 0; i <= h->cfg.nt_max; ++i) full[(size_t)i] = U_at(h, i);
  cudaError_t e = cudaMemcpyAsync(h->d_U, full.data(), sizeof(double) * full.size(),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_interaction copy");
  return KBE_OK;
}

kbe_status kbe_set_drive(kbe_handle *h, int len, const double *A, const double *dir) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);   // captured kernels carry the old inputs
  if (len < 0) return fail(h, KBE_ERR_ARG, "set_drive: negative length");
  if (A && len > 0) {
    for (int i = 0; i < len; ++i)
      if (!std::isfinite(A[i])) return fail(h, KBE_ERR_NONFINITE, "set_drive: non-finite A");
    h->A.assign(A, A + len);
  } else {
    h->A.clear();
  }
  if (dir) {
    if (!std::isfinite(dir[0]) || (h->cfg.dim == 2 && !std::isfinite(dir[1])))
      return fail(h, KBE_ERR_NONFINITE, "set_drive: non-finite direction");
    h->dir[0] = dir[0];
    h->dir[1] = h->cfg.dim == 2 ? dir[1] : 0.0;
  }
  return KBE_OK;
}

kbe_status kbe_set_dipole(kbe_handle *h, int len, const double *E, const double *M) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);   // captured kernels carry the old inputs
  if (len < 0 || (E && len > 0 && !M)) return fail(h, KBE_ERR_ARG, "set_dipole: bad arguments");
  if (!E || len == 0) {
    h->dipE.clear();
    return KBE_OK;
  }
  for (int i = 0; i < len; ++i)
    if (!std::isfinite(E[i])) return fail(h, KBE_ERR_NONFINITE, "set_dipole: non-finite field");
  for (int i = 0; i < 2 * h->nb2; ++i)
    if (!std::isfinite(M[i])) return fail(h, KBE_ERR_NONFINITE, "set_dipole: non-finite coupling");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && !h->d_dipM) e = cudaMalloc((void **)&h->d_dipM, sizeof(double2) * h->nb2);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_dipM, M, sizeof(double2) * h->nb2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_dipole");
  h->dipE.assign(E, E + len);
  return KBE_OK;
}

kbe_status kbe_reset(kbe_handle *h) {
  if (!h) return KBE_ERR_ARG;
  if (!h->ham_set) return fail(h, KBE_ERR_STATE, "reset: set_hamiltonian first");
  if (h->poisoned)
    return fail(h, KBE_ERR_STATE, "reset: an undrained copy timed out on this handle; destroy and recreate it");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "reset sync");
  h->sticky = KBE_OK;
  cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  cudaMemsetAsync(h->obs_ticket, 0, sizeof(unsigned), h->stream);
  h->Ip = h->Ip0;   // a fixed order, so that a replayed graph sees the pointers it captured
  h->Ic = h->Ic0;
  cudaMemsetAsync(h->Ip, 0, sizeof(double2) * 2 * h->blk, h->stream);
  cudaMemsetAsync(h->Ic, 0, sizeof(double2) * 2 * h->blk, h->stream);
  e = kbe::launch_init_state(h->mesh, hop_table(h), h->cfg.beta, h->cfg.mu, frow(h, 0), h->status, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "init_state");
  if (h->prof) h->stats.launches += 1;
  h->n = 0;
  kbe_status ps = publish(h, 0);
  if (ps != KBE_OK) return ps;
  kbe_status s = density(h, 0, h->rho);
  if (s != KBE_OK) return s;
  s = observables(h, 0, h->Ip);
  if (s != KBE_OK) return s;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "reset");
  return KBE_OK;
}

kbe_status kbe_step(kbe_handle *h, int nsteps) {
  if (!h) return KBE_ERR_ARG;
  if (h->sticky != KBE_OK) return fail(h, h->sticky, "step: handle has a sticky error; reset it");
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "step: call kbe_reset first");
  if (nsteps < 0) return fail(h, KBE_ERR_ARG, "step: negative count");
  if (h->n + nsteps > h->cfg.nt_max) return fail(h, KBE_ERR_STATE, "step: past nt_max");
  if (h->graphs && !h->prof && !h->inject && h->stream != nullptr && nsteps > 0) return step_graph(h, nsteps);
  for (int i = 0; i < nsteps; ++i) {
    kbe_status s = one_step(h);
    if (s != KBE_OK) return s;
  }
  return KBE_OK;
}

kbe_status kbe_autotune(kbe_handle *h, int *targets) {
  if (!h) return KBE_ERR_ARG;
  if (h->sticky != KBE_OK) return fail(h, h->sticky, "autotune: handle has a sticky error; reset it");
  int out[KBE_AUTOTUNE_BUCKETS];
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess)
    e = kbe::tune_sweep(h->mesh, h->cfg.precision, h->cfg.quadrature, h->cfg.nt_max, h->cfg.dt, h->H, h->Sig, h->Ic,
                        h->coef, h->stream, out, KBE_AUTOTUNE_BUCKETS, h->cfg.nt_max + 1);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  drop_graphs(h);   // captured sweeps carry the old splits
  if (targets)
    for (int b = 0; b < KBE_AUTOTUNE_BUCKETS; ++b) targets[b] = out[b];
  return KBE_OK;
}

kbe_status kbe_debug_inject(kbe_handle *h, int fault) {
  if (!h) return KBE_ERR_ARG;
  if (fault != 0 && fault != KBE_INJECT_STAGED_COPY_LOSS) return fail(h, KBE_ERR_ARG, "debug_inject: unknown fault");
  if (fault == KBE_INJECT_STAGED_COPY_LOSS &&
      !(h->cfg.precision == KBE_PREC_C64 && h->cfg.nb >= 4 && h->mesh.nk % 2 == 0 && h->cfg.nb != 6 && h->cfg.nb != 12))
    return fail(h, KBE_ERR_UNSUPPORTED, "debug_inject: the handle's sweep is not the staged C64 form");
  h->inject = fault;
  return KBE_OK;
}

kbe_status kbe_set_graphs(kbe_handle *h, int enable) {
  if (!h) return KBE_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_graphs");
  drop_graphs(h);
  h->graphs = enable != 0;
  return KBE_OK;
}

kbe_status kbe_synchronize(kbe_handle *h) {
  if (!h) return KBE_ERR_ARG;
  return check_device_status(h);
}

kbe_status kbe_current_step(const kbe_handle *h, int *n) {
  if (!h || !n) return KBE_ERR_ARG;
  *n = h->n;
  return KBE_OK;
}

kbe_status kbe_observables(kbe_handle *h, int step, double *n_kb, double *scalars) {
  if (!h) return KBE_ERR_ARG;
  if (step < 0 || step > h->n) return fail(h, KBE_ERR_ARG, "observables: step out of range");
  kbe_status s = check_device_status(h);
  if (s != KBE_OK) return s;
  cudaError_t e = cudaSuccess;
  if (n_kb)
    e = cudaMemcpy(n_kb, h->nkb + (size_t)step * h->mesh.nk * h->cfg.nb,
                   sizeof(double) * h->mesh.nk * h->cfg.nb, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && scalars)
    e = cudaMemcpy(scalars, h->obs + (size_t)step * 6, sizeof(double) * 6, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "observables copy");
  return KBE_OK;
}

kbe_status kbe_observables_all(kbe_handle *h, double *n_kb, double *scalars) {
  if (!h) return KBE_ERR_ARG;
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "observables_all: call kbe_reset first");
  kbe_status s = check_device_status(h);
  if (s != KBE_OK) return s;
  const size_t rows = (size_t)h->n + 1;
  cudaError_t e = cudaSuccess;
  if (n_kb)
    e = cudaMemcpyAsync(n_kb, h->nkb, sizeof(double) * rows * h->mesh.nk * h->cfg.nb,
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && scalars)
    e = cudaMemcpyAsync(scalars, h->obs, sizeof(double) * rows * 6, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "observables_all copy");
  return KBE_OK;
}

kbe_status kbe_observables_all_dev(kbe_handle *h, double *n_kb_dev, double *scalars_dev) {
  if (!h) return KBE_ERR_ARG;
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "observables_all_dev: call kbe_reset first");
  const size_t rows = (size_t)h->n + 1;
  cudaError_t e = cudaSuccess;
  if (n_kb_dev)
    e = cudaMemcpyAsync(n_kb_dev, h->nkb, sizeof(double) * rows * h->mesh.nk * h->cfg.nb,
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && scalars_dev)
    e = cudaMemcpyAsync(scalars_dev, h->obs, sizeof(double) * rows * 6, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "observables_all_dev copy");
  return KBE_OK;
}

kbe_status kbe_get_row_dev(kbe_handle *h, int i, int which, void *out_dev) {
  if (!h || !out_dev) return KBE_ERR_ARG;
  if (i < 0 || i > h->n || (which != 0 && which != 1)) return fail(h, KBE_ERR_ARG, "get_row_dev: bad row or component");
  const bool fp64_copy = i >= h->n - 1;   // the two newest rows are kept in FP64
  cudaError_t e = kbe::launch_row_out(h->cfg.precision, fp64_copy ? frow(h, i) : nullptr,
                                      (const char *)h->H + kbe::history_row_offset(h->mesh, h->cfg.precision, i),
                                      (size_t)i + 1, h->mesh, which, (double2 *)out_dev, h->stream, i,
                                      h->cfg.nt_max + 1);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_row_dev");
  return KBE_OK;
}

kbe_status kbe_get_row(kbe_handle *h, int i, int which, double *out) {
  if (!h || !out) return KBE_ERR_ARG;
  if (i < 0 || i > h->n || (which != 0 && which != 1)) return fail(h, KBE_ERR_ARG, "get_row: bad row or component");
  kbe_status s = check_device_status(h);
  if (s != KBE_OK && s != KBE_ERR_NONFINITE) return s;
  const size_t nblk = (size_t)i + 1;
  const size_t cnt = nblk * 2 * h->blk;
  if (h->cfg.precision == KBE_PREC_F16X2 && i < h->n - 1) {
    // the split-FP16 storage spreads the row over its strips: decode it on the
    // device into the Sigma row buffer (a whole row of complex128, rewritten by
    // the next step before use), then copy it out
    cudaError_t e = kbe::launch_row_out(h->cfg.precision, nullptr, h->H, nblk, h->mesh, which, h->Sig, h->stream, i,
                                        h->cfg.nt_max + 1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, h->Sig, sizeof(double2) * nblk * h->blk, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_row decode");
    return KBE_OK;
  }
  std::vector<double2> tmp(cnt);
  cudaError_t e;
  if (i >= h->n - 1) {                                        // an FP64 copy exists
    e = cudaMemcpyAsync(tmp.data(), frow(h, i), sizeof(double2) * cnt, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  } else {                                                    // unpack the stored row
    const size_t off = kbe::history_row_offset(h->mesh, h->cfg.precision, i);
    std::vector<char> raw(kbe::history_row_offset(h->mesh, h->cfg.precision, i + 1) - off);
    e = cudaMemcpyAsync(raw.data(), (char *)h->H + off, raw.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) {
      const float *f = (const float *)raw.data();
      const double2 *d = (const double2 *)raw.data();
      for (size_t q = 0; q < cnt; ++q) {
        if (h->cfg.precision == KBE_PREC_DF64)
          tmp[q] = make_double2((double)f[4 * q] + (double)f[4 * q + 1], (double)f[4 * q + 2] + (double)f[4 * q + 3]);
        else if (h->cfg.precision == KBE_PREC_C64)
          tmp[q] = make_double2((double)f[2 * q], (double)f[2 * q + 1]);
        else
          tmp[q] = d[q];
      }
      for (size_t bq = 0; bq < nblk; ++bq)   // (G^<, dG) -> (G^<, G^> = G^< - dG)
        for (size_t r = 0; r < h->blk; ++r) {
          const double2 gl = tmp[(bq * 2) * h->blk + r], dg = tmp[(bq * 2 + 1) * h->blk + r];
          tmp[(bq * 2 + 1) * h->blk + r] = make_double2(gl.x - dg.x, gl.y - dg.y);
        }
    }
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "get_row copy");
  const int nb = h->cfg.nb, nk = h->mesh.nk;
  double2 *o = (double2 *)out;
  for (size_t j = 0; j < nblk; ++j) {
    const double2 *src = tmp.data() + (j * 2 + which) * h->blk;
    for (int k = 0; k < nk; ++k)
      for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b)
          o[((j * nk + k) * nb + a) * nb + b] = src[((size_t)a * nb + b) * nk + k];
  }
  return KBE_OK;
}

kbe_status kbe_corrector_iterations(kbe_handle *h, int *out) {
  if (!h || !out) return KBE_ERR_ARG;
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "corrector_iterations: call kbe_reset first");
  const size_t rows = (size_t)h->n + 1;
  if (h->cfg.corr_tol > 0.0) {
    cudaError_t e = cudaMemcpyAsync(out, h->d_iters, sizeof(int) * rows, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "corrector_iterations copy");
  } else {
    for (size_t i = 0; i < rows; ++i) out[i] = i == 0 ? 0 : h->cfg.n_corr;
  }
  out[0] = 0;
  return KBE_OK;
}

kbe_status kbe_profile_enable(kbe_handle *h, int enable) {
  if (!h) return KBE_ERR_ARG;
  cudaStreamSynchronize(h->stream);   // (profiled steps run without graphs)
  h->prof = enable != 0;
  h->ev_used = 0;
  h->bev_used = 0;
  h->stats = kbe_profile_stats{};
  return KBE_OK;
}

kbe_status kbe_profile_read(kbe_handle *h, kbe_profile_stats *out) {
  if (!h || !out) return KBE_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile sync");
  kbe_profile_stats s = h->stats;
  s.sweep_launches = 0;
  s.sweep_ms = s.sweep_flops = s.sweep_flops_executed = s.sweep_bytes = 0.0;
  for (size_t i = 0; i < h->ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[i].first, h->ev[i].second) == cudaSuccess) {
      s.sweep_ms += ms;
      s.sweep_flops += h->ev_flops[i];
      s.sweep_flops_executed += h->ev_flops_x[i];
      s.sweep_bytes += h->ev_bytes[i];
      s.sweep_launches++;
    }
  }
  for (int q = 0; q < 4; ++q) s.backward_ms[q] = 0.0;
  s.backward_sweep_flops = 0.0;
  for (size_t i = 0; i < h->bev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->bev[i].a, h->bev[i].b) == cudaSuccess) {
      s.backward_ms[h->bev[i].phase] += ms;
      s.backward_sweep_flops += h->bev[i].flops;
    }
  }
  *out = s;
  return KBE_OK;
}

// ---- checkpoint / resume --------------------------------------------------

namespace {
struct CkptHeader {
  char magic[8];
  int version, nb, dim, L0, L1, nt_max, precision, n;
};

// the device regions of the state after row n, in file order
struct Region {
  const void *dev;
  void *dev_w;
  size_t bytes;
};

std::vector<Region> state_regions(kbe_handle *h) {
  const int n = h->n;
  const size_t row = (size_t)(n + 1) * 2 * h->blk * sizeof(double2);
  std::vector<Region> r;
  // (the split-FP16 storage spreads every row over its strips: all of it)
  r.push_back({h->H, h->H, kbe::history_bytes(h->mesh, h->cfg.precision,
                                              h->cfg.precision == KBE_PREC_F16X2 ? h->cfg.nt_max : n)});
  r.push_back({frow(h, n), frow(h, n), row});
  if (n >= 1) r.push_back({frow(h, n - 1), frow(h, n - 1), (size_t)n * 2 * h->blk * sizeof(double2)});
  r.push_back({h->Ip, h->Ip, row});
  r.push_back({h->rho, h->rho, (size_t)(n + 1) * h->nb2 * sizeof(double2)});
  r.push_back({h->obs, h->obs, (size_t)(n + 1) * 6 * sizeof(double)});
  r.push_back({h->nkb, h->nkb, (size_t)(n + 1) * h->mesh.nk * h->cfg.nb * sizeof(double)});
  r.push_back({h->d_iters, h->d_iters, (size_t)(n + 1) * sizeof(int)});
  return r;
}
}  // namespace

size_t kbe_checkpoint_bytes(const kbe_handle *h) {
  if (!h || h->n < 0) return 0;
  size_t b = sizeof(CkptHeader);
  for (const Region &r : state_regions(const_cast<kbe_handle *>(h))) b += r.bytes;
  return b;
}

kbe_status kbe_checkpoint_save(kbe_handle *h, void *host, size_t bytes) {
  if (!h || !host) return KBE_ERR_ARG;
  if (h->n < 0) return fail(h, KBE_ERR_STATE, "checkpoint_save: nothing to save before kbe_reset");
  if (bytes < kbe_checkpoint_bytes(h)) return fail(h, KBE_ERR_ARG, "checkpoint_save: buffer too small");
  kbe_status st = check_device_status(h);
  if (st != KBE_OK) return st;
  CkptHeader hd{};
  memcpy(hd.magic, "KBECKPT", 8);
  hd.version = 2;
  hd.nb = h->cfg.nb;
  hd.dim = h->cfg.dim;
  hd.L0 = h->cfg.L[0];
  hd.L1 = h->cfg.L[1];
  hd.nt_max = h->cfg.nt_max;
  hd.precision = h->cfg.precision;
  hd.n = h->n;
  char *p = (char *)host;
  memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  for (const Region &r : state_regions(h)) {
    cudaError_t e = cudaMemcpyAsync(p, r.dev, r.bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint_save");
    p += r.bytes;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint_save");
  return KBE_OK;
}

kbe_status kbe_checkpoint_load(kbe_handle *h, const void *host, size_t bytes) {
  if (!h || !host || bytes < sizeof(CkptHeader)) return KBE_ERR_ARG;
  if (h->poisoned)
    return fail(h, KBE_ERR_STATE, "checkpoint_load: an undrained copy timed out on this handle; recreate it");
  CkptHeader hd;
  memcpy(&hd, host, sizeof hd);
  if (memcmp(hd.magic, "KBECKPT", 8) != 0 || hd.version != 2 || hd.nb != h->cfg.nb ||
      hd.dim != h->cfg.dim || hd.L0 != h->cfg.L[0] || hd.L1 != h->cfg.L[1] ||
      hd.nt_max != h->cfg.nt_max || hd.precision != h->cfg.precision || hd.n < 0 || hd.n > h->cfg.nt_max)
    return fail(h, KBE_ERR_ARG, "checkpoint_load: checkpoint does not match this handle's configuration");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint_load");
  const int keep = h->n;
  h->n = hd.n;
  size_t need = sizeof hd;
  for (const Region &r : state_regions(h)) need += r.bytes;
  if (bytes < need) {
    h->n = keep;
    return fail(h, KBE_ERR_ARG, "checkpoint_load: buffer too small");
  }
  const char *p = (const char *)host + sizeof hd;
  for (const Region &r : state_regions(h)) {
    e = cudaMemcpyAsync(r.dev_w, p, r.bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint_load");
    p += r.bytes;
  }
  cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint_load");
  h->sticky = KBE_OK;
  return KBE_OK;
}

size_t kbe_memory_bytes(const kbe_config *cfg) {
  if (!cfg || !nb_ok(cfg->nb) || cfg->L[0] < 1 || cfg->L[1] < 1 || cfg->nt_max < 1 ||
      (long)cfg->L[0] * cfg->L[1] > kbe::kMaxNk || !kbe::precision_supported(cfg->precision))
    return 0;
  return handle_bytes(cfg);
}

// ---- reverse mode ----------------------------------------------------------

size_t kbe_backward_memory_bytes(const kbe_config *cfg) {
  if (!cfg || !nb_ok(cfg->nb) || cfg->L[0] < 1 || cfg->L[1] < 1 || cfg->nt_max < 1 ||
      (long)cfg->L[0] * cfg->L[1] > kbe::kMaxNk || cfg->n_corr < 0 || cfg->n_corr > 64)
    return 0;
  AdjPtrs p{};
  const Mesh m{cfg->nb, cfg->L[0], cfg->L[1], cfg->L[0] * cfg->L[1]};
  return adj_carve(cfg, m, nullptr, &p);
}

kbe_status kbe_backward(kbe_handle *h, const double *dL_dn, double *dL_dA, double *dL_dU) {
  if (!h) return KBE_ERR_ARG;
  if (!dL_dn || !dL_dA || !dL_dU) return fail(h, KBE_ERR_ARG, "backward: null argument");
  if (h->sticky != KBE_OK) return fail(h, h->sticky, "backward: handle has a sticky error; reset it");
  if (h->n < 1) return fail(h, KBE_ERR_STATE, "backward: no step to differentiate (call kbe_step first)");
  if (h->cfg.precision != KBE_PREC_FP64)
    return fail(h, KBE_ERR_UNSUPPORTED, "backward: needs the FP64 history (KBE_PREC_FP64)");
  const int nk = h->mesh.nk, nb = h->cfg.nb;
  for (int i = 0; i < nk * nb; ++i)
    if (!std::isfinite(dL_dn[i])) return fail(h, KBE_ERR_NONFINITE, "backward: non-finite dL/dn");
  kbe_status s = check_device_status(h);
  if (s != KBE_OK) return s;
  AdjPtrs P{};
  if (!h->adj) {
    const size_t bytes = adj_carve(&h->cfg, h->mesh, nullptr, &P);
    cudaError_t e = cudaMalloc(&h->adj, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->adj = nullptr;
      return fail(h, e == cudaErrorMemoryAllocation ? KBE_ERR_OOM : KBE_ERR_CUDA,
                  std::string("backward: device allocation failed (") + cudaGetErrorString(e) + ")");
    }
    h->adj_bytes = bytes;
  }
  adj_carve(&h->cfg, h->mesh, (char *)h->adj, &P);
  const int N = h->n;
  const size_t blk = h->blk, nb2 = (size_t)h->nb2;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemsetAsync(P.lamH, 0, (tri(N, N) + 1) * 2 * blk * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.lamRho, 0, (size_t)(N + 1) * nb2 * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.gA, 0, (size_t)h->cfg.nt_max * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.gU, 0, (size_t)(h->cfg.nt_max + 1) * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.lamIa, 0, (size_t)(N + 1) * 2 * blk * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.lamIb, 0, (size_t)(N + 1) * 2 * blk * sizeof(double2), st);
  // n_kb = Im G^<_bb(k; N, N): dL = Re conj(i g) dG^<_bb for g = dL/dn_kb
  std::vector<double2> seed(blk, make_double2(0.0, 0.0));
  for (int k = 0; k < nk; ++k)
    for (int b = 0; b < nb; ++b) seed[(size_t)(b * nb + b) * nk + k] = make_double2(0.0, dL_dn[(size_t)k * nb + b]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P.lamH + tri(N, N) * 2 * blk, seed.data(), blk * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "backward setup");
  std::vector<int> iters((size_t)N + 1, h->cfg.n_corr);
  if (h->cfg.corr_tol > 0.0) {   // replay the passes each step ran
    e = cudaMemcpyAsync(iters.data(), h->d_iters, sizeof(int) * iters.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "backward corrector counts");
  }
  double2 *lamIcur = P.lamIa, *lamIprev = P.lamIb;
  for (int n = N; n >= 1; --n) {
    s = backward_step(h, P, n, iters[(size_t)n], lamIcur, lamIprev);
    if (s != KBE_OK) return s;
    std::swap(lamIcur, lamIprev);
    e = cudaMemsetAsync(lamIprev, 0, (size_t)n * 2 * blk * sizeof(double2), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "backward memset");
  }
  std::vector<double> gA((size_t)N), gUs((size_t)h->cfg.nt_max + 1);
  int stat = 0;
  e = cudaMemcpyAsync(gA.data(), P.gA, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(gUs.data(), P.gU, sizeof(double) * gUs.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&stat, h->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "backward result copy");
  if (stat & kbe::kDevAdjUnsupported) {   // the forward state is intact: clear the flag, keep the handle usable
    const int keep = stat & ~kbe::kDevAdjUnsupported;
    e = cudaMemcpyAsync(h->status, &keep, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "backward status");
    return fail(h, KBE_ERR_UNSUPPORTED,
                "backward: a step needed the scaled-and-squared propagators (dt ||h|| > 1/4), which have no adjoint");
  }
  s = check_device_status(h);
  if (s != KBE_OK) return s;
  for (int i = 0; i < h->cfg.nt_max; ++i) dL_dA[i] = i < N ? gA[(size_t)i] : 0.0;
  if (h->Useq.size() == 1) {   // one parameter: the sum over the samples it stands for
    double t = 0.0;
    for (double x : gUs) t += x;
    dL_dU[0] = t;
  } else {
    for (size_t i = 0; i < gUs.size(); ++i) dL_dU[i] = gUs[i];
  }
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(gA[(size_t)i])) return fail(h, KBE_ERR_NONFINITE, "backward: non-finite gradient");
  for (double x : gUs)
    if (!std::isfinite(x)) return fail(h, KBE_ERR_NONFINITE, "backward: non-finite gradient");
  return KBE_OK;
}

const char *kbe_last_error(const kbe_handle *h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

// ---- stateless operations ------------------------------------------------

size_t kbe_op_sigma_row_workspace(const kbe_mesh *m, int n) {
  if (!mesh_ok(m) || n < 0) return 0;
  return kbe::sigma_workspace_bytes(to_mesh(m), n);
}

kbe_status kbe_op_sigma_row(const kbe_mesh *m, const double *v, int n, double Un,
                            const double *Ul_dev, const void *Grow_dev, void *Sigma_dev,
                            void *work_dev, size_t work_bytes, void *stream) {
  if (!mesh_ok(m) || !v || n < 0 || !Grow_dev || !Sigma_dev || !work_dev)
    return fail(nullptr, KBE_ERR_ARG, "op_sigma_row: bad arguments");
  const Mesh mm = to_mesh(m);
  if (work_bytes < kbe::sigma_workspace_bytes(mm, n))
    return fail(nullptr, KBE_ERR_ARG, "op_sigma_row: workspace too small");
  cudaError_t e = kbe::sigma_row(mm, v, n, Un, Ul_dev, (const double2 *)Grow_dev, (double2 *)Sigma_dev,
                                 (double2 *)work_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_sigma_row: ") + cudaGetErrorString(e));
  return KBE_OK;
}

size_t kbe_op_collision_row_workspace(const kbe_mesh *m, int n, int precision) {
  if (!mesh_ok(m) || n < 0 || !kbe::precision_supported(precision)) return 0;
  return kbe::sweep_workspace_bytes(to_mesh(m), n, precision);
}

kbe_status kbe_op_pack(int precision, const void *src_dev, void *dst_dev, size_t nblocks,
                       size_t block_elems, void *stream) {
  if (!kbe::precision_supported(precision) || (nblocks && block_elems && (!src_dev || !dst_dev)))
    return fail(nullptr, KBE_ERR_ARG, "op_pack: bad arguments");
  if (precision == KBE_PREC_F16X2)
    return fail(nullptr, KBE_ERR_UNSUPPORTED, "op_pack: the split-FP16 layout needs the mesh (kbe_op_pack_mesh)");
  cudaError_t e = kbe::launch_pack(precision, (const double2 *)src_dev, dst_dev, nblocks, block_elems,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_pack: ") + cudaGetErrorString(e));
  return KBE_OK;
}

size_t kbe_history_bytes(const kbe_mesh *m, int n, int precision) {
  if (!mesh_ok(m) || n < 0 || !kbe::precision_supported(precision)) return 0;
  if (precision == KBE_PREC_F16X2 && m->nb != 4 && m->nb != 8) return 0;
  return kbe::history_bytes(to_mesh(m), precision, n);
}

kbe_status kbe_op_pack_mesh(const kbe_mesh *m, int precision, const void *src_dev, void *dst_dev,
                            size_t nblocks, void *stream) {
  if (!mesh_ok(m) || !kbe::precision_supported(precision) || (nblocks && (!src_dev || !dst_dev)))
    return fail(nullptr, KBE_ERR_ARG, "op_pack_mesh: bad arguments");
  const kbe::Mesh mm = to_mesh(m);
  int cap = 0;   // the F16X2 layout holds rows 0 .. cap - 1: nblocks must be a triangle
  while ((size_t)cap * (cap + 1) / 2 < nblocks) ++cap;
  if (precision == KBE_PREC_F16X2 && (size_t)cap * (cap + 1) / 2 != nblocks)
    return fail(nullptr, KBE_ERR_ARG, "op_pack_mesh: F16X2 needs a whole triangle, nblocks = (n+1)(n+2)/2");
  cudaError_t e = kbe::launch_pack(precision, (const double2 *)src_dev, dst_dev, nblocks,
                                   (size_t)mm.nb * mm.nb * mm.nk, (cudaStream_t)stream, nullptr, mm.nb, -1, cap);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_pack_mesh: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_op_collision_row(const kbe_mesh *m, int n, double dt, int precision,
                                const void *H_dev, const void *Sigma_dev, void *I_dev,
                                void *work_dev, size_t work_bytes, void *stream) {
  if (!mesh_ok(m) || n < 0 || !H_dev || !Sigma_dev || !I_dev || !(dt > 0.0))
    return fail(nullptr, KBE_ERR_ARG, "op_collision_row: bad arguments");
  if (!kbe::precision_supported(precision)) return fail(nullptr, KBE_ERR_UNSUPPORTED, "op_collision_row: precision");
  const size_t need = kbe::sweep_workspace_bytes(to_mesh(m), n, precision);
  if (!work_dev || work_bytes < need)
    return fail(nullptr, KBE_ERR_ARG, "op_collision_row: workspace too small");
  cudaError_t e = kbe::launch_sweep(to_mesh(m), n, dt, precision, H_dev, (const double2 *)Sigma_dev,
                                    (double2 *)I_dev, work_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_collision_row: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_op_collision_row_quad(const kbe_mesh *m, int n, double dt, int precision, int quadrature,
                                     const void *H_dev, const void *Sigma_dev, void *I_dev,
                                     void *work_dev, size_t work_bytes, void *stream) {
  if (!mesh_ok(m) || n < 0 || !H_dev || !Sigma_dev || !I_dev || !(dt > 0.0) ||
      (quadrature != KBE_QUAD_TRAPEZOID && quadrature != KBE_QUAD_GREGORY))
    return fail(nullptr, KBE_ERR_ARG, "op_collision_row: bad arguments");
  if (!kbe::precision_supported(precision)) return fail(nullptr, KBE_ERR_UNSUPPORTED, "op_collision_row: precision");
  const size_t need = kbe::sweep_workspace_bytes(to_mesh(m), n, precision);
  if (!work_dev || work_bytes < need)
    return fail(nullptr, KBE_ERR_ARG, "op_collision_row: workspace too small");
  cudaError_t e = kbe::launch_sweep(to_mesh(m), n, dt, precision, H_dev, (const double2 *)Sigma_dev,
                                    (double2 *)I_dev, work_dev, (cudaStream_t)stream, nullptr, quadrature);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_collision_row: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_op_propagators(const kbe_mesh *m, double dt, const void *h_dev, void *U_dev,
                              void *V_dev, void *stream) {
  if (!mesh_ok(m) || !h_dev || !U_dev || !V_dev || !(dt > 0.0) || !std::isfinite(dt))
    return fail(nullptr, KBE_ERR_ARG, "op_propagators: bad arguments");
  kbe::HopTable hop{};
  kbe::PropParams p{};
  cudaError_t e = kbe::launch_build_props(to_mesh(m), hop, p, dt, (const double2 *)h_dev, nullptr,
                                          (double2 *)U_dev, (double2 *)V_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_propagators: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_op_update_row(const kbe_mesh *m, int n, double dt, double theta, const void *h_dev,
                             const void *U_dev, const void *V_dev, const void *Gprev_dev,
                             const void *Iprev_dev, const void *Icur_dev, void *out_dev, void *stream) {
  if (!mesh_ok(m) || n < 1 || !h_dev || !U_dev || !V_dev || !Gprev_dev || !Iprev_dev || !out_dev ||
      !(dt > 0.0) || !std::isfinite(dt) || (theta != 0.0 && !Icur_dev))
    return fail(nullptr, KBE_ERR_ARG, "op_update_row: bad arguments");
  cudaError_t e = kbe::launch_update_row(to_mesh(m), n, dt, theta, (const double2 *)h_dev,
                                         (const double2 *)U_dev, (const double2 *)V_dev,
                                         (const double2 *)Gprev_dev, (const double2 *)Iprev_dev,
                                         (const double2 *)Icur_dev, (double2 *)out_dev,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, KBE_ERR_CUDA, std::string("op_update_row: ") + cudaGetErrorString(e));
  return KBE_OK;
}

kbe_status kbe_set_sweep_choice(const kbe_mesh *m, int precision, int quadrature, int bucket, int choice) {
  if (!mesh_ok(m) || !kbe::precision_supported(precision) ||
      (quadrature != KBE_QUAD_TRAPEZOID && quadrature != KBE_QUAD_GREGORY))
    return fail(nullptr, KBE_ERR_ARG, "set_sweep_choice: bad mesh, precision or quadrature");
  if (!kbe::set_sweep_choice(to_mesh(m), precision, quadrature, bucket, choice))
    return fail(nullptr, KBE_ERR_ARG, "set_sweep_choice: choice or bucket out of range for this shape");
  return KBE_OK;
}

}  // extern "C"
