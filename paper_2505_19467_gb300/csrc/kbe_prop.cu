// (a3) mean-field Hamiltonian and step propagators, (a4) row / diagonal
// update, (a5) equal-time observables, and the t = 0 state.
//
// All of these are O(n_k N_b^3) or O(n n_k N_b^3) per call, small next to the
// collision sweep; they run in FP64.
//
// Time stepping (Algorithm 1, "solve Eq. 5"): with h fixed over the step and
// the collision term replaced by a constant average Ibar, the row equation
// i dG(t, t_j)/dt = h G + Ibar has the exact one-step solution
//   G(n, j) = U G(n-1, j) + V Ibar(j),  U = e^{-i dt h},  V = (U - 1) h^{-1},
// and the time diagonal i dG(t,t)/dt = [h, G] + Sbar, Sbar = Ibar + Ibar^+,
//   G(n, n) = U G(n-1, n-1) U^+ - i X,  X = int_0^dt e^{-i h u} Sbar e^{i h u} du.
// The matrix functions are evaluated per k by one CTA group of N_b^2 threads
// (one per matrix element), as power series in tau = dt / 2^s with
// tau ||h|| <= 1/4, followed by s doublings:
//   U_tau = sum_m (-i tau h)^m / m!,          U_2tau = U_tau^2,
//   V_tau = -i tau sum_m (-i tau h)^m/(m+1)!,  V_2tau = (U_tau + 1) V_tau,
//   X_tau = tau sum_m (-i tau)^m ad_h^m(S) / (m+1)!, X_2tau = X_tau + U_tau X_tau U_tau^+,
// with ad_h(S) = h S - S h; each series stops before its first term whose
// bound (nu^m / m!, (2 nu)^m / (m+1)!, nu = tau ||h||) is below 2^-60: at most
// 13 and 15 terms at nu = 1/4, fewer at smaller nu. The trace of X is dt Tr S exactly in
// exact arithmetic, so the particle number is conserved. A Jacobi
// eigen-solver is used only for the Fermi function of the initial state.
#include "kbe_internal.cuh"
#include "kbe_matgroup.cuh"

namespace kbe {

namespace {

// Hermitian eigen-decomposition A = W diag(lam) W^+ by cyclic complex Jacobi
// rotations (phase of A_pq removed, then the real rotation with the smaller
// root t of t^2 + 2 tau t - 1 = 0, tau = (A_qq - A_pp) / 2|A_pq|).
// A is overwritten. Returns false if 60 sweeps did not converge.
template <int NB>
__device__ bool herm_eig(double2 *A, double *lam, double2 *W) {
#pragma unroll 1
  for (int i = 0; i < NB * NB; ++i) W[i] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int i = 0; i < NB; ++i) {
    W[i * NB + i] = make_double2(1.0, 0.0);
    A[i * NB + i].y = 0.0;
  }
  bool conv = false;
#pragma unroll 1
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
#pragma unroll 1
    for (int p = 0; p < NB; ++p)
#pragma unroll 1
      for (int q = 0; q < NB; ++q) {
        const double2 z = A[p * NB + q];
        const double m2 = z.x * z.x + z.y * z.y;
        tot += m2;
        if (p != q) off += m2;
      }
    if (off == 0.0 || off <= 1e-34 * tot) {
      conv = true;
      break;
    }
#pragma unroll 1
    for (int p = 0; p < NB - 1; ++p)
#pragma unroll 1
      for (int q = p + 1; q < NB; ++q) {
        const double2 apq = A[p * NB + q];
        const double r = hypot(apq.x, apq.y);
        if (r == 0.0) continue;
        const double2 e = make_double2(apq.x / r, apq.y / r);   // e^{i phi}
        const double2 ec = c_conj(e);
        const double tau = (A[q * NB + q].x - A[p * NB + p].x) / (2.0 * r);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
#pragma unroll 1
        for (int i = 0; i < NB; ++i) {   // A <- A J ; W <- W J
          const double2 x = A[i * NB + p], y = A[i * NB + q];
          A[i * NB + p] = c_sub(c_scale(c, x), c_scale(s, c_mul(ec, y)));
          A[i * NB + q] = c_add(c_scale(s, x), c_scale(c, c_mul(ec, y)));
          const double2 wx = W[i * NB + p], wy = W[i * NB + q];
          W[i * NB + p] = c_sub(c_scale(c, wx), c_scale(s, c_mul(ec, wy)));
          W[i * NB + q] = c_add(c_scale(s, wx), c_scale(c, c_mul(ec, wy)));
        }
#pragma unroll 1
        for (int jj = 0; jj < NB; ++jj) {   // A <- J^+ A
          const double2 x = A[p * NB + jj], y = A[q * NB + jj];
          A[p * NB + jj] = c_sub(c_scale(c, x), c_scale(s, c_mul(e, y)));
          A[q * NB + jj] = c_add(c_scale(s, x), c_scale(c, c_mul(e, y)));
        }
        A[p * NB + q] = make_double2(0.0, 0.0);
        A[q * NB + p] = make_double2(0.0, 0.0);
        A[p * NB + p].y = 0.0;
        A[q * NB + q].y = 0.0;
      }
  }
#pragma unroll 1
  for (int i = 0; i < NB; ++i) lam[i] = A[i * NB + i].x;
  return conv;
}

// h0_ab(k - A d) = sum_r t_ab(R_r) exp(i (k - A d).R_r)
template <int NB>
__device__ void bare_h(const HopTable &hop, int k, int L0, int L1, double A, double2 *h) {
  const int k0 = k / L1, k1 = k - (k / L1) * L1;
#pragma unroll 1
  for (int i = 0; i < NB * NB; ++i) h[i] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int r = 0; r < hop.nhop; ++r) {
    const int R0 = hop.R[2 * r], R1 = hop.R[2 * r + 1];
    // reduce the lattice phase exactly before converting to an angle
    const int m0 = ((k0 * R0) % L0 + L0) % L0, m1 = ((k1 * R1) % L1 + L1) % L1;
    const double th = 2.0 * M_PI * ((double)m0 / L0 + (double)m1 / L1) - A * (hop.d0 * R0 + hop.d1 * R1);
    double s, c;
    sincos(th, &s, &c);
    const double2 ph = make_double2(c, s);
    const double2 *T = hop.T + (size_t)r * NB * NB;
#pragma unroll 1
    for (int i = 0; i < NB * NB; ++i) h[i] = c_fma(T[i], ph, h[i]);
  }
}

// h(k) for the step: Peierls h0, mean field, -U n_c; U, V; h written out
template <int NB>
__global__ void __launch_bounds__(256) build_props_kernel(Mesh m, HopTable hop, PropParams p,
                                                          const double2 *__restrict__ hin, double dt,
                                                          double2 *__restrict__ hout,
                                                          double2 *__restrict__ U,
                                                          double2 *__restrict__ V, int kpc,
                                                          const int *__restrict__ skip) {
  if (skip && *skip) return;
  using G = MatGroup<NB>;
  const int span = kpc * G::E;
  double2 *sh[4] = {kbe_dsm, kbe_dsm + span, kbe_dsm + 2 * span, kbe_dsm + 3 * span};
  double *red = (double *)(kbe_dsm + 4 * span);
  const G g;
  const int k = blockIdx.x * kpc + g.kk;
  const bool active = k < m.nk;
  const int nvalid = min(kpc, m.nk - (int)blockIdx.x * kpc);
  const int o = g.kk * G::E + g.e;
  double2 hv = make_double2(0.0, 0.0);
  if (!hin) {
    // h0_ab(k - A d) = sum_r t_ab(R_r) exp(i (k - A d).R_r), this thread's element;
    // the phases of a k-point are computed once, N_b^2 at a time by its threads
    double2 *ph = sh[1] + g.kk * G::E;   // sh[1] is free until the series
    const int k0 = k / m.L1, k1 = k - (k / m.L1) * m.L1;
    for (int r0 = 0; r0 < hop.nhop; r0 += G::E) {
      const int r = r0 + g.e;
      if (active && r < hop.nhop) {
        const int R0 = hop.R[2 * r], R1 = hop.R[2 * r + 1];
        const int m0 = ((k0 * R0) % m.L0 + m.L0) % m.L0, m1 = ((k1 * R1) % m.L1 + m.L1) % m.L1;
        const double th = 2.0 * M_PI * ((double)m0 / m.L0 + (double)m1 / m.L1) - p.A * (hop.d0 * R0 + hop.d1 * R1);
        double sn, cs;
        sincos(th, &sn, &cs);
        ph[g.e] = make_double2(cs, sn);
      }
      __syncthreads();
      if (active)
        for (int q = 0; q < G::E && r0 + q < hop.nhop; ++q)
          hv = c_fma(hop.T[(size_t)(r0 + q) * G::E + g.e], ph[q], hv);
      __syncthreads();
    }
  }
  if (active) {
    if (hin) {
      hv = hin[(size_t)g.e * m.nk + k];
    } else {
      if (p.hf) {   // S_ab = U (delta_ab sum_c v_ac rho_cc - v_ab rho_ab), rho = ca rho_a + cb rho_b
        const double2 rab = c_add(c_scale(p.ca, p.rho_a[g.e]), c_scale(p.cb, p.rho_b[g.e]));
        double2 x = c_scale(-p.v[g.e], rab);
        if (g.a == g.b)
          for (int c = 0; c < NB; ++c) {
            const int ec = c * NB + c;
            x = c_add(x, c_scale(p.v[g.a * NB + c], c_add(c_scale(p.ca, p.rho_a[ec]), c_scale(p.cb, p.rho_b[ec]))));
          }
        hv = c_add(hv, c_scale(p.Umid, x));
      }
      if (p.paper_shift && g.a == NB - 1 && g.b == NB - 1) hv.x -= p.Umid;
      if (p.dipM && p.dipE != 0.0) hv = c_add(hv, c_scale(p.dipE, p.dipM[g.e]));   // Eq. 4
    }
  }
  sh[0][o] = hv;
  __syncthreads();
  const SeriesPlan sp = series_plan<NB>(g, sh[0], kpc, nvalid, dt, red);
  const double tau = ldexp(dt, -sp.s);
  double2 u, v;
  exp_and_phi<NB>(g, sh[0], tau, sp.s, sh[1], sh[2], sh[3], u, v, sp.mexp);
  if (active) {
    const size_t go = (size_t)g.e * m.nk + k;
    if (hout) hout[go] = hv;
    U[go] = u;
    V[go] = v;
  }
}

// time diagonal of row n: G^<(n,n) = U G^<(n-1,n-1) U^+ - i X(Sbar)
template <int NB>
__global__ void __launch_bounds__(256) update_diag_kernel(int n, int nk, double dt, double theta,
                                                          const double2 *__restrict__ h,
                                                          const double2 *__restrict__ Gprev,
                                                          const double2 *__restrict__ Ip,
                                                          const double2 *__restrict__ Ic,
                                                          double2 *__restrict__ out, int kpc,
                                                          const int *__restrict__ skip,
                                                          unsigned long long *maxdiff, void *__restrict__ packed,
                                                          int prec, int cap, const double2 *__restrict__ Uin) {
  if (skip && *skip) return;
  using G = MatGroup<NB>;
  const int span = kpc * G::E;
  double2 *H = kbe_dsm, *Qs = kbe_dsm + span, *T = kbe_dsm + 2 * span, *P = kbe_dsm + 3 * span,
          *Wk = kbe_dsm + 4 * span;
  double *red = (double *)(kbe_dsm + 5 * span);
  const G g;
  const int k = blockIdx.x * kpc + g.kk;
  const bool active = k < nk;
  const int nvalid = min(kpc, nk - (int)blockIdx.x * kpc);
  const int o = g.kk * G::E + g.e;
  const size_t blk = (size_t)G::E * nk;
  double2 hv = make_double2(0, 0), sv = make_double2(0, 0), gd = make_double2(0, 0);
  if (active) {
    const size_t oab = (size_t)g.e * nk + k, oba = (size_t)(g.b * NB + g.a) * nk + k;
    hv = h[oab];
    const double2 *ipd = Ip + (size_t)(n - 1) * 2 * blk;   // I^<_{n-1}(n-1)
    sv = c_scale(1.0 - theta, c_add(ipd[oab], c_conj(ipd[oba])));
    if (theta != 0.0) {
      const double2 *icd = Ic + (size_t)n * 2 * blk;       // I^<_n(n)
      sv = c_add(sv, c_scale(theta, c_add(icd[oab], c_conj(icd[oba]))));
    }
    gd = Gprev[(size_t)(n - 1) * 2 * blk + oab];            // G^<(n-1, n-1)
  }
  H[o] = hv;
  Qs[o] = sv;
  __syncthreads();
  const SeriesPlan sp = series_plan<NB>(g, H, kpc, nvalid, dt, red);
  const int s = sp.s;
  const double tau = ldexp(dt, -s);
  // X_tau = tau sum_m Q_m / (m+1), Q_m = (-i tau / m) [h, Q_{m-1}], Q_0 = Sbar.
  // Sbar is Hermitian, and so is every Q_m (h is): [h, Q] = hQ - (hQ)^+, one
  // product per term; the element (b, a) of hQ comes through shared memory (T).
  // Formed this way every Q_m is exactly Hermitian in floating point.
  double2 x = c_scale(tau, sv);
  for (int m = 1; m <= sp.mx; ++m) {
    const double cm = tau * kSeriesInv[m], cx = tau * kSeriesInv[m + 1];
    const double2 pm = g.mm(H, Qs);   // (h Q_{m-1})_ab
    T[o] = pm;
    __syncthreads();
    const double2 pt = T[g.kk * G::E + g.b * NB + g.a];   // (h Q_{m-1})_ba
    const double2 c = make_double2(pm.x - pt.x, pm.y + pt.y);   // (hQ)_ab - conj((hQ)_ba)
    const double2 q = make_double2(cm * c.y, -cm * c.x);
    Qs[o] = q;
    x = c_add(x, c_scale(cx, q));
    __syncthreads();
  }
  double2 u, v;
  if (s == 0 && Uin) {   // U_tau = U_dt: the step's propagator, built from the same h by the same series
    u = active ? Uin[(size_t)g.e * nk + k] : make_double2(0.0, 0.0);
  } else {
    exp_and_phi<NB>(g, H, tau, 0, P, T, Wk, u, v, sp.mexp);   // U_tau
    (void)v;
  }
  for (int r = 0; r < s; ++r) {   // X <- X + U X U^+, U <- U U
    P[o] = u;
    Qs[o] = x;
    __syncthreads();
    T[o] = g.mm_adj(Qs, P);   // X U^+
    const double2 un = g.mm(P, P);
    __syncthreads();
    x = c_add(x, g.mm(P, T));
    u = un;
    __syncthreads();
  }
  // G = U Gd U^+ - i X
  P[o] = u;
  Qs[o] = gd;
  __syncthreads();
  T[o] = g.mm_adj(Qs, P);
  __syncthreads();
  const double2 gg = c_sub(g.mm(P, T), c_i(x));
  if (active) {
    double2 *ol = out + (size_t)n * 2 * blk + (size_t)g.e * nk + k;
    if (maxdiff) {
      const double2 d = c_sub(gg, ol[0]);
      atomicMax(maxdiff, (unsigned long long)__double_as_longlong(sqrt(d.x * d.x + d.y * d.y)));
    }
    const double2 gG = (g.a == g.b) ? make_double2(gg.x, gg.y - 1.0) : gg;
    ol[0] = gg;
    ol[blk] = gG;
    if (packed) {
      const size_t o0 = (size_t)n * 2 * blk + (size_t)g.e * nk + k;
      pack_store(prec, packed, o0, o0 + blk, gg, c_sub(gg, gG), NB, nk, n, cap);
    }
  }
}

// t = 0: G^<(k;0,0) = i W f(lam) W^+ of h0(k), G^> = G^< - i
template <int NB>
__global__ void init_state_kernel(Mesh m, HopTable hop, double beta, double mu, double2 *H00,
                                  int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.nk) return;
  double2 h[NB * NB], Wl[NB * NB];
  double ll[NB], f[NB];
  bare_h<NB>(hop, k, m.L0, m.L1, 0.0, h);
  if (!herm_eig<NB>(h, ll, Wl)) atomicOr(status, kDevEigNoConv);
#pragma unroll 1
  for (int c = 0; c < NB; ++c) {
    const double x = beta * (ll[c] - mu);
    if (x > 0) {
      const double y = exp(-x);
      f[c] = y / (1.0 + y);
    } else {
      f[c] = 1.0 / (1.0 + exp(x));
    }
  }
  const size_t blk = (size_t)NB * NB * m.nk;
#pragma unroll 1
  for (int a = 0; a < NB; ++a)
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
      double2 r = make_double2(0, 0);
#pragma unroll 1
      for (int c = 0; c < NB; ++c) r = c_add(r, c_scale(f[c], c_mulc(Wl[a * NB + c], Wl[b * NB + c])));
      const double2 gl = c_i(r);
      const size_t o = (size_t)(a * NB + b) * m.nk + k;
      H00[o] = gl;
      H00[blk + o] = (a == b) ? make_double2(gl.x, gl.y - 1.0) : gl;
    }
}

// rho_loc_ab = (1/n_k) sum_k (-i) G^<_ab(k; n, n); one CTA, a warp per element
__global__ void local_density_kernel(int nb, int nk, const double2 *__restrict__ G, double2 *out,
                                     const int *__restrict__ skip) {
  if (skip && *skip) return;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int e = warp; e < nb * nb; e += nw) {
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < nk; k += 32) {
      const double2 g = G[(size_t)e * nk + k];
      sr += g.y;    // Re(-i g) = Im g
      si -= g.x;    // Im(-i g) = -Re g
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, off);
      si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) out[e] = make_double2(sr / nk, si / nk);
  }
}

// rows j < n: G^x(n,j) = U G^x(n-1,j) + V [(1-theta) Ip^x(j) + theta Ic^x(j)];
// one thread per (j, b, k) and a chunk of UA rows a (all N_b rows up to N_b =
// 8): the column b of G(n-1, j) and of the blended Ibar(j) is loaded and
// blended once per thread and reused for every row a of the chunk (the FP64
// blend was 3/7 of the pipe work when every output formed it again). Each
// output accumulates in the same order as a per-output sum over c. The thread
// forms both components of its outputs, so that it can also store the
// history's (G^<, dG) pair of each (packed != NULL).
template <int NB>
__host__ __device__ constexpr int update_chunk() { return NB <= 8 ? NB : 4; }

template <int NB>
__global__ void update_rows_kernel(int n, int nk, double theta, const double2 *__restrict__ U,
                                   const double2 *__restrict__ V, const double2 *__restrict__ Gprev,
                                   const double2 *__restrict__ Ip, const double2 *__restrict__ Ic,
                                   double2 *__restrict__ out, const int *__restrict__ skip,
                                   unsigned long long *maxdiff, void *__restrict__ packed, int prec, int cap) {
  if (skip && *skip) return;
  constexpr int UA = update_chunk<NB>(), NCH = NB / UA;
  const size_t blk = (size_t)NB * NB * nk;
  const size_t total = (size_t)n * NCH * NB * nk;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dmax = 0.0;
  if (idx < total) {
    const int k = (int)(idx % nk);
    size_t t = idx / nk;
    const int b = (int)(t % NB);
    t /= NB;
    const int a0 = (int)(t % NCH) * UA;
    const size_t j = t / NCH;
    const size_t base = j * 2 * blk;
    double2 acc0[UA], acc1[UA];
#pragma unroll
    for (int q = 0; q < UA; ++q) acc0[q] = acc1[q] = make_double2(0, 0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const size_t oc = (size_t)(c * NB + b) * nk + k;
      // Ibar = (1 - theta) Ip + theta Ic with real scalars (the same values as
      // complex products with a zero imaginary part, at half the FP64 work)
      double2 ib0 = Ip[base + oc], ib1 = Ip[base + blk + oc];
      if (theta != 0.0) {
        const double2 c0 = Ic[base + oc], c1 = Ic[base + blk + oc];
        ib0 = make_double2(fma(theta, c0.x, (1.0 - theta) * ib0.x), fma(theta, c0.y, (1.0 - theta) * ib0.y));
        ib1 = make_double2(fma(theta, c1.x, (1.0 - theta) * ib1.x), fma(theta, c1.y, (1.0 - theta) * ib1.y));
      }
      const double2 g0 = Gprev[base + oc], g1 = Gprev[base + blk + oc];
#pragma unroll
      for (int q = 0; q < UA; ++q) {
        const size_t ou = (size_t)((a0 + q) * NB + c) * nk + k;
        const double2 u = U[ou], v = V[ou];
        acc0[q] = c_fma(u, g0, acc0[q]);
        acc0[q] = c_fma(v, ib0, acc0[q]);
        acc1[q] = c_fma(u, g1, acc1[q]);
        acc1[q] = c_fma(v, ib1, acc1[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < UA; ++q) {
      const size_t oo = base + (size_t)((a0 + q) * NB + b) * nk + k;
      if (maxdiff) {   // G^< entries
        const double2 d = c_sub(acc0[q], out[oo]);
        dmax = fmax(dmax, sqrt(d.x * d.x + d.y * d.y));
      }
      out[oo] = acc0[q];
      out[oo + blk] = acc1[q];
      if (packed) pack_store(prec, packed, oo, oo + blk, acc0[q], c_sub(acc0[q], acc1[q]), NB, nk, n, cap);
    }
  }
  if (maxdiff) {   // every lane reaches here (blockDim is a multiple of 32)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    if ((threadIdx.x & 31) == 0 && dmax > 0.0)
      atomicMax(maxdiff, (unsigned long long)__double_as_longlong(dmax));
  }
}

__global__ void corr_check_kernel(unsigned long long *maxdiff, double tol, int *skip, int *iters) {
  if (*skip) return;
  *iters += 1;
  if (__longlong_as_double((long long)*maxdiff) <= tol) *skip = 1;
  *maxdiff = 0ull;
}

// equal-time observables of row n. One matrix group per k-point (kpc k-points
// per CTA, as the propagator kernels): the threads of a k-point compute its
// Peierls phases together, N_b^2 at a time, then thread (a, b) forms h0_ab(k)
// and its terms of the sums; each CTA reduces its terms in a fixed tree and
// writes (N, K, C) to part[3 blockIdx]; the CTA that finishes last (a ticket
// counter, reset by it) adds the partials in CTA order and writes obs. The
// result does not depend on the order in which the CTAs ran.
template <int NB>
__global__ void __launch_bounds__(256) observables_kernel(Mesh m, HopTable hop, ObsParams p,
                                                          const double2 *__restrict__ G,
                                                          const double2 *__restrict__ Idg,
                                                          const double2 *__restrict__ rho, double *obs, double *nkb,
                                                          int *status, int kpc, double *part, unsigned *ticket) {
  using Gp = MatGroup<NB>;
  double2 *ph = kbe_dsm;                                   // [kk][E] phases
  double *red = (double *)(kbe_dsm + (size_t)kpc * Gp::E);  // [3][threads]
  __shared__ bool last;
  const Gp g;
  const int k = blockIdx.x * kpc + g.kk;
  const bool active = k < m.nk;
  const int nt = blockDim.x;
  double2 hv = make_double2(0.0, 0.0);
  const int k0 = k / m.L1, k1 = k - (k / m.L1) * m.L1;
  for (int r0 = 0; r0 < hop.nhop; r0 += Gp::E) {
    const int r = r0 + g.e;
    if (active && r < hop.nhop) {
      const int R0 = hop.R[2 * r], R1 = hop.R[2 * r + 1];
      // reduce the lattice phase exactly before converting to an angle
      const int m0 = ((k0 * R0) % m.L0 + m.L0) % m.L0, m1 = ((k1 * R1) % m.L1 + m.L1) % m.L1;
      const double th = 2.0 * M_PI * ((double)m0 / m.L0 + (double)m1 / m.L1) - p.Abar * (hop.d0 * R0 + hop.d1 * R1);
      double sn, cs;
      sincos(th, &sn, &cs);
      ph[g.kk * Gp::E + g.e] = make_double2(cs, sn);
    }
    __syncthreads();
    if (active)
      for (int q = 0; q < Gp::E && r0 + q < hop.nhop; ++q)
        hv = c_fma(hop.T[(size_t)(r0 + q) * Gp::E + g.e], ph[g.kk * Gp::E + q], hv);
    __syncthreads();
  }
  double sN = 0.0, sK = 0.0, sC = 0.0;
  if (active) {
    const double2 gba = G[(size_t)(g.b * NB + g.a) * m.nk + k];   // rho_ba = -i G_ba
    sK = c_mul(hv, make_double2(gba.y, -gba.x)).x;
    if (g.a == g.b) {
      sN = gba.y;                                                 // Re(-i G_aa)
      nkb[(size_t)k * NB + g.a] = sN;
      sC = Idg[(size_t)(g.a * NB + g.a) * m.nk + k].y;            // Re(-i I_aa)
    }
  }
  red[threadIdx.x] = sN;
  red[nt + threadIdx.x] = sK;
  red[2 * nt + threadIdx.x] = sC;
  __syncthreads();
  int span = 1;
  while (span < nt) span <<= 1;
  for (int st = span >> 1; st > 0; st >>= 1) {   // fixed tree over the CTA's threads
    if ((int)threadIdx.x < st && (int)threadIdx.x + st < nt)
      for (int q = 0; q < 3; ++q) red[q * nt + threadIdx.x] += red[q * nt + threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = red[q * nt];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double N = 0, K = 0, C = 0;
  for (int c = 0; c < (int)gridDim.x; ++c) {
    N += __ldcg(part + 3 * c);
    K += __ldcg(part + 3 * c + 1);
    C += __ldcg(part + 3 * c + 2);
  }
  *ticket = 0u;   // ready for the next launch (stream order)
  double Ehf = 0.0, Esh = 0.0;
  if (p.hf) {
    for (int jj = 0; jj < NB; ++jj)
      for (int mm = 0; mm < NB; ++mm) {
        double2 x = c_scale(-p.v[jj * NB + mm], rho[jj * NB + mm]);
        if (jj == mm)
          for (int a = 0; a < NB; ++a) x = c_add(x, c_scale(p.v[jj * NB + a], rho[a * NB + a]));
        Ehf += 0.5 * c_mul(c_scale(p.Un, x), rho[mm * NB + jj]).x;
      }
  }
  if (p.paper_shift) Esh = -p.Un * rho[(NB - 1) * NB + NB - 1].x;
  obs[0] = N / m.nk;
  obs[1] = K / m.nk;
  obs[2] = Ehf;
  obs[3] = 0.5 * C / m.nk;
  obs[4] = Esh;
  obs[5] = obs[1] + obs[2] + obs[3] + obs[4];
  if (!isfinite(obs[0]) || !isfinite(obs[5])) atomicOr(status, kDevNonFinite);
}

}  // namespace

template <int NB>
size_t obs_smem(int nk) {
  return sizeof(double2) * (size_t)matgroup_kpc<NB>(nk) * NB * NB + sizeof(double) * 3 * matgroup_threads<NB>(nk);
}

cudaError_t launch_init_state(const Mesh &m, const HopTable &hop, double beta, double mu,
                              double2 *H00, int *status, cudaStream_t st) {
  const int threads = 64, blocks = (m.nk + threads - 1) / threads;
  KBE_NB_SWITCH(m.nb, (init_state_kernel<NB><<<blocks, threads, 0, st>>>(m, hop, beta, mu, H00, status)));
  return cudaGetLastError();
}

cudaError_t launch_local_density(const Mesh &m, const double2 *Gdiag, double2 *rho_out,
                                 cudaStream_t st, const int *skip) {
  local_density_kernel<<<1, 256, 0, st>>>(m.nb, m.nk, Gdiag, rho_out, skip);
  return cudaGetLastError();
}

cudaError_t launch_build_props(const Mesh &m, const HopTable &hop, const PropParams &p, double dt,
                               const double2 *h_in, double2 *h_out, double2 *U, double2 *V,
                               cudaStream_t st, const int *skip) {
  KBE_NB_SWITCH(m.nb, (build_props_kernel<NB><<<matgroup_blocks<NB>(m.nk), matgroup_threads<NB>(m.nk),
                                                 matgroup_smem<NB>(m.nk, 4), st>>>(
                          m, hop, p, h_in, dt, h_out, U, V, matgroup_kpc<NB>(m.nk), skip)));
  return cudaGetLastError();
}

cudaError_t launch_update_row(const Mesh &m, int n, double dt, double theta, const double2 *h,
                              const double2 *U, const double2 *V, const double2 *Gprev,
                              const double2 *Iprev, const double2 *Icur, double2 *out,
                              cudaStream_t st, const int *skip, unsigned long long *maxdiff, void *packed,
                              int prec, int cap) {
  const size_t total = (size_t)n * (m.nb / (m.nb <= 8 ? m.nb : 4)) * m.nb * m.nk;   // (j, a chunk, b, k)
  const int threads = 256;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  const double2 *ic = (theta != 0.0) ? Icur : Iprev;
  KBE_NB_SWITCH(m.nb, (update_diag_kernel<NB><<<matgroup_blocks<NB>(m.nk), matgroup_threads<NB>(m.nk),
                                                 matgroup_smem<NB>(m.nk, 5), st>>>(
                          n, m.nk, dt, theta, h, Gprev, Iprev, ic, out, matgroup_kpc<NB>(m.nk), skip,
                          maxdiff, packed, prec, cap, U)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || total == 0) return e;
  KBE_NB_SWITCH(m.nb, (update_rows_kernel<NB><<<blocks, threads, 0, st>>>(n, m.nk, theta, U, V, Gprev, Iprev, ic,
                                                                           out, skip, maxdiff, packed, prec, cap)));
  return cudaGetLastError();
}

cudaError_t launch_corr_check(unsigned long long *maxdiff, double tol, int *skip, int *iters,
                              cudaStream_t st) {
  corr_check_kernel<<<1, 1, 0, st>>>(maxdiff, tol, skip, iters);
  return cudaGetLastError();
}

cudaError_t launch_observables(const Mesh &m, const HopTable &hop, const ObsParams &p,
                               const double2 *Gdiag, const double2 *Idiag, const double2 *rho_n,
                               double *obs_out, double *nkb_out, int *status, double *part, unsigned *ticket,
                               cudaStream_t st) {
  KBE_NB_SWITCH(m.nb, (observables_kernel<NB><<<matgroup_blocks<NB>(m.nk), matgroup_threads<NB>(m.nk),
                                                 obs_smem<NB>(m.nk), st>>>(
                          m, hop, p, Gdiag, Idiag, rho_n, obs_out, nkb_out, status, matgroup_kpc<NB>(m.nk), part,
                          ticket)));
  return cudaGetLastError();
}

}  // namespace kbe
