/*
 * FP64 CPU oracle for the Kadanoff-Baym time stepping of arXiv 2505.19467,
 * "GPU Acceleration of Non-equilibrium Green's Function Calculation using
 * OpenACC and CUDA FORTRAN".
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg load this library. It shares no code,
 * header, table or helper with the CUDA library, and it is slow on purpose:
 * plain loops over k, bands and times, std C99 complex doubles, OpenMP only
 * over independent outputs.
 *
 * What it computes (paper sections / equations):
 *   - Two-band lattice model, Sec. 2 Eqs. 2-4, generalised to N_b bands with a
 *     density-density pairing pattern v_ab (v = 1 - delta reduces to the
 *     paper's bar convention at N_b = 2) and a Peierls drive h0(k - A d).
 *   - Second-Born self-energy, Eq. 7, in the factorised form of Eqs. 8-9 for
 *     the direct term and an exchange intermediate X_jba(d) for the second
 *     term (O(n_k^2) per time pair); orc_sigma_pair_literal is Eq. 7 summed
 *     directly over both momenta (O(n_k^3)).
 *   - Collision integrals, Eq. 6, read as the left (Sigma * G) form
 *         I^x(n,j) = sum_{l<=n} w^(n)_l [S^> - S^<](n,l) G^x(l,j)
 *                  + sum_{l<=j} w^(j)_l  S^x(n,l) [G^< - G^>](l,j)
 *     with composite trapezoid weights (Sec. 2, "standard second order").
 *   - Algorithm 1: predictor with the stored I of row n-1, n_corr corrector
 *     passes with I averaged over rows n-1 and n, then a final evaluation
 *     whose I row is kept for the next step.
 *   - Exponential row update G(n,j) = U G(n-1,j) + V Ibar(j), U = e^{-i dt h},
 *     V = (U - 1) h^{-1}; the time diagonal by the divided-difference form
 *     G(n,n) = U G(n-1,n-1) U^+ - i W[(W^+ Sbar W) o D] W^+.
 *   - Hartree-Fock mean field and the -U n_c term of Eq. 2 inside h.
 *   - Equal-time observables (density, particle number, energies).
 *   - Full-grid mode (tiny grids): the upper triangle propagated on its own
 *     with the right-hand equation and Eq. 6 as printed (G * Sigma), so that
 *     the adjoint symmetry becomes a checked result instead of an assumption.
 *
 * Storage: the lower triangle of the two-time grid, block (i, j), i >= j, at
 * index i(i+1)/2 + j; every block is [k][a][b] complex. G(l, j) for l < j is
 * obtained through G^x(t,t')^+ = -G^x(t',t).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#undef I
typedef double complex cplx;
#define IU (_Complex_I)
#define MAXNB 16

/* ------------------------------------------------------------------------ */
/* small dense helpers on n x n row-major complex matrices                   */
/* ------------------------------------------------------------------------ */

static void mat_mul(int n, const cplx *A, const cplx *B, cplx *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0;
      for (int m = 0; m < n; ++m) s += A[i * n + m] * B[m * n + j];
      C[i * n + j] = s;
    }
}

/* C = A * B^+ */
static void mat_mul_adj(int n, const cplx *A, const cplx *B, cplx *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0;
      for (int m = 0; m < n; ++m) s += A[i * n + m] * conj(B[j * n + m]);
      C[i * n + j] = s;
    }
}

/* C = A^+ * B */
static void mat_adj_mul(int n, const cplx *A, const cplx *B, cplx *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cplx s = 0;
      for (int m = 0; m < n; ++m) s += conj(A[m * n + i]) * B[m * n + j];
      C[i * n + j] = s;
    }
}

/*
 * Eigen-decomposition of a Hermitian matrix by cyclic Jacobi rotations:
 * A = W diag(lam) W^+, W unitary with eigenvectors as columns.
 * Each rotation first removes the phase of A_pq, then applies the real
 * symmetric Jacobi rotation with t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
 * tau = (A_qq - A_pp) / (2 |A_pq|).
 */
static void herm_eig(int n, const cplx *Ain, double *lam, cplx *W) {
  cplx A[MAXNB * MAXNB];
  memcpy(A, Ain, sizeof(cplx) * n * n);
  for (int i = 0; i < n * n; ++i) W[i] = 0;
  for (int i = 0; i < n; ++i) W[i * n + i] = 1;
  for (int i = 0; i < n; ++i) A[i * n + i] = creal(A[i * n + i]);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, tot = 0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        double m2 = creal(A[p * n + q]) * creal(A[p * n + q]) + cimag(A[p * n + q]) * cimag(A[p * n + q]);
        tot += m2;
        if (p != q) off += m2;
      }
    if (off == 0.0 || off <= 1e-34 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        cplx apq = A[p * n + q];
        double r = cabs(apq);
        if (r == 0.0) continue;
        cplx e = apq / r;
        double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
        double tau = (aqq - app) / (2.0 * r);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        cplx ce = conj(e);
        for (int i = 0; i < n; ++i) { /* A <- A J */
          cplx x = A[i * n + p], y = A[i * n + q];
          A[i * n + p] = c * x - s * ce * y;
          A[i * n + q] = s * x + c * ce * y;
        }
        for (int j = 0; j < n; ++j) { /* A <- J^+ A */
          cplx x = A[p * n + j], y = A[q * n + j];
          A[p * n + j] = c * x - s * e * y;
          A[q * n + j] = s * x + c * e * y;
        }
        for (int i = 0; i < n; ++i) { /* W <- W J */
          cplx x = W[i * n + p], y = W[i * n + q];
          W[i * n + p] = c * x - s * ce * y;
          W[i * n + q] = s * x + c * ce * y;
        }
        A[p * n + q] = 0;
        A[q * n + p] = 0;
        A[p * n + p] = creal(A[p * n + p]);
        A[q * n + q] = creal(A[q * n + q]);
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = creal(A[i * n + i]);
}

/* Fermi function 1 / (e^{beta (e - mu)} + 1), written to avoid overflow. */
static double fermi(double e, double beta, double mu) {
  double x = beta * (e - mu);
  if (x > 0) {
    double y = exp(-x);
    return y / (1.0 + y);
  }
  return 1.0 / (1.0 + exp(x));
}

/* ------------------------------------------------------------------------ */
/* k mesh                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int L0, L1;
} mesh;

static int k_add(mesh m, int a, int b) {
  int a0 = a / m.L1, a1 = a % m.L1, b0 = b / m.L1, b1 = b % m.L1;
  return ((a0 + b0) % m.L0) * m.L1 + (a1 + b1) % m.L1;
}
static int k_sub(mesh m, int a, int b) {
  int a0 = a / m.L1, a1 = a % m.L1, b0 = b / m.L1, b1 = b % m.L1;
  return ((a0 - b0 + m.L0) % m.L0) * m.L1 + (a1 - b1 + m.L1) % m.L1;
}

/* ------------------------------------------------------------------------ */
/* second-Born self-energy, Eq. 7                                            */
/* ------------------------------------------------------------------------ */

/*
 * One component x of Sigma for one time pair (t_n, t_l), Eqs. 7-9:
 *   G  = G^x(k; n, l),  Gp = G^{xbar}(k; n, l)  (both [k][a][b]),
 *   Gt_ab(k) = G^{xbar}_ab(k; l, n) = -conj(Gp_ba(k))   (adjoint symmetry).
 * Direct term (Eqs. 8-9): P_ab(q) = sum_k' G_ab(k'+q) Gt_ba(k'),
 *   S1_jm(k) = sum_q [sum_ab v_ja v_mb P_ab(q)] G_jm(k-q).
 * Exchange term: X_jba(d) = sum_k' G_jb(k') Gt_ba(k'+d),
 *   S2_jm(k) = sum_ab v_ja v_mb sum_q X_jba(q-k) G_am(q).
 * Sigma^x = U(t_n) U(t_l) / n_k^2 (S1 - S2).
 */
static void sigma_one(int nb, mesh m, const double *v, double UnUl, const cplx *G,
                      const cplx *Gp, cplx *S) {
  int nk = m.L0 * m.L1, nb2 = nb * nb;
  cplx *Gt = malloc(sizeof(cplx) * nk * nb2);
  cplx *P = malloc(sizeof(cplx) * nk * nb2);
  cplx *Q = malloc(sizeof(cplx) * nk * nb2);
  cplx *X = malloc(sizeof(cplx) * (size_t)nk * nb * nb2);
  for (int k = 0; k < nk; ++k)
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) Gt[k * nb2 + a * nb + b] = -conj(Gp[k * nb2 + b * nb + a]);
  /* Eq. 8 */
  for (int q = 0; q < nk; ++q)
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx s = 0;
        for (int kp = 0; kp < nk; ++kp)
          s += G[k_add(m, kp, q) * nb2 + a * nb + b] * Gt[kp * nb2 + b * nb + a];
        P[q * nb2 + a * nb + b] = s;
      }
  for (int q = 0; q < nk; ++q)
    for (int j = 0; j < nb; ++j)
      for (int mm = 0; mm < nb; ++mm) {
        cplx s = 0;
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) s += v[j * nb + a] * v[mm * nb + b] * P[q * nb2 + a * nb + b];
        Q[q * nb2 + j * nb + mm] = s;
      }
  /* exchange intermediate */
  for (int d = 0; d < nk; ++d)
    for (int j = 0; j < nb; ++j)
      for (int b = 0; b < nb; ++b)
        for (int a = 0; a < nb; ++a) {
          cplx s = 0;
          for (int kp = 0; kp < nk; ++kp)
            s += G[kp * nb2 + j * nb + b] * Gt[k_add(m, kp, d) * nb2 + b * nb + a];
          X[((size_t)d * nb + j) * nb2 + b * nb + a] = s;
        }
  double scale = UnUl / ((double)nk * nk);
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nb; ++j)
      for (int mm = 0; mm < nb; ++mm) {
        cplx s1 = 0, s2 = 0;
        for (int q = 0; q < nk; ++q) s1 += Q[q * nb2 + j * nb + mm] * G[k_sub(m, k, q) * nb2 + j * nb + mm];
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) {
            double vv = v[j * nb + a] * v[mm * nb + b];
            if (vv == 0.0) continue;
            cplx s = 0;
            for (int q = 0; q < nk; ++q)
              s += X[((size_t)k_sub(m, q, k) * nb + j) * nb2 + b * nb + a] * G[q * nb2 + a * nb + mm];
            s2 += vv * s;
          }
        S[k * nb2 + j * nb + mm] = scale * (s1 - s2);
      }
  free(Gt);
  free(P);
  free(Q);
  free(X);
}

/* Sigma^<(n,l) and Sigma^>(n,l) from G^<(n,l), G^>(n,l) (Eq. 7; > is < with
 * the lesser and greater functions exchanged). Layout [k][a][b]. */
void orc_sigma_pair(int nb, int L0, int L1, const double *v, double UnUl, const double *Gl,
                    const double *Gg, double *Sl, double *Sg) {
  mesh m = {L0, L1};
  sigma_one(nb, m, v, UnUl, (const cplx *)Gl, (const cplx *)Gg, (cplx *)Sl);
  sigma_one(nb, m, v, UnUl, (const cplx *)Gg, (const cplx *)Gl, (cplx *)Sg);
}

/*
 * Eq. 7 summed term by term over the two momenta, O(n_k^3) per time pair,
 * with both time orderings given explicitly:
 *   Gf = G^x(k; t, t')      and   Gb = G^{xbar}(k; t', t),   both [k][a][b].
 * For every output (k, j, m), every interacting pair of bands (a, b) with
 * weight v_ja v_mb, every transfer p (the paper's q) and loop momentum r (the
 * paper's k'):
 *   + Gf_ab(r + p) Gb_ba(r) Gf_jm(k - p)          (direct term)
 *   - Gf_jb(r) Gb_ba(r + p - k) Gf_am(p)          (exchange term)
 * scaled by U(t) U(t') / n_k^2. With v == NULL (N_b = 2 only) the band
 * indices are the paper's bar convention: the one pair a = 1 - j, b = 1 - m.
 * No symmetry of G is used here; the caller decides where Gb comes from.
 */
static void sigma_eq7(int nb, mesh m, const double *v, double UtUt, const cplx *Gf, const cplx *Gb,
                      cplx *S) {
  int nk = m.L0 * m.L1, nb2 = nb * nb;
  double scale = UtUt / ((double)nk * nk);
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nb; ++j)
      for (int mm = 0; mm < nb; ++mm) {
        cplx acc = 0;
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) {
            double wgt;
            if (v == NULL) wgt = (a == 1 - j && b == 1 - mm) ? 1.0 : 0.0;
            else wgt = v[j * nb + a] * v[mm * nb + b];
            if (wgt == 0.0) continue;
            cplx direct = 0, exch = 0;
            for (int p = 0; p < nk; ++p) {
              int kmp = k_sub(m, k, p);
              for (int r = 0; r < nk; ++r) {
                int rp = k_add(m, r, p), rpk = k_sub(m, rp, k);
                direct += Gf[rp * nb2 + a * nb + b] * Gb[r * nb2 + b * nb + a] * Gf[kmp * nb2 + j * nb + mm];
                exch += Gf[r * nb2 + j * nb + b] * Gb[rpk * nb2 + b * nb + a] * Gf[p * nb2 + a * nb + mm];
              }
            }
            acc += wgt * (direct - exch);
          }
        S[k * nb2 + j * nb + mm] = scale * acc;
      }
}

/* Eq. 7 as a direct sum for the pair (t_n, t_l), given G^<, G^>(k; t_n, t_l):
 * the reversed-time factors come from the adjoint symmetry,
 * G^{xbar}_ab(k; t_l, t_n) = -conj(G^{xbar}_ba(k; t_n, t_l)). */
void orc_sigma_pair_literal(int nb, int L0, int L1, const double *v, double UnUl,
                            const double *Gl_, const double *Gg_, double *Sl, double *Sg) {
  mesh m = {L0, L1};
  int nk = L0 * L1, nb2 = nb * nb;
  const cplx *Gl = (const cplx *)Gl_, *Gg = (const cplx *)Gg_;
  cplx *Bl = malloc(sizeof(cplx) * nk * nb2), *Bg = malloc(sizeof(cplx) * nk * nb2);
  for (int k = 0; k < nk; ++k)
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        Bl[k * nb2 + a * nb + b] = -conj(Gl[k * nb2 + b * nb + a]);
        Bg[k * nb2 + a * nb + b] = -conj(Gg[k * nb2 + b * nb + a]);
      }
  sigma_eq7(nb, m, v, UnUl, Gl, Bg, (cplx *)Sl);
  sigma_eq7(nb, m, v, UnUl, Gg, Bl, (cplx *)Sg);
  free(Bl);
  free(Bg);
}

/* ------------------------------------------------------------------------ */
/* collision integrals, Eq. 6 (left form)                                    */
/* ------------------------------------------------------------------------ */

static size_t tri(int i, int j) { return (size_t)i * (i + 1) / 2 + j; }

/* composite trapezoid weight of node l on [0, t_m] (zero for m = 0) */
static double trap_w(int m, int l, double dt) {
  if (m == 0) return 0.0;
  double w = dt;
  if (l == 0) w -= 0.5 * dt;
  if (l == m) w -= 0.5 * dt;
  return w;
}

/* Weight of node l for the integral over [0, t_m] with quadrature quad:
 * 0 the composite trapezoid rule; 1 the fourth-order Gregory rule (end
 * corrections 3/8, 7/6, 23/24 of the trapezoid's unit interior weight) when
 * m >= 5, and for 1 <= m <= 4 the closed Newton-Cotes rule over all m + 1
 * nodes (trapezoid, Simpson 1/3, Simpson 3/8, Boole). Zero for m = 0. */
static double quad_w(int quad, int m, int l, double dt) {
  static const double newton_cotes[5][5] = {
      {0.0},
      {1.0 / 2, 1.0 / 2},
      {1.0 / 3, 4.0 / 3, 1.0 / 3},
      {3.0 / 8, 9.0 / 8, 9.0 / 8, 3.0 / 8},
      {14.0 / 45, 64.0 / 45, 24.0 / 45, 64.0 / 45, 14.0 / 45}};
  static const double gregory_end[3] = {3.0 / 8, 7.0 / 6, 23.0 / 24};
  if (quad == 0) return trap_w(m, l, dt);
  if (m <= 4) return dt * newton_cotes[m][l];
  int d = l <= m - l ? l : m - l; /* distance to the nearer end */
  return dt * (d < 3 ? gregory_end[d] : 1.0);
}

/* block G^x(l, j) at one k for any l, j, from the lower triangle H */
static void fetch(int nb, int nk, const cplx *H, int l, int j, int k, cplx *out) {
  size_t blk = (size_t)nk * nb * nb;
  if (l >= j) {
    memcpy(out, H + tri(l, j) * blk + (size_t)k * nb * nb, sizeof(cplx) * nb * nb);
  } else {
    const cplx *s = H + tri(j, l) * blk + (size_t)k * nb * nb;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) out[a * nb + b] = -conj(s[b * nb + a]);
  }
}

/* block G^x(l, j) at one k: from the lower triangle H when l >= j, else from
 * the separately propagated column store C (full-grid mode; nothing is
 * mirrored), or, with C == NULL, by the adjoint symmetry from H */
static void fetch_grid(int nb, int nk, const cplx *H, const cplx *C, int l, int j, int k, cplx *out) {
  if (l < j && C != NULL)
    memcpy(out, C + tri(j, l) * (size_t)nk * nb * nb + (size_t)k * nb * nb, sizeof(cplx) * nb * nb);
  else
    fetch(nb, nk, H, l, j, k, out);
}

/*
 * I^x(n, j), j = 0..n, x in {<, >}:
 *   sum_{l=0}^{n} w^(n)_l [S^>(n,l) - S^<(n,l)] G^x(l,j)
 * + sum_{l=0}^{j} w^(j)_l S^x(n,l) [G^<(l,j) - G^>(l,j)].
 * H*: triangle with rows 0..n; C*: column store or NULL; S*: [l][k][a][b],
 * l <= n; I*: [j][k][a][b].
 */
static void collision_left(int nb, int nk, int n, double dt, int quad, const cplx *Hl, const cplx *Hg,
                           const cplx *Cl, const cplx *Cg, const cplx *Sl, const cplx *Sg, cplx *Il,
                           cplx *Ig) {
  size_t blk = (size_t)nk * nb * nb;
  int nb2 = nb * nb;
#pragma omp parallel for schedule(dynamic) collapse(2)
  for (int j = 0; j <= n; ++j)
    for (int k = 0; k < nk; ++k) {
      cplx gl[MAXNB * MAXNB], gg[MAXNB * MAXNB], sr[MAXNB * MAXNB], dg[MAXNB * MAXNB];
      cplx tl[MAXNB * MAXNB], tg[MAXNB * MAXNB], accl[MAXNB * MAXNB], accg[MAXNB * MAXNB];
      for (int e = 0; e < nb2; ++e) accl[e] = accg[e] = 0;
      for (int l = 0; l <= n; ++l) {
        const cplx *sl = Sl + l * blk + (size_t)k * nb2, *sg = Sg + l * blk + (size_t)k * nb2;
        fetch_grid(nb, nk, Hl, Cl, l, j, k, gl);
        fetch_grid(nb, nk, Hg, Cg, l, j, k, gg);
        double w1 = quad_w(quad, n, l, dt);
        for (int e = 0; e < nb2; ++e) sr[e] = w1 * (sg[e] - sl[e]);
        mat_mul(nb, sr, gl, tl);
        mat_mul(nb, sr, gg, tg);
        for (int e = 0; e < nb2; ++e) {
          accl[e] += tl[e];
          accg[e] += tg[e];
        }
        if (l <= j) {
          double w2 = quad_w(quad, j, l, dt);
          for (int e = 0; e < nb2; ++e) dg[e] = gl[e] - gg[e];
          mat_mul(nb, sl, dg, tl);
          mat_mul(nb, sg, dg, tg);
          for (int e = 0; e < nb2; ++e) {
            accl[e] += w2 * tl[e];
            accg[e] += w2 * tg[e];
          }
        }
      }
      memcpy(Il + j * blk + (size_t)k * nb2, accl, sizeof(cplx) * nb2);
      memcpy(Ig + j * blk + (size_t)k * nb2, accg, sizeof(cplx) * nb2);
    }
}

void orc_collision_row_q(int nb, int nk, int n, double dt, int quad, const double *Hl, const double *Hg,
                         const double *Sl, const double *Sg, double *Il, double *Ig) {
  collision_left(nb, nk, n, dt, quad, (const cplx *)Hl, (const cplx *)Hg, NULL, NULL, (const cplx *)Sl,
                 (const cplx *)Sg, (cplx *)Il, (cplx *)Ig);
}

void orc_collision_row(int nb, int nk, int n, double dt, const double *Hl, const double *Hg,
                       const double *Sl, const double *Sg, double *Il, double *Ig) {
  orc_collision_row_q(nb, nk, n, dt, 0, Hl, Hg, Sl, Sg, Il, Ig);
}

/* ------------------------------------------------------------------------ */
/* propagators and the time-step update                                      */
/* ------------------------------------------------------------------------ */

/* (e^{-i x} - 1) / x * dt with x = lam dt, cancellation-free; -i dt at x=0 */
static cplx phi_v(double lam, double dt) {
  double x = lam * dt;
  if (x == 0.0) return -IU * dt;
  double s2 = sin(0.5 * x);
  return dt * (-2.0 * s2 * s2 / x - IU * sin(x) / x);
}

/* D = (1 - e^{-i y}) / (i y) * dt with y = (lam_a - lam_b) dt; dt at y = 0 */
static cplx phi_d(double dl, double dt) {
  double y = dl * dt;
  if (y == 0.0) return dt;
  double s2 = sin(0.5 * y);
  return dt * (sin(y) / y - IU * 2.0 * s2 * s2 / y);
}

/* per k: h = W diag(lam) W^+, U = e^{-i dt h}, V = (U - 1) h^{-1} */
void orc_propagators(int nb, int nk, double dt, const double *h_, double *U_, double *V_,
                     double *W_, double *lam) {
  const cplx *h = (const cplx *)h_;
  cplx *U = (cplx *)U_, *V = (cplx *)V_, *W = (cplx *)W_;
  int nb2 = nb * nb;
  for (int k = 0; k < nk; ++k) {
    const cplx *hk = h + (size_t)k * nb2;
    cplx *Wk = W + (size_t)k * nb2;
    double *lk = lam + (size_t)k * nb;
    herm_eig(nb, hk, lk, Wk);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx su = 0, sv = 0;
        for (int c = 0; c < nb; ++c) {
          cplx wc = Wk[a * nb + c] * conj(Wk[b * nb + c]);
          su += wc * cexp(-IU * lk[c] * dt);
          sv += wc * phi_v(lk[c], dt);
        }
        U[(size_t)k * nb2 + a * nb + b] = su;
        V[(size_t)k * nb2 + a * nb + b] = sv;
      }
  }
}

/*
 * Row n from row n-1 (Algorithm 1, "solve Eq. 5"): for j < n and x in {<,>}
 *   G^x(n,j) = U G^x(n-1,j) + V Ibar^x(j),
 *   Ibar = (1 - theta) I_{n-1}(j) + theta I_n(j);
 * time diagonal with Sbar = (1-theta) S_{n-1} + theta S_n, S_m = I^<(m,m) + h.c.:
 *   G^<(n,n) = U G^<(n-1,n-1) U^+ - i W [(W^+ Sbar W) o D] W^+,
 *   G^>(n,n) = G^<(n,n) - i.
 * Gprev*: blocks j = 0..n-1 of row n-1 (incl. its diagonal); Ip*: I row n-1
 * (n blocks); Ic*: I row n (n+1 blocks, may be NULL when theta == 0);
 * out*: n+1 blocks of row n. All blocks [k][a][b].
 */
void orc_update_row(int nb, int nk, int n, double dt, double theta, const double *U_,
                    const double *V_, const double *W_, const double *lam, const double *Gpl_,
                    const double *Gpg_, const double *Ipl_, const double *Ipg_,
                    const double *Icl_, const double *Icg_, double *outl_, double *outg_) {
  const cplx *U = (const cplx *)U_, *V = (const cplx *)V_, *W = (const cplx *)W_;
  const cplx *Gpl = (const cplx *)Gpl_, *Gpg = (const cplx *)Gpg_;
  const cplx *Ipl = (const cplx *)Ipl_, *Ipg = (const cplx *)Ipg_;
  const cplx *Icl = (const cplx *)Icl_, *Icg = (const cplx *)Icg_;
  cplx *outl = (cplx *)outl_, *outg = (cplx *)outg_;
  size_t blk = (size_t)nk * nb * nb;
  int nb2 = nb * nb;
#pragma omp parallel for collapse(2)
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < nk; ++k) {
      size_t o = j * blk + (size_t)k * nb2;
      const cplx *Uk = U + (size_t)k * nb2, *Vk = V + (size_t)k * nb2;
      cplx ib[MAXNB * MAXNB], t1[MAXNB * MAXNB], t2[MAXNB * MAXNB];
      for (int x = 0; x < 2; ++x) {
        const cplx *gp = (x == 0 ? Gpl : Gpg) + o;
        const cplx *ip = (x == 0 ? Ipl : Ipg) + o;
        const cplx *ic = theta != 0.0 ? (x == 0 ? Icl : Icg) + o : NULL;
        for (int e = 0; e < nb2; ++e) ib[e] = (1.0 - theta) * ip[e] + (ic ? theta * ic[e] : 0.0);
        mat_mul(nb, Uk, gp, t1);
        mat_mul(nb, Vk, ib, t2);
        cplx *dst = (x == 0 ? outl : outg) + o;
        for (int e = 0; e < nb2; ++e) dst[e] = t1[e] + t2[e];
      }
    }
#pragma omp parallel for
  for (int k = 0; k < nk; ++k) {
    const cplx *Uk = U + (size_t)k * nb2, *Wk = W + (size_t)k * nb2;
    const double *lk = lam + (size_t)k * nb;
    cplx S[MAXNB * MAXNB], T[MAXNB * MAXNB], T2[MAXNB * MAXNB], G[MAXNB * MAXNB];
    const cplx *ipd = Ipl + (size_t)(n - 1) * blk + (size_t)k * nb2;
    const cplx *icd = theta != 0.0 ? Icl + (size_t)n * blk + (size_t)k * nb2 : NULL;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx s = (1.0 - theta) * (ipd[a * nb + b] + conj(ipd[b * nb + a]));
        if (icd) s += theta * (icd[a * nb + b] + conj(icd[b * nb + a]));
        S[a * nb + b] = s;
      }
    /* W^+ S W, Hadamard with D, back-transform */
    mat_adj_mul(nb, Wk, S, T);
    mat_mul(nb, T, Wk, T2);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) T2[a * nb + b] *= phi_d(lk[a] - lk[b], dt);
    mat_mul(nb, Wk, T2, T);
    mat_mul_adj(nb, T, Wk, T2); /* W (.) W^+ */
    const cplx *gd = Gpl + (size_t)(n - 1) * blk + (size_t)k * nb2;
    mat_mul(nb, Uk, gd, T);
    mat_mul_adj(nb, T, Uk, G); /* U G U^+ */
    cplx *dl = outl + (size_t)n * blk + (size_t)k * nb2, *dgp = outg + (size_t)n * blk + (size_t)k * nb2;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx g = G[a * nb + b] - IU * T2[a * nb + b];
        dl[a * nb + b] = g;
        dgp[a * nb + b] = g - (a == b ? IU : 0.0);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* the stateful stepper                                                      */
/* ------------------------------------------------------------------------ */

typedef struct orc {
  int nb, dim, L0, L1, nk, nt_max, n_corr, hf, paper_shift;
  double corr_tol; /* Algorithm 1's epsilon (0: always n_corr passes) */
  int quad;        /* collision-integral quadrature: 0 trapezoid, 1 Gregory */
  int *iters;      /* corrector passes run at each step */
  double dt, beta, mu;
  int nhop;
  int *hopR;
  cplx *hopT;
  int nU;
  double *Useq;
  double v[MAXNB * MAXNB];
  int nA;
  double *Aseq;
  double dir[2];
  int nE;    /* dipole field samples E_i (Eq. 4), coupling M [nb][nb] */
  double *Eseq;
  cplx dipM[MAXNB * MAXNB];
  int n; /* last completed row, -1 before reset */
  size_t blk;
  cplx *Hl, *Hg;
  cplx *Ipl, *Ipg, *Icl, *Icg;
  cplx *Sl, *Sg;
  cplx *rho; /* local density per row, [(nt_max+1)][nb][nb] */
  cplx *h, *Uk, *Vk, *Wk;
  double *lam;
  double *obs; /* [(nt_max+1)][6] */
  double *nkb; /* [(nt_max+1)][nk][nb] */
  /* full-grid mode (orc_enable_full): the strict upper triangle G(j, i),
   * j < i, kept as its own column at index tri(i, j) and propagated with the
   * right-hand equation; right-form collision rows I_R(j, n) and the column
   * self-energy Sigma(l, n) */
  int full;
  int right_limit_printed; /* 1: the second integral of I_R up to t as printed */
  cplx *Cl, *Cg;
  cplx *Rpl, *Rpg, *Rcl, *Rcg;
  cplx *Tl, *Tg;
} orc;

orc *orc_create(int nb, int dim, int L0, int L1, int nt_max, double dt, double beta, double mu,
                int n_corr, int hf, int paper_shift) {
  if (nb < 1 || nb > MAXNB || L0 < 1 || L1 < 1 || nt_max < 1 || dt <= 0 || n_corr < 0) return NULL;
  orc *s = calloc(1, sizeof(orc));
  s->nb = nb;
  s->dim = dim;
  s->L0 = L0;
  s->L1 = L1;
  s->nk = L0 * L1;
  s->nt_max = nt_max;
  s->dt = dt;
  s->beta = beta;
  s->mu = mu;
  s->n_corr = n_corr;
  s->hf = hf;
  s->paper_shift = paper_shift;
  s->n = -1;
  s->blk = (size_t)s->nk * nb * nb;
  size_t ntri = tri(nt_max, nt_max) + 1;
  s->Hl = malloc(sizeof(cplx) * ntri * s->blk);
  s->Hg = malloc(sizeof(cplx) * ntri * s->blk);
  size_t rowb = sizeof(cplx) * (size_t)(nt_max + 1) * s->blk;
  s->Ipl = malloc(rowb);
  s->Ipg = malloc(rowb);
  s->Icl = malloc(rowb);
  s->Icg = malloc(rowb);
  s->Sl = malloc(rowb);
  s->Sg = malloc(rowb);
  s->rho = calloc((size_t)(nt_max + 1) * nb * nb, sizeof(cplx));
  s->h = malloc(sizeof(cplx) * s->blk);
  s->Uk = malloc(sizeof(cplx) * s->blk);
  s->Vk = malloc(sizeof(cplx) * s->blk);
  s->Wk = malloc(sizeof(cplx) * s->blk);
  s->lam = malloc(sizeof(double) * s->nk * nb);
  s->obs = calloc((size_t)(nt_max + 1) * 6, sizeof(double));
  s->nkb = calloc((size_t)(nt_max + 1) * s->nk * nb, sizeof(double));
  s->iters = calloc((size_t)(nt_max + 1), sizeof(int));
  if (!s->Hl || !s->Hg || !s->Ipl || !s->Ipg || !s->Icl || !s->Icg || !s->Sl || !s->Sg) {
    free(s->Hl); free(s->Hg); free(s->Ipl); free(s->Ipg); free(s->Icl); free(s->Icg);
    free(s->Sl); free(s->Sg); free(s->rho); free(s->h); free(s->Uk); free(s->Vk);
    free(s->Wk); free(s->lam); free(s->obs); free(s->nkb); free(s);
    return NULL;
  }
  for (int a = 0; a < nb; ++a)
    for (int b = 0; b < nb; ++b) s->v[a * nb + b] = (a == b) ? 0.0 : 1.0;
  s->nU = 1;
  s->Useq = calloc(1, sizeof(double));
  s->dir[0] = 1.0;
  return s;
}

void orc_destroy(orc *s) {
  if (!s) return;
  free(s->hopR); free(s->hopT); free(s->Useq); free(s->Aseq); free(s->Eseq);
  free(s->Hl); free(s->Hg); free(s->Ipl); free(s->Ipg); free(s->Icl); free(s->Icg);
  free(s->Sl); free(s->Sg); free(s->rho); free(s->h); free(s->Uk); free(s->Vk);
  free(s->Wk); free(s->lam); free(s->obs); free(s->nkb); free(s->iters);
  free(s->Cl); free(s->Cg); free(s->Rpl); free(s->Rpg); free(s->Rcl); free(s->Rcg);
  free(s->Tl); free(s->Tg);
  free(s);
}

int orc_set_hamiltonian(orc *s, int nhop, const int *R, const double *t) {
  free(s->hopR);
  free(s->hopT);
  s->nhop = nhop;
  s->hopR = malloc(sizeof(int) * 2 * nhop);
  s->hopT = malloc(sizeof(cplx) * nhop * s->nb * s->nb);
  memcpy(s->hopR, R, sizeof(int) * 2 * nhop);
  memcpy(s->hopT, t, sizeof(cplx) * nhop * s->nb * s->nb);
  return 0;
}

/* v must be symmetric: the interaction U sum_ab v_ab n_a n_b of Eq. 2 is, and
 * an asymmetric v would make the mean field non-Hermitian (the propagators
 * below diagonalise h as a Hermitian matrix). */
int orc_set_interaction(orc *s, int len, const double *U, const double *v) {
  if (len != 1 && len < s->nt_max + 1) return -1;
  if (v)
    for (int a = 0; a < s->nb; ++a)
      for (int b = a + 1; b < s->nb; ++b) {
        double x = v[a * s->nb + b], y = v[b * s->nb + a];
        if (fabs(x - y) > 1e-12 * (fabs(x) + fabs(y))) return -2;
      }
  free(s->Useq);
  s->nU = len;
  s->Useq = malloc(sizeof(double) * len);
  memcpy(s->Useq, U, sizeof(double) * len);
  if (v) memcpy(s->v, v, sizeof(double) * s->nb * s->nb);
  return 0;
}

int orc_set_drive(orc *s, int len, const double *A, const double *dir) {
  free(s->Aseq);
  s->Aseq = NULL;
  s->nA = 0;
  if (A && len > 0) {
    s->nA = len;
    s->Aseq = malloc(sizeof(double) * len);
    memcpy(s->Aseq, A, sizeof(double) * len);
  }
  if (dir) {
    s->dir[0] = dir[0];
    s->dir[1] = s->dim == 2 ? dir[1] : 0.0;
  }
  return 0;
}

/* dipole drive of Eq. 4 in the length gauge: h gains E_i M during step i */
int orc_set_dipole(orc *s, int len, const double *E, const double *M) {
  free(s->Eseq);
  s->Eseq = NULL;
  s->nE = 0;
  if (E && len > 0) {
    s->nE = len;
    s->Eseq = malloc(sizeof(double) * len);
    memcpy(s->Eseq, E, sizeof(double) * len);
    memcpy(s->dipM, M, sizeof(cplx) * s->nb * s->nb);
  }
  return 0;
}

static double U_at(const orc *s, int i) { return s->nU == 1 ? s->Useq[0] : s->Useq[i]; }

/* Peierls sample A_i = A(t_{i+1/2}); indices clamped to the sampled range */
static double A_at(const orc *s, int i) {
  if (s->nA == 0) return 0.0;
  if (i < 0) i = 0;
  if (i >= s->nA) i = s->nA - 1;
  return s->Aseq[i];
}

/* h0_ab(k - A d) = sum_R t_ab(R) exp(i (k - A d).R) */
static void h0_at(const orc *s, int k, double A, cplx *out) {
  int nb2 = s->nb * s->nb;
  int k0 = k / s->L1, k1 = k % s->L1;
  for (int e = 0; e < nb2; ++e) out[e] = 0;
  for (int r = 0; r < s->nhop; ++r) {
    int R0 = s->hopR[2 * r], R1 = s->hopR[2 * r + 1];
    double th = 2.0 * M_PI * ((double)k0 * R0 / s->L0 + (double)k1 * R1 / s->L1) -
                A * (s->dir[0] * R0 + s->dir[1] * R1);
    cplx ph = cexp(IU * th);
    for (int e = 0; e < nb2; ++e) out[e] += s->hopT[(size_t)r * nb2 + e] * ph;
  }
}

/* Hartree-Fock mean field: S_jm = U (delta_jm sum_a v_ja rho_aa - v_jm rho_jm) */
static void hf_field(const orc *s, const cplx *rho, double U, cplx *out) {
  int nb = s->nb;
  for (int j = 0; j < nb; ++j)
    for (int m = 0; m < nb; ++m) {
      cplx x = -s->v[j * nb + m] * rho[j * nb + m];
      if (j == m)
        for (int a = 0; a < nb; ++a) x += s->v[j * nb + a] * rho[a * nb + a];
      out[j * nb + m] = U * x;
    }
}

/* local density rho_loc = (1/n_k) sum_k (-i) G^<(k; n, n) */
static void local_density(const orc *s, int n, cplx *out) {
  int nb2 = s->nb * s->nb;
  const cplx *g = s->Hl + tri(n, n) * s->blk;
  for (int e = 0; e < nb2; ++e) out[e] = 0;
  for (int k = 0; k < s->nk; ++k)
    for (int e = 0; e < nb2; ++e) out[e] += -IU * g[(size_t)k * nb2 + e];
  for (int e = 0; e < nb2; ++e) out[e] /= s->nk;
}

/* h(k) for the step t_{n-1} -> t_n: Peierls h0 at A_{n-1}, mean field from
 * the given local density and U at the step midpoint, the -U n_c term. */
static void build_h_and_props(orc *s, int n, const cplx *rho_mid) {
  int nb = s->nb, nb2 = nb * nb;
  double Umid = 0.5 * (U_at(s, n - 1) + U_at(s, n));
  cplx hf[MAXNB * MAXNB];
  for (int e = 0; e < nb2; ++e) hf[e] = 0;
  if (s->hf) hf_field(s, rho_mid, Umid, hf);
  for (int k = 0; k < s->nk; ++k) {
    cplx *hk = s->h + (size_t)k * nb2;
    h0_at(s, k, A_at(s, n - 1), hk);
    for (int e = 0; e < nb2; ++e) hk[e] += hf[e];
    if (s->paper_shift) hk[(nb - 1) * nb + (nb - 1)] -= Umid;
    if (n - 1 < s->nE)
      for (int e = 0; e < nb2; ++e) hk[e] += s->Eseq[n - 1] * s->dipM[e];
  }
  orc_propagators(nb, s->nk, s->dt, (const double *)s->h, (double *)s->Uk, (double *)s->Vk,
                  (double *)s->Wk, s->lam);
}

/* Sigma row n (all l <= n) and the collision row n into Icl/Icg */
static void evaluate_row(orc *s, int n) {
  size_t blk = s->blk;
#pragma omp parallel for schedule(dynamic)
  for (int l = 0; l <= n; ++l) {
    double UnUl = U_at(s, n) * U_at(s, l);
    orc_sigma_pair(s->nb, s->L0, s->L1, s->v, UnUl, (const double *)(s->Hl + tri(n, l) * blk),
                   (const double *)(s->Hg + tri(n, l) * blk), (double *)(s->Sl + l * blk),
                   (double *)(s->Sg + l * blk));
  }
  orc_collision_row_q(s->nb, s->nk, n, s->dt, s->quad, (const double *)s->Hl, (const double *)s->Hg,
                      (const double *)s->Sl, (const double *)s->Sg, (double *)s->Icl,
                      (double *)s->Icg);
}

/* One evaluation of row n as orc_step performs it (the Sigma row from the
 * triangle's row n, then the collision row), on caller arrays: Hl, Hg the
 * triangle with rows 0..n, S* and I* (n+1) blocks each, all [k][a][b]. U(t)
 * is the constant U. Used to time the oracle at sampled rows of a long
 * trajectory without running the steps before them. */
void orc_evaluate_row_on(int nb, int L0, int L1, const double *v, double U, int n, double dt,
                         const double *Hl_, const double *Hg_, double *Sl_, double *Sg_, double *Il_,
                         double *Ig_) {
  const cplx *Hl = (const cplx *)Hl_, *Hg = (const cplx *)Hg_;
  cplx *Sl = (cplx *)Sl_, *Sg = (cplx *)Sg_;
  size_t blk = (size_t)L0 * L1 * nb * nb;
#pragma omp parallel for schedule(dynamic)
  for (int l = 0; l <= n; ++l)
    orc_sigma_pair(nb, L0, L1, v, U * U, (const double *)(Hl + tri(n, l) * blk),
                   (const double *)(Hg + tri(n, l) * blk), (double *)(Sl + l * blk), (double *)(Sg + l * blk));
  collision_left(nb, L0 * L1, n, dt, 0, Hl, Hg, NULL, NULL, Sl, Sg, (cplx *)Il_, (cplx *)Ig_);
}

static void update(orc *s, int n, double theta) {
  size_t blk = s->blk;
  orc_update_row(s->nb, s->nk, n, s->dt, theta, (const double *)s->Uk, (const double *)s->Vk,
                 (const double *)s->Wk, s->lam, (const double *)(s->Hl + tri(n - 1, 0) * blk),
                 (const double *)(s->Hg + tri(n - 1, 0) * blk), (const double *)s->Ipl,
                 (const double *)s->Ipg, (const double *)s->Icl, (const double *)s->Icg,
                 (double *)(s->Hl + tri(n, 0) * blk), (double *)(s->Hg + tri(n, 0) * blk));
}

/* equal-time observables at row n (uses the final I row of step n in Icl) */
static void observables(orc *s, int n) {
  int nb = s->nb, nb2 = nb * nb, nk = s->nk;
  const cplx *g = s->Hl + tri(n, n) * s->blk;
  const cplx *il = s->Icl + (size_t)n * s->blk;
  double Abar = 0.5 * (A_at(s, n - 1) + A_at(s, n));
  double N = 0, Ekin = 0, Ecorr = 0;
  cplx h0[MAXNB * MAXNB];
  for (int k = 0; k < nk; ++k) {
    const cplx *gk = g + (size_t)k * nb2;
    h0_at(s, k, Abar, h0);
    for (int a = 0; a < nb; ++a) {
      s->nkb[((size_t)n * nk + k) * nb + a] = creal(-IU * gk[a * nb + a]);
      N += creal(-IU * gk[a * nb + a]);
      for (int b = 0; b < nb; ++b) Ekin += creal(h0[a * nb + b] * (-IU) * gk[b * nb + a]);
      Ecorr += creal(-IU * il[(size_t)k * nb2 + a * nb + a]);
    }
  }
  const cplx *rl = s->rho + (size_t)n * nb2;
  double Ehf = 0, Esh = 0, Un = U_at(s, n);
  if (s->hf) {
    cplx hf[MAXNB * MAXNB];
    hf_field(s, rl, Un, hf);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) Ehf += 0.5 * creal(hf[a * nb + b] * rl[b * nb + a]);
  }
  if (s->paper_shift) Esh = -Un * creal(rl[(nb - 1) * nb + (nb - 1)]);
  double *o = s->obs + (size_t)n * 6;
  o[0] = N / nk;
  o[1] = Ekin / nk;
  o[2] = Ehf;
  o[3] = 0.5 * Ecorr / nk;
  o[4] = Esh;
  o[5] = o[1] + o[2] + o[3] + o[4];
}

/* ------------------------------------------------------------------------ */
/* full two-time grid (tiny grids only)                                      */
/* ------------------------------------------------------------------------ */
/*
 * A second way through the same equations that never uses the adjoint
 * symmetry G^x(t,t')^+ = -G^x(t',t): the row G(t_n, t_j) is advanced with the
 * left equation i d/dt G = h G + I_L as in orc_step, and the column
 * G(t_j, t_n), j < n, with the right equation -i d/dt' G = G h + I_R, whose
 * collision integral is Eq. 6 as printed (the G * Sigma form):
 *   I_R^x(j, n) = sum_{l<=j} w^(j)_l [G^> - G^<](j,l) Sigma^x(l,n)
 *               + sum_{l<=L} w^(L)_l G^x(j,l) [Sigma^< - Sigma^>](l,n),
 * L = n (the second upper limit read as t'), or L = j (the limit t as printed,
 * right_limit_printed = 1). Every block with l < j comes from the column
 * store; Sigma(n, l) and Sigma(l, n) are both summed from Eq. 7 with the
 * stored G(n, l) and G(l, n). The exponential step of the right equation is
 * G(j, n) = G(j, n-1) U^+ + Ibar_R(j) V^+ (the adjoint of the row step), and
 * the time diagonal i dG(t,t)/dt = [h, G] + I_L(t,t) - I_R(t,t) takes the
 * divided-difference form with Sbar = Ibar_L(n,n) - Ibar_R(n,n).
 */
static const cplx *grid_block(const orc *s, const cplx *H, const cplx *C, int l, int j) {
  return l >= j ? H + tri(l, j) * s->blk : C + tri(j, l) * s->blk;
}

int orc_enable_full(orc *s, int right_limit_printed) {
  if (s->n > 0) return -4;
  size_t ntri = tri(s->nt_max, s->nt_max) + 1;
  size_t rowb = sizeof(cplx) * (size_t)(s->nt_max + 1) * s->blk;
  if (!s->full) {
    s->Cl = calloc(ntri * s->blk, sizeof(cplx));
    s->Cg = calloc(ntri * s->blk, sizeof(cplx));
    s->Rpl = calloc(1, rowb);
    s->Rpg = calloc(1, rowb);
    s->Rcl = calloc(1, rowb);
    s->Rcg = calloc(1, rowb);
    s->Tl = calloc(1, rowb);
    s->Tg = calloc(1, rowb);
    if (!s->Cl || !s->Cg || !s->Rpl || !s->Rpg || !s->Rcl || !s->Rcg || !s->Tl || !s->Tg) return -2;
  }
  s->full = 1;
  s->right_limit_printed = right_limit_printed ? 1 : 0;
  return 0;
}

/* Sigma(n, l) into S* and Sigma(l, n) into T*, l = 0..n, each from Eq. 7 */
static void full_sigma(orc *s, int n) {
  mesh m = {s->L0, s->L1};
  size_t blk = s->blk;
#pragma omp parallel for schedule(dynamic)
  for (int l = 0; l <= n; ++l) {
    double UU = U_at(s, n) * U_at(s, l);
    const cplx *fl = grid_block(s, s->Hl, s->Cl, n, l), *fg = grid_block(s, s->Hg, s->Cg, n, l);
    const cplx *bl = grid_block(s, s->Hl, s->Cl, l, n), *bg = grid_block(s, s->Hg, s->Cg, l, n);
    sigma_eq7(s->nb, m, s->v, UU, fl, bg, s->Sl + l * blk);
    sigma_eq7(s->nb, m, s->v, UU, fg, bl, s->Sg + l * blk);
    sigma_eq7(s->nb, m, s->v, UU, bl, fg, s->Tl + l * blk);
    sigma_eq7(s->nb, m, s->v, UU, bg, fl, s->Tg + l * blk);
  }
}

/* I_R^x(j, n), j = 0..n, into Rcl / Rcg (Eq. 6 as printed, G * Sigma) */
static void full_collision_right(orc *s, int n) {
  int nb = s->nb, nb2 = nb * nb, nk = s->nk;
  size_t blk = s->blk;
#pragma omp parallel for collapse(2)
  for (int j = 0; j <= n; ++j)
    for (int k = 0; k < nk; ++k) {
      cplx d[MAXNB * MAXNB], t[MAXNB * MAXNB], accl[MAXNB * MAXNB], accg[MAXNB * MAXNB];
      for (int e = 0; e < nb2; ++e) accl[e] = accg[e] = 0;
      for (int l = 0; l <= j; ++l) { /* retarded G on [0, t_j] */
        const cplx *gl = grid_block(s, s->Hl, s->Cl, j, l) + (size_t)k * nb2;
        const cplx *gg = grid_block(s, s->Hg, s->Cg, j, l) + (size_t)k * nb2;
        double w = quad_w(s->quad, j, l, s->dt);
        for (int e = 0; e < nb2; ++e) d[e] = w * (gg[e] - gl[e]);
        mat_mul(nb, d, s->Tl + l * blk + (size_t)k * nb2, t);
        for (int e = 0; e < nb2; ++e) accl[e] += t[e];
        mat_mul(nb, d, s->Tg + l * blk + (size_t)k * nb2, t);
        for (int e = 0; e < nb2; ++e) accg[e] += t[e];
      }
      int L = s->right_limit_printed ? j : n;
      for (int l = 0; l <= L; ++l) { /* advanced Sigma on [0, t_L] */
        const cplx *tl = s->Tl + l * blk + (size_t)k * nb2, *tg = s->Tg + l * blk + (size_t)k * nb2;
        double w = quad_w(s->quad, L, l, s->dt);
        for (int e = 0; e < nb2; ++e) d[e] = w * (tl[e] - tg[e]);
        mat_mul(nb, grid_block(s, s->Hl, s->Cl, j, l) + (size_t)k * nb2, d, t);
        for (int e = 0; e < nb2; ++e) accl[e] += t[e];
        mat_mul(nb, grid_block(s, s->Hg, s->Cg, j, l) + (size_t)k * nb2, d, t);
        for (int e = 0; e < nb2; ++e) accg[e] += t[e];
      }
      memcpy(s->Rcl + j * blk + (size_t)k * nb2, accl, sizeof(cplx) * nb2);
      memcpy(s->Rcg + j * blk + (size_t)k * nb2, accg, sizeof(cplx) * nb2);
    }
}

static void full_evaluate(orc *s, int n) {
  full_sigma(s, n);
  collision_left(s->nb, s->nk, n, s->dt, s->quad, s->Hl, s->Hg, s->Cl, s->Cg, s->Sl, s->Sg, s->Icl, s->Icg);
  full_collision_right(s, n);
}

/* row n (left equation), column n (right equation) and the time diagonal */
static void full_update(orc *s, int n, double theta) {
  int nb = s->nb, nb2 = nb * nb, nk = s->nk;
  size_t blk = s->blk;
  /* rows j < n exactly as in triangle mode; its diagonal is replaced below */
  update(s, n, theta);
#pragma omp parallel for collapse(2)
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < nk; ++k) {
      const cplx *Uk = s->Uk + (size_t)k * nb2, *Vk = s->Vk + (size_t)k * nb2;
      cplx ib[MAXNB * MAXNB], t1[MAXNB * MAXNB], t2[MAXNB * MAXNB];
      for (int x = 0; x < 2; ++x) {
        const cplx *gp = grid_block(s, x ? s->Hg : s->Hl, x ? s->Cg : s->Cl, j, n - 1) + (size_t)k * nb2;
        const cplx *rp = (x ? s->Rpg : s->Rpl) + j * blk + (size_t)k * nb2;
        const cplx *rc = (x ? s->Rcg : s->Rcl) + j * blk + (size_t)k * nb2;
        for (int e = 0; e < nb2; ++e) ib[e] = (1.0 - theta) * rp[e] + (theta != 0.0 ? theta * rc[e] : 0.0);
        mat_mul_adj(nb, gp, Uk, t1);
        mat_mul_adj(nb, ib, Vk, t2);
        cplx *dst = (x ? s->Cg : s->Cl) + tri(n, j) * blk + (size_t)k * nb2;
        for (int e = 0; e < nb2; ++e) dst[e] = t1[e] + t2[e];
      }
    }
  for (int k = 0; k < nk; ++k) {
    const cplx *Uk = s->Uk + (size_t)k * nb2, *Wk = s->Wk + (size_t)k * nb2;
    const double *lk = s->lam + (size_t)k * nb;
    cplx S[MAXNB * MAXNB], T[MAXNB * MAXNB], T2[MAXNB * MAXNB], G[MAXNB * MAXNB];
    size_t op = (size_t)(n - 1) * blk + (size_t)k * nb2, oc = (size_t)n * blk + (size_t)k * nb2;
    for (int e = 0; e < nb2; ++e) {
      S[e] = (1.0 - theta) * (s->Ipl[op + e] - s->Rpl[op + e]);
      if (theta != 0.0) S[e] += theta * (s->Icl[oc + e] - s->Rcl[oc + e]);
    }
    mat_adj_mul(nb, Wk, S, T);
    mat_mul(nb, T, Wk, T2);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) T2[a * nb + b] *= phi_d(lk[a] - lk[b], s->dt);
    mat_mul(nb, Wk, T2, T);
    mat_mul_adj(nb, T, Wk, T2);
    mat_mul(nb, Uk, s->Hl + tri(n - 1, n - 1) * blk + (size_t)k * nb2, T);
    mat_mul_adj(nb, T, Uk, G);
    cplx *dl = s->Hl + tri(n, n) * blk + (size_t)k * nb2, *dg = s->Hg + tri(n, n) * blk + (size_t)k * nb2;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx g = G[a * nb + b] - IU * T2[a * nb + b];
        dl[a * nb + b] = g;
        dg[a * nb + b] = g - (a == b ? IU : 0.0);
      }
  }
}

/* one step of Algorithm 1 on the full grid (fixed corrector count) */
static void full_step(orc *s) {
  int nb2 = s->nb * s->nb, n = s->n + 1;
  cplx mid[MAXNB * MAXNB], cur[MAXNB * MAXNB];
  const cplx *r1 = s->rho + (size_t)(n - 1) * nb2;
  const cplx *r2 = s->rho + (size_t)(n >= 2 ? n - 2 : 0) * nb2;
  for (int e = 0; e < nb2; ++e) mid[e] = n >= 2 ? 1.5 * r1[e] - 0.5 * r2[e] : r1[e];
  build_h_and_props(s, n, mid);
  full_update(s, n, 0.0);
  s->iters[n] = 0;
  for (int c = 0; c < s->n_corr; ++c) {
    local_density(s, n, cur);
    for (int e = 0; e < nb2; ++e) mid[e] = 0.5 * (r1[e] + cur[e]);
    build_h_and_props(s, n, mid);
    full_evaluate(s, n);
    full_update(s, n, 0.5);
    s->iters[n] += 1;
  }
  full_evaluate(s, n);
  local_density(s, n, s->rho + (size_t)n * nb2);
  s->n = n;
  observables(s, n);
  cplx *t;
  t = s->Ipl; s->Ipl = s->Icl; s->Icl = t;
  t = s->Ipg; s->Ipg = s->Icg; s->Icg = t;
  t = s->Rpl; s->Rpl = s->Rcl; s->Rcl = t;
  t = s->Rpg; s->Rpg = s->Rcg; s->Rcg = t;
}

/* t = 0: uncorrelated Fermi state of the field-free h0, G^<(0,0) = i f(h0) */
int orc_reset(orc *s) {
  int nb = s->nb, nb2 = nb * nb;
  if (s->nhop == 0) return -1;
  for (int k = 0; k < s->nk; ++k) {
    cplx h0[MAXNB * MAXNB], W[MAXNB * MAXNB];
    double lam[MAXNB];
    h0_at(s, k, 0.0, h0);
    herm_eig(nb, h0, lam, W);
    cplx *gl = s->Hl + (size_t)k * nb2, *gg = s->Hg + (size_t)k * nb2;
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        cplx r = 0;
        for (int c = 0; c < nb; ++c) r += W[a * nb + c] * fermi(lam[c], s->beta, s->mu) * conj(W[b * nb + c]);
        gl[a * nb + b] = IU * r;
        gg[a * nb + b] = IU * r - (a == b ? IU : 0.0);
      }
  }
  memset(s->Ipl, 0, sizeof(cplx) * s->blk);
  memset(s->Ipg, 0, sizeof(cplx) * s->blk);
  memset(s->Icl, 0, sizeof(cplx) * s->blk);
  memset(s->Icg, 0, sizeof(cplx) * s->blk);
  if (s->full) {
    memset(s->Rpl, 0, sizeof(cplx) * s->blk);
    memset(s->Rpg, 0, sizeof(cplx) * s->blk);
    memset(s->Rcl, 0, sizeof(cplx) * s->blk);
    memset(s->Rcg, 0, sizeof(cplx) * s->blk);
  }
  s->n = 0;
  local_density(s, 0, s->rho);
  observables(s, 0);
  return 0;
}

/* Algorithm 1 for rows n = s->n + 1, ... : P(EC)^n_corr E */
int orc_step(orc *s, int nsteps) {
  int nb2 = s->nb * s->nb;
  if (s->n < 0) return -4;
  if (s->n + nsteps > s->nt_max) return -4;
  if (s->full) {
    if (s->corr_tol > 0.0) return -1; /* the full-grid mode runs a fixed corrector count */
    for (int it = 0; it < nsteps; ++it) full_step(s);
    return 0;
  }
  for (int it = 0; it < nsteps; ++it) {
    int n = s->n + 1;
    cplx mid[MAXNB * MAXNB], cur[MAXNB * MAXNB];
    const cplx *r1 = s->rho + (size_t)(n - 1) * nb2;
    const cplx *r2 = s->rho + (size_t)(n >= 2 ? n - 2 : 0) * nb2;
    for (int e = 0; e < nb2; ++e) mid[e] = n >= 2 ? 1.5 * r1[e] - 0.5 * r2[e] : r1[e];
    build_h_and_props(s, n, mid);
    update(s, n, 0.0); /* predictor: Ibar = I_{n-1} */
    /* the corrector loop of Algorithm 1: at most n_corr passes; with
     * corr_tol > 0 it ends once the largest change of the new G^< row,
     * max_{j,k,a,b} |G^< - G_0^<| (the reading of the algorithm's norm), is
     * <= corr_tol */
    const size_t rowlen = (size_t)(n + 1) * s->blk;
    cplx *G0 = s->corr_tol > 0.0 ? malloc(sizeof(cplx) * rowlen) : NULL;
    s->iters[n] = 0;
    for (int c = 0; c < s->n_corr; ++c) {
      if (G0) memcpy(G0, s->Hl + tri(n, 0) * s->blk, sizeof(cplx) * rowlen);
      local_density(s, n, cur);
      for (int e = 0; e < nb2; ++e) mid[e] = 0.5 * (r1[e] + cur[e]);
      build_h_and_props(s, n, mid);
      evaluate_row(s, n);
      update(s, n, 0.5);
      s->iters[n] += 1;
      if (G0) {
        double d = 0.0;
        const cplx *G = s->Hl + tri(n, 0) * s->blk;
        for (size_t q = 0; q < rowlen; ++q) {
          double a = cabs(G[q] - G0[q]);
          if (a > d) d = a;
        }
        if (d <= s->corr_tol) break;
      }
    }
    free(G0);
    evaluate_row(s, n); /* final evaluation: I_n for the next predictor */
    local_density(s, n, s->rho + (size_t)n * nb2);
    s->n = n;
    observables(s, n);
    cplx *t;
    t = s->Ipl; s->Ipl = s->Icl; s->Icl = t;
    t = s->Ipg; s->Ipg = s->Icg; s->Icg = t;
  }
  return 0;
}

int orc_current(const orc *s) { return s->n; }

void orc_set_corr_tol(orc *s, double tol) { s->corr_tol = tol > 0.0 ? tol : 0.0; }

void orc_set_quadrature(orc *s, int quad) { s->quad = quad == 1 ? 1 : 0; }

/* corrector passes run at steps 0..n */
int orc_get_iters(const orc *s, int *out) {
  if (s->n < 0) return -1;
  memcpy(out, s->iters, sizeof(int) * (size_t)(s->n + 1));
  return 0;
}

/* G^x(i, j) for any i, j <= n (x = 0: lesser, 1: greater), [k][a][b]; for
 * i < j in full-grid mode the propagated column, otherwise -G^x(j, i)^+ */
int orc_get_block(const orc *s, int i, int j, int which, double *out) {
  if (i < 0 || j < 0 || i > s->n || j > s->n) return -1;
  const cplx *H = which == 0 ? s->Hl : s->Hg;
  const cplx *C = s->full ? (which == 0 ? s->Cl : s->Cg) : NULL;
  for (int k = 0; k < s->nk; ++k)
    fetch_grid(s->nb, s->nk, H, C, i, j, k, (cplx *)out + (size_t)k * s->nb * s->nb);
  return 0;
}

/* the stored I row of the last completed step, blocks j = 0..n */
int orc_get_irow(const orc *s, int which, double *out) {
  if (s->n < 0) return -1;
  memcpy(out, which == 0 ? s->Ipl : s->Ipg, sizeof(cplx) * (size_t)(s->n + 1) * s->blk);
  return 0;
}

int orc_observables(const orc *s, int step, double *nkb, double *scalars) {
  if (step < 0 || step > s->n) return -1;
  if (nkb) memcpy(nkb, s->nkb + (size_t)step * s->nk * s->nb, sizeof(double) * s->nk * s->nb);
  if (scalars) memcpy(scalars, s->obs + (size_t)step * 6, sizeof(double) * 6);
  return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
