"""Pin of the oracle-side reference gradient (oracle/gradient.py) on CPU.

At U = 0 the self-energy (order U^2), the mean field and the shift (order U)
vanish, every stage of a step sees the same h, and the collision integrals
are zero. A step is then exactly G(n,n) = P_n G(n-1,n-1) P_n^+ with
P_n = exp(-i dt h_n), h_n = h0(k - A_{n-1} d) + U [hf(mid_n) - shift], so
  dG(N,N)/dA_i: the step i+1 factor varies by the Frechet derivative of exp
                at -i dt h_{i+1} along -i dt dh0/dA,
  dG(N,N)/dU:   every step varies along -i dt [hf(mid_n) - shift], mid_n the
                density the last corrector uses, 0.5 (rho_{n-1} + rho_n)
                (at U = 0 all stages of a step produce the same row).
This is computed here with numpy/scipy only (eigen-solver Fermi state,
scipy.linalg.expm / expm_frechet) and compared with the oracle's
Richardson-extrapolated central differences.
"""
import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from oracle import gradient as og

scipy_linalg = pytest.importorskip("scipy.linalg")


def bare_h(sys, A):
    out = np.zeros((sys.nk, sys.nb, sys.nb), complex)
    dh = np.zeros_like(out)
    for k in range(sys.nk):
        k0, k1 = divmod(k, sys.L[1])
        for R, t in zip(sys.hop_R, sys.hop_T):
            dR = sys.direction[0] * R[0] + (sys.direction[1] * R[1] if sys.dim == 2 else 0.0)
            th = 2 * np.pi * (k0 * R[0] / sys.L[0] + k1 * R[1] / sys.L[1]) - A * dR
            out[k] += t * np.exp(1j * th)
            dh[k] += t * np.exp(1j * th) * (-1j * dR)
    return out, dh


def hf_matrix(sys, rho):
    nb = sys.nb
    x = -sys.v * rho
    x = x + np.diag([sum(sys.v[j, a] * rho[a, a] for a in range(nb)) for j in range(nb)])
    if sys.paper_shift:
        x[nb - 1, nb - 1] -= 1.0
    return x


def closed_form(sys, N, target, per_step_u=False):
    """(L, dL/dA [N], dL/dU) at U = 0 by exact propagators; with per_step_u,
    dL/dU is the list of each step's share (the derivative along U_mid of that
    step)"""
    expm, frechet = scipy_linalg.expm, scipy_linalg.expm_frechet
    h0, _ = bare_h(sys, 0.0)
    G = []
    for k in range(sys.nk):
        w, V = np.linalg.eigh(h0[k])
        f = 1.0 / (np.exp(sys.beta * (w - sys.mu)) + 1.0)
        G.append(1j * (V * f) @ V.conj().T)
    Gs = [np.array(G)]
    Ps, dPs = [], []
    rho = [(-1j * Gs[0]).mean(axis=0)]
    for n in range(1, N + 1):
        h, dh = bare_h(sys, sys.A[n - 1])
        P = np.array([expm(-1j * sys.dt * h[k]) for k in range(sys.nk)])
        Gn = np.einsum('kab,kbc,kdc->kad', P, Gs[-1], P.conj())
        Gs.append(Gn)
        rho.append((-1j * Gn).mean(axis=0))
        Ps.append(P)
        dPs.append((h, dh))
    n_N = np.imag(np.einsum('kbb->kb', Gs[N]))
    L = ((n_N - target) ** 2).sum()
    lam = 2 * (n_N - target)      # dL/dn

    def dL_from(dG):               # dL = sum lam Im dG_bb
        return float((lam * np.imag(np.einsum('kbb->kb', dG))).sum())

    def propagate(n, dGn):         # push a variation of G(n,n) to G(N,N)
        for m in range(n + 1, N + 1):
            P = Ps[m - 1]
            dGn = np.einsum('kab,kbc,kdc->kad', P, dGn, P.conj())
        return dGn

    def step_variation(n, E):      # variation of G(n,n) when h_n varies by E (per k)
        P = Ps[n - 1]
        dP = np.array([frechet(-1j * sys.dt * dPs[n - 1][0][k], -1j * sys.dt * E[k], compute_expm=False)
                       for k in range(sys.nk)])
        Gp = Gs[n - 1]
        return (np.einsum('kab,kbc,kdc->kad', dP, Gp, P.conj())
                + np.einsum('kab,kbc,kdc->kad', P, Gp, dP.conj()))

    gA = np.array([dL_from(propagate(i + 1, step_variation(i + 1, dPs[i][1]))) for i in range(N)])
    gU = []
    for n in range(1, N + 1):
        mid = 0.5 * (rho[n - 1] + rho[n])
        E = np.repeat(hf_matrix(sys, mid)[None], sys.nk, axis=0) if sys.hf else \
            np.repeat(np.diag([0.0] * (sys.nb - 1) + [-float(sys.paper_shift)])[None], sys.nk, axis=0)
        gU.append(dL_from(propagate(n, step_variation(n, E))))
    return L, gA, (gU if per_step_u else sum(gU))


@pytest.mark.parametrize("nb,L,shift", [(2, (4, 1), 1), (3, (2, 2), 0)])
def test_reference_gradient_matches_u0_closed_form(nb, L, shift):
    sys = ki.small_system(nb, L, 6, 0.05, 0.0, seed=11, drive_amp=0.6, paper_shift=shift,
                          band_velocity=0.5)
    N = 6
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    Lc, gA_c, gU_c = closed_form(sys, N, tgt)
    assert abs(og.loss(sys, N, tgt) - Lc) < 1e-12 * max(1.0, Lc)
    gA, gU = og.gradient(sys, N, tgt)
    scale = np.abs(gA_c).max()
    assert np.abs(gA - gA_c).max() < 1e-8 * scale, (gA, gA_c)
    assert abs(gU - gU_c) < 1e-8 * max(abs(gU_c), scale), (gU, gU_c)


def test_reference_gradient_detects_a_dropped_drive_derivative():
    """the closed form is sensitive: scaling dh0/dA by 1/2 breaks the match"""
    sys = ki.small_system(2, (4, 1), 4, 0.05, 0.0, seed=3, drive_amp=0.5, paper_shift=1,
                          band_velocity=0.5)
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    _, gA_c, _ = closed_form(sys, 4, tgt)
    gA, _ = og.gradient(sys, 4, tgt, with_U=False)
    assert np.abs(gA - 0.5 * gA_c).max() > 1e-3 * np.abs(gA_c).max()


def test_reference_gradient_per_u_sample_at_u0():
    """U(t) samples, all zero: step n uses U_mid = (U_{n-1} + U_n) / 2 in its mean
    field and shift, and Sigma (U_n U_l) has no first-order term, so
    dL/dU_i = (g_i + g_{i+1}) / 2 with g_n the step-n share of the closed form"""
    sys = ki.small_system(2, (4, 1), 5, 0.05, 0.0, seed=11, drive_amp=0.6, paper_shift=1,
                          band_velocity=0.5)
    N = 5
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    _, _, g = closed_form(sys, N, tgt, per_step_u=True)
    ref = np.zeros(N + 1)
    for n in range(1, N + 1):
        ref[n - 1] += 0.5 * g[n - 1]
        ref[n] += 0.5 * g[n - 1]
    got = og.gradient_samples(sys, N, tgt, np.zeros(sys.nt + 1))
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max(), (got, ref)
