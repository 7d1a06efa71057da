"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a closed
form, an exact solution computed another way (matrix exponentials, exact
diagonalisation), the literal printed formula (Eq. 7 / Algorithm 2), or a
conservation law / convergence order of the method. A plausible mistake (a
dropped term, a wrong sign, a transposed operand, a wrong weight or limit)
fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import kbe_inputs as ki
import oracle

RNG = np.random.default_rng(20250519)


def h0_of(sys, k, A=0.0):
    """Bare Bloch Hamiltonian from the hopping table (test-side, for closed forms)."""
    k0, k1 = divmod(k, sys.L[1])
    h = np.zeros((sys.nb, sys.nb), complex)
    for R, t in zip(sys.hop_R, sys.hop_T):
        th = 2 * np.pi * (k0 * R[0] / sys.L[0] + k1 * R[1] / sys.L[1]) \
            - A * (sys.direction[0] * R[0] + sys.direction[1] * R[1])
        h += t * np.exp(1j * th)
    return h


def fermi_matrix(h, beta, mu):
    w, V = np.linalg.eigh(h)
    return V @ np.diag(1.0 / (np.exp(beta * (w - mu)) + 1.0)) @ V.conj().T


# --------------------------------------------------------------------------
# Eq. 7: factorised self-energy (Eqs. 8-9 + exchange intermediate) against the
# printed O(n_k^3) sum (Algorithm 2), bar form and generalised pairing form.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nb,L,vmode", [
    (2, (4, 1), "bar"), (2, (8, 1), "bar"), (2, (3, 3), "bar"), (2, (4, 4), "bar"),
    (3, (3, 2), "rand"), (4, (2, 3), "pair"), (2, (5, 1), "pair"),
])
def test_sigma_factorised_equals_literal_eq7(nb, L, vmode):
    nk = L[0] * L[1]
    Gl = ki.random_blocks(RNG, (nk, nb, nb))
    Gg = ki.random_blocks(RNG, (nk, nb, nb))
    if vmode == "bar":
        v, vlit = ki.pair_pattern(nb), None
    elif vmode == "rand":
        v = RNG.uniform(0, 1, (nb, nb))
        v = v + v.T
        vlit = v
    else:
        v = vlit = ki.pair_pattern(nb)
    Sl, Sg = oracle.sigma_pair(nb, L, v, 0.7, Gl, Gg)
    Tl, Tg = oracle.sigma_pair_literal(nb, L, vlit, 0.7, Gl, Gg)
    assert np.abs(Sl - Tl).max() <= 1e-13 * np.abs(Tl).max()
    assert np.abs(Sg - Tg).max() <= 1e-13 * np.abs(Tg).max()


def test_sigma_literal_bar_single_point_by_hand():
    """One output of Eq. 7 at n_k = 2 summed by hand in the test."""
    nb, L, nk = 2, (2, 1), 2
    Gl = ki.random_blocks(RNG, (nk, nb, nb))
    Gg = ki.random_blocks(RNG, (nk, nb, nb))
    Sl, _ = oracle.sigma_pair_literal(nb, L, None, 1.3, Gl, Gg)
    Gt = lambda k, a, b: -np.conj(Gg[k, b, a])   # G^>_ab(k; t', t)
    k, j, m = 1, 0, 1
    jb, mb = 1 - j, 1 - m
    s = 0
    for q in range(nk):
        for kp in range(nk):
            s += Gl[(kp + q) % nk, jb, mb] * Gt(kp, mb, jb) * Gl[(k - q) % nk, j, m]
            s -= Gl[kp, j, mb] * Gt((kp + q - k) % nk, mb, jb) * Gl[q, jb, m]
    assert abs(Sl[k, j, m] - 1.3 * s / nk ** 2) < 1e-14


def test_sigma_zero_when_one_band_empty_of_partners():
    """v = 0 (no inter-band pairs) gives Sigma = 0 identically."""
    nb, L = 3, (3, 1)
    Gl = ki.random_blocks(RNG, (3, nb, nb))
    Gg = ki.random_blocks(RNG, (3, nb, nb))
    Sl, Sg = oracle.sigma_pair(nb, L, np.zeros((nb, nb)), 1.0, Gl, Gg)
    assert np.abs(Sl).max() == 0 and np.abs(Sg).max() == 0


# --------------------------------------------------------------------------
# Eq. 6 (left form) with trapezoid weights against exact integrals of
# exponentials; the leading trapezoid error (Euler-Maclaurin) must match.
# --------------------------------------------------------------------------
def _antiherm(rng, nb):
    a = ki.random_blocks(rng, (nb, nb))
    return a - a.conj().T


@pytest.mark.parametrize("nb,nk", [(1, 1), (2, 1), (3, 2)])
def test_collision_integral_against_exact_integrals(nb, nk):
    rng = np.random.default_rng(nb * 10 + nk)
    gl = np.stack([_antiherm(rng, nb) for _ in range(nk)])
    gg = np.stack([_antiherm(rng, nb) for _ in range(nk)])
    sl = ki.random_blocks(rng, (nk, nb, nb))
    sg = ki.random_blocks(rng, (nk, nb, nb))
    alpha, beta, T = 1.7, -0.6, 2.0
    kappa = alpha - beta

    def F(t):           # int_0^t e^{i kappa s} ds
        return (np.exp(1j * kappa * t) - 1) / (1j * kappa)

    def Ftrap_err(t):   # leading trapezoid error of F, dt^2/12 (f'(t) - f'(0))
        return 1j * kappa * (np.exp(1j * kappa * t) - 1) / 12.0

    errs = []
    for n in (20, 40):
        dt = T / n
        tri = [(i, j) for i in range(n + 1) for j in range(i + 1)]
        Hl = np.stack([gl * np.exp(-1j * beta * (i - j) * dt) for i, j in tri])
        Hg = np.stack([gg * np.exp(-1j * beta * (i - j) * dt) for i, j in tri])
        Sl = np.stack([sl * np.exp(-1j * alpha * (n - l) * dt) for l in range(n + 1)])
        Sg = np.stack([sg * np.exp(-1j * alpha * (n - l) * dt) for l in range(n + 1)])
        Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg)
        t = n * dt
        worst = 0.0
        for j in range(n + 1):
            tp = j * dt
            ph = np.exp(-1j * alpha * t + 1j * beta * tp)
            for x, (I, g, s) in enumerate(((Il, gl, sl), (Ig, gg, sg))):
                exact = ph * ((sg - sl) @ g * F(t) + s @ (gl - gg) * F(tp))
                lead = ph * ((sg - sl) @ g * Ftrap_err(t) + s @ (gl - gg) * Ftrap_err(tp)) * dt ** 2
                resid = np.abs(I[j] - exact - lead).max()
                worst = max(worst, resid)
                # the O(dt^2) term itself is resolved
                assert np.abs(I[j] - exact).max() <= 1.05 * np.abs(lead).max() + 1e-12
        errs.append(worst)
    # after removing the leading term the residual is O(dt^4)
    assert errs[1] < errs[0] / 10


def test_equal_time_collision_integrals_coincide():
    """I^>(n,n) = I^<(n,n): at j = n the two terms share weights and cancel."""
    nb, nk, n, dt = 2, 3, 7, 0.1
    ntri = (n + 1) * (n + 2) // 2
    Hl = ki.random_blocks(RNG, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(RNG, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(RNG, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(RNG, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg)
    assert np.abs(Il[n] - Ig[n]).max() < 1e-13 * np.abs(Il[n]).max()
    assert np.abs(Il[0] - Ig[0]).max() > 1e-3   # not trivially equal elsewhere


# --------------------------------------------------------------------------
# propagators and the row / diagonal update against matrix exponentials
# --------------------------------------------------------------------------
def _herm(rng, nb, scale=1.0):
    a = ki.random_blocks(rng, (nb, nb), scale)
    return 0.5 * (a + a.conj().T)


def test_propagators_against_expm():
    nb, nk, dt = 4, 3, 0.07
    h = np.stack([_herm(RNG, nb, 2.0) for _ in range(nk)])
    h[1] = np.diag([0.0, 0.5, 0.5, -1.0])      # exact zero and degenerate eigenvalues
    U, V, W, lam = oracle.propagators(nb, nk, dt, h)
    for k in range(nk):
        Ue = sla.expm(-1j * dt * h[k])
        assert np.abs(U[k] - Ue).max() < 1e-14
        assert np.abs(h[k] @ V[k] - (Ue - np.eye(nb))).max() < 1e-14
        assert np.abs(W[k] @ np.diag(lam[k]) @ W[k].conj().T - h[k]).max() < 1e-13
        assert np.abs(W[k].conj().T @ W[k] - np.eye(nb)).max() < 1e-14
        # V against the augmented exponential of y' = -i h y - i c
        aug = np.zeros((2 * nb, 2 * nb), complex)
        aug[:nb, :nb] = -1j * h[k]
        aug[:nb, nb:] = -1j * np.eye(nb)
        Ve = sla.expm(dt * aug)[:nb, nb:]
        assert np.abs(V[k] - Ve).max() < 1e-14


def test_update_row_against_exact_constant_source_solutions():
    nb, nk, n, dt, theta = 3, 2, 5, 0.05, 0.5
    h = np.stack([_herm(RNG, nb, 1.5) for _ in range(nk)])
    U, V, W, lam = oracle.propagators(nb, nk, dt, h)
    Gpl = ki.random_blocks(RNG, (n, nk, nb, nb))
    Gpg = ki.random_blocks(RNG, (n, nk, nb, nb))
    Gpl[n - 1] = np.stack([1j * _herm(RNG, nb) for _ in range(nk)])   # anti-Hermitian diagonal
    Ipl = ki.random_blocks(RNG, (n, nk, nb, nb))
    Ipg = ki.random_blocks(RNG, (n, nk, nb, nb))
    Icl = ki.random_blocks(RNG, (n + 1, nk, nb, nb))
    Icg = ki.random_blocks(RNG, (n + 1, nk, nb, nb))
    outl, outg = oracle.update_row(nb, nk, n, dt, theta, U, V, W, lam, Gpl, Gpg, Ipl, Ipg, Icl, Icg)
    I3 = np.eye(nb)
    for k in range(nk):
        # rows: y' = -i h y - i Ibar, exact over one step
        aug = np.zeros((2 * nb, 2 * nb), complex)
        aug[:nb, :nb] = -1j * h[k]
        aug[:nb, nb:] = -1j * I3
        E = sla.expm(dt * aug)
        for j in range(n):
            for (out, Gp, Ip, Ic) in ((outl, Gpl, Ipl, Icl), (outg, Gpg, Ipg, Icg)):
                ib = (1 - theta) * Ip[j, k] + theta * Ic[j, k]
                exact = E[:nb, :nb] @ Gp[j, k] + E[:nb, nb:] @ ib
                assert np.abs(out[j, k] - exact).max() < 1e-13
        # diagonal: i G' = [h, G] + S, S = Ibar + Ibar^+, vectorised exactly
        S = (1 - theta) * (Ipl[n - 1, k] + Ipl[n - 1, k].conj().T) + theta * (Icl[n, k] + Icl[n, k].conj().T)
        Lop = -1j * (np.kron(h[k], I3) - np.kron(I3, h[k].T))
        aug2 = np.zeros((nb * nb + 1, nb * nb + 1), complex)
        aug2[:nb * nb, :nb * nb] = Lop
        aug2[:nb * nb, nb * nb] = -1j * S.reshape(-1)
        y = sla.expm(dt * aug2) @ np.concatenate([Gpl[n - 1, k].reshape(-1), [1.0]])
        exact = y[:nb * nb].reshape(nb, nb)
        assert np.abs(outl[n, k] - exact).max() < 1e-13
        assert np.abs(outg[n, k] - (exact - 1j * I3)).max() < 1e-13


# --------------------------------------------------------------------------
# whole-step pins
# --------------------------------------------------------------------------
def test_c1_bands_match_stated_dispersion():
    s = ki.config("c1")
    for k in range(s.nk):
        kk = 2 * np.pi * k / 8
        e = np.linalg.eigvalsh(h0_of(s, k))
        want = sorted(-2 * np.cos(kk + b * np.pi / 2) + 0.5 * b for b in range(2))
        assert np.allclose(sorted(e), want, atol=1e-14)


@pytest.mark.parametrize("driven", [False, True])
def test_noninteracting_closed_form(driven):
    """U = 0: G^<(k; t_n, t_j) = i Uc_n rho0 Uc_j^+ with Uc the product of the
    per-step exponentials of h0(k - A_i); undriven this is i f(e) e^{-i e (t-t')}."""
    s = ki.small_system(3, (3, 2), 24, 0.05, 0.0, seed=3, drive_amp=0.6 if driven else 0.0)
    o = oracle.Oracle(s)
    o.step(s.nt)
    for k in range(s.nk):
        rho0 = fermi_matrix(h0_of(s, k), s.beta, s.mu)
        Uc = [np.eye(s.nb, dtype=complex)]
        for i in range(s.nt):
            A = 0.0 if s.A is None else s.A[i]
            Uc.append(sla.expm(-1j * s.dt * h0_of(s, k, A)) @ Uc[-1])
        for (i, j) in [(0, 0), (5, 2), (13, 13), (24, 0), (24, 17), (3, 9)]:
            want = 1j * Uc[i] @ rho0 @ Uc[j].conj().T
            got = o.block(i, j, 0)[k]
            assert np.abs(got - want).max() < 1e-13, (i, j)
            gotg = o.block(i, j, 1)[k]
            wantg = want - 1j * Uc[i] @ Uc[j].conj().T
            assert np.abs(gotg - wantg).max() < 1e-13, (i, j)
    if not driven:   # time-translation invariance in equilibrium
        a, b = o.block(20, 7, 0), o.block(13, 0, 0)
        assert np.abs(a - b).max() < 1e-13


def test_noninteracting_closed_form_with_dipole_kick():
    """U = 0 with the dipole drive of Eq. 4: G^<(t_n, t_j) = i Uc_n rho0 Uc_j^+
    with Uc the product of exp(-i dt (h0(k) + E_i M)); the kick moves weight
    from the valence to the conduction band."""
    s = ki.config("paper", nt=40)
    s.L = (16, 1)
    s.U = 0.0
    s.dipole_E = ki.kick(40, s.dt, 0.3, 0.4)
    o = oracle.Oracle(s)
    o.step(40)
    nkb0 = o.observables(0)[0]
    nkb1 = o.observables(40)[0]
    assert np.abs(nkb1[:, 1] - nkb0[:, 1]).max() > 1e-3
    for k in (0, 5, 11):
        rho0 = fermi_matrix(h0_of(s, k), s.beta, s.mu)
        Uc = [np.eye(2, dtype=complex)]
        for i in range(40):
            Uc.append(sla.expm(-1j * s.dt * (h0_of(s, k) + s.dipole_E[i] * s.dipole_M)) @ Uc[-1])
        for (i, j) in [(10, 3), (20, 14), (40, 0), (40, 40), (7, 33)]:
            want = 1j * Uc[i] @ rho0 @ Uc[j].conj().T
            assert np.abs(o.block(i, j, 0)[k] - want).max() < 1e-13, (i, j)


def test_particle_number_conserved_driven_interacting():
    s = ki.small_system(3, (3, 3), 40, 0.04, 1.2, seed=5, drive_amp=0.5)
    o = oracle.Oracle(s)
    o.step(s.nt)
    N = np.array([o.observables(n)[1][0] for n in range(s.nt + 1)])
    assert np.abs(N - N[0]).max() < 1e-12 * abs(N[0])
    nkb = np.array([o.observables(n)[0] for n in range(s.nt + 1)])
    assert np.abs(nkb - nkb[0]).max() > 1e-3   # the drive does move occupations


def test_equal_time_lesser_is_antihermitian_and_greater_offset():
    s = ki.config("c1", nt=20)
    o = oracle.Oracle(s)
    o.step(20)
    for n in (0, 7, 20):
        g = o.block(n, n, 0)
        assert np.abs(g + np.conj(np.swapaxes(g, 1, 2))).max() < 1e-15
        assert np.abs(o.block(n, n, 1) - (g - 1j * np.eye(2))).max() < 1e-15


def _full_grid_errors(o, f, n):
    """symmetry defect of the full-grid column and its row's distance from the
    triangle oracle, both relative to the largest |G| of row n"""
    scale = max(np.abs(o.row(n, 0)).max(), np.abs(o.row(n, 1)).max())
    sym = tri = 0.0
    for x in (0, 1):
        col = np.stack([f.block(j, n, x) for j in range(n + 1)])   # propagated, never mirrored
        row = np.stack([f.block(n, j, x) for j in range(n + 1)])
        sym = max(sym, np.abs(col + np.conj(np.swapaxes(row, -1, -2))).max() / scale)
        tri = max(tri, np.abs(row - o.row(n, x)).max() / scale)
    return sym, tri


@pytest.mark.parametrize("case", ["ring_driven", "mesh_general_v", "gregory_Ut"])
def test_full_grid_column_is_adjoint_of_row(case):
    """The oracle's full-grid mode advances the upper triangle G(t_j, t_n) with
    the right equation and Eq. 6 as printed (G * Sigma, second limit t'), with
    Eq. 7 summed from the stored G(t_n, t_l) and G(t_l, t_n) and no use of the
    adjoint symmetry. The column it produces must be -G(t_n, t_j)^+ of the row
    the left equation produces, and that row must be the triangle oracle's:
    this pins G^x(t,t')^+ = -G^x(t',t) and the left-form reading of Eq. 6."""
    import dataclasses
    if case == "ring_driven":
        s = ki.small_system(2, (4, 1), 12, 0.05, 0.8, seed=9, drive_amp=0.4, paper_shift=1)
        Us = None
    elif case == "mesh_general_v":
        s = ki.small_system(3, (2, 2), 10, 0.05, 1.1, seed=6, drive_amp=0.5)
        v = np.random.default_rng(8).uniform(0.2, 1.4, (3, 3))
        s.v = np.triu(v, 1) + np.triu(v, 1).T
        Us = None
    else:
        s = dataclasses.replace(ki.small_system(2, (3, 1), 12, 0.05, 0.9, seed=4, drive_amp=0.3),
                                quadrature=1)
        Us = 0.9 + 0.3 * np.sin(0.4 * np.arange(13))
    o = oracle.Oracle(s, U=Us)
    f = oracle.Oracle(s, U=Us, full_grid=True)
    o.step(s.nt)
    f.step(s.nt)
    for n in (1, 5, s.nt):
        sym, tri = _full_grid_errors(o, f, n)
        assert sym < 1e-13, (n, sym)
        assert tri < 1e-13, (n, tri)
    assert np.abs(f.observables(s.nt)[1] - o.observables(s.nt)[1]).max() < 1e-13
    # not trivially symmetric: the interaction moved the system off its free evolution
    assert np.abs(o.observables(s.nt)[1][3]) > 1e-4


def test_full_grid_printed_upper_limit_breaks_symmetry():
    """Eq. 6 printed with t as the second upper limit: the column propagated
    with it is no longer the adjoint of the row (O(1e-3) after a few steps),
    so the limit must be t' (the reading the library and the oracle take)."""
    s = ki.small_system(2, (4, 1), 12, 0.05, 0.8, seed=9, drive_amp=0.4, paper_shift=1)
    o = oracle.Oracle(s)
    p = oracle.Oracle(s, full_grid=True, right_limit_printed=True)
    o.step(12)
    p.step(12)
    sym, _ = _full_grid_errors(o, p, 12)
    assert sym > 1e-3, sym


def test_energy_drift_is_second_order_in_dt():
    """Undriven c1: E_tot is conserved by the continuous equations of a
    conserving approximation; the discrete drift must fall ~4x per dt halving.
    A wrong sign of the correlation energy breaks this (drift O(1e-2), no decay)."""
    drifts = []
    for dt in (0.05, 0.025, 0.0125):
        s = ki.config("c1")
        s.dt, s.nt = dt, int(round(1.6 / dt))
        o = oracle.Oracle(s)
        o.step(s.nt)
        drifts.append(abs(o.observables(s.nt)[1][5] - o.observables(0)[1][5]))
    r1, r2 = drifts[0] / drifts[1], drifts[1] / drifts[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, drifts
    assert drifts[0] < 1e-4


def test_time_step_order_two():
    """Interacting c1-like ring: G at t = 1.2 converges at second order in dt."""
    def run(dt):
        s = ki.config("c1")
        s.L = (4, 1)
        s.dt, s.nt = dt, int(round(1.2 / dt))
        o = oracle.Oracle(s)
        o.step(s.nt)
        return o.block(s.nt, s.nt // 2, 0)
    ref = run(0.05 / 8)
    e = [np.abs(run(dt) - ref).max() for dt in (0.05, 0.025, 0.0125)]
    # Richardson-corrected ratios against a finite-dt reference
    assert 3.0 < e[0] / e[1] < 5.0 and 3.0 < e[1] / e[2] < 5.5, e


# --------------------------------------------------------------------------
# exact diagonalisation: second Born + HF is exact through O(U^2) for an
# uncorrelated initial state, so the density error must scale as U^3.
# --------------------------------------------------------------------------
def _ed_density(sys, U, T, dt):
    nb, nk, L = sys.nb, sys.nk, sys.L
    M = nb * nk
    dim = 2 ** M
    c = []
    for m in range(M):
        op = np.zeros((dim, dim))
        for st in range(dim):
            if st >> m & 1:
                sign = (-1) ** bin(st & ((1 << m) - 1)).count("1")
                op[st ^ (1 << m), st] = sign
        c.append(op)
    cd = [x.T for x in c]
    H0 = np.zeros((dim, dim), complex)
    for k in range(nk):
        hk = h0_of(sys, k)
        for a in range(nb):
            for b in range(nb):
                if hk[a, b] != 0:
                    H0 += hk[a, b] * cd[k * nb + a] @ c[k * nb + b]
    Hint = np.zeros((dim, dim), complex)
    for i0 in range(L[0]):
        for i1 in range(L[1]):
            dens = []
            for a in range(nb):
                op = sum(np.exp(2j * np.pi * ((k // L[1]) * i0 / L[0] + (k % L[1]) * i1 / L[1]))
                         * c[k * nb + a] for k in range(nk)) / math.sqrt(nk)
                dens.append(op.conj().T @ op)
            for a in range(nb):
                for b in range(a + 1, nb):
                    Hint += sys.v[a, b] * dens[a] @ dens[b]
    Hsh = np.zeros((dim, dim), complex)
    if sys.paper_shift:
        for k in range(nk):
            Hsh -= cd[k * nb + nb - 1] @ c[k * nb + nb - 1]
    Ntot = sum(cd[m] @ c[m] for m in range(M))
    w, V = np.linalg.eigh(H0 - sys.mu * Ntot)
    rho = V @ np.diag(np.exp(-sys.beta * (w - w.min()))) @ V.conj().T
    rho /= np.trace(rho)
    ew, EV = np.linalg.eigh(H0 + U * Hint + U * Hsh)
    nops = [cd[m] @ c[m] for m in range(M)]
    out = []
    nt = int(round(T / dt))
    for i in range(nt + 1):
        Ut = EV @ np.diag(np.exp(-1j * ew * i * dt)) @ EV.conj().T
        r = Ut @ rho @ Ut.conj().T
        out.append(np.array([np.trace(r @ x).real for x in nops]).reshape(nk, nb))
    return np.array(out)


@pytest.mark.slow
def test_exact_diagonalisation_error_scales_as_U_cubed():
    T, dt = 1.0, 0.02
    errs = []
    for U in (0.8, 0.4, 0.2):
        s = ki.small_system(2, (4, 1), int(round(T / dt)), dt, U, seed=11, beta=5.0,
                            hf=1, paper_shift=1)
        ed = _ed_density(s, U, T, dt)
        o = oracle.Oracle(s)
        o.step(s.nt)
        kbe = np.array([o.observables(n)[0] for n in range(s.nt + 1)])
        errs.append(np.abs(kbe - ed).max())
        assert np.abs(ed - ed[0]).max() > 20 * errs[-1]    # the dynamics is resolved
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.5 and 7.0 < r2 < 9.5, errs


def _ed_three_band(U, vmode, T=1.0, dt=0.01):
    """N_b = 3 on a 3-site ring; band b disperses as -2 cos(k + b pi/3), so no
    k -> -k symmetry hides an index error in the momentum sums (with h(k) =
    h(-k) the bubble obeys P(q) = P(-q) and a swapped band pattern cancels)."""
    s = ki.small_system(3, (3, 1), int(round(T / dt)), dt, U, seed=12, beta=5.0, hf=1, paper_shift=0)
    for b in range(3):
        s.hop_T[1, b, b] *= np.exp(1j * b * np.pi / 3)
        s.hop_T[2, b, b] *= np.exp(-1j * b * np.pi / 3)
    if vmode == "random":
        v = np.random.default_rng(21).uniform(0.3, 1.5, (3, 3))
        s.v = np.triu(v, 1) + np.triu(v, 1).T
    ed = _ed_density(s, U, T, dt)
    o = oracle.Oracle(s)
    o.step(s.nt)
    kbe = np.array([o.observables(n)[0] for n in range(s.nt + 1)])
    return kbe, ed


@pytest.mark.slow
@pytest.mark.parametrize("vmode", ["pair", "random"])
def test_exact_diagonalisation_second_order_three_bands(vmode):
    """Second Born + HF is exact through O(U^2) for an uncorrelated start, so
    the U^2 coefficient of the density, c2 = [n(U) + n(-U) - 2 n(0)] / (2 U^2),
    must agree with exact diagonalisation up to O(U^2) (and the time step's
    O(dt^2)). N_b = 3 exercises the band pattern v_ja v_mb of the generalised
    Eq. 7 beyond the paper's two bands, for v = 1 - delta and a random
    symmetric v: swapping it to v_jb v_ma leaves a ~1 % discrepancy that does
    not fall with U."""
    k0, e0 = _ed_three_band(0.0, vmode)
    assert np.abs(k0 - e0).max() < 1e-12      # U = 0: both exact
    d2, d1, c2s = [], [], []
    for U in (0.2, 0.1, 0.05):
        kp, ep = _ed_three_band(U, vmode)
        km, em = _ed_three_band(-U, vmode)
        c2k, c2e = (kp + km - 2 * k0) / (2 * U * U), (ep + em - 2 * e0) / (2 * U * U)
        c1k, c1e = (kp - km) / (2 * U), (ep - em) / (2 * U)
        d2.append(np.abs(c2k - c2e).max())
        d1.append(np.abs(c1k - c1e).max())
        c2s.append(np.abs(c2e).max())
    assert c2s[-1] > 1e-2                       # the second-order response is resolved
    assert d2[0] / d2[1] > 3.0 and d2[1] / d2[2] > 2.0, d2
    assert d2[2] < 2e-3 * c2s[-1], (d2, c2s)
    # first order (HF): the odd difference carries the O(U^3) error as U^2
    assert d1[0] / d1[1] > 3.0 and d1[1] / d1[2] > 3.0, d1


def test_corrector_tolerance_limits_of_algorithm_1():
    """Algorithm 1's corrector loop with its epsilon: a tolerance no pass can meet
    runs all n_corr passes and reproduces the fixed-count run exactly; one every
    pass meets stops after the first and reproduces n_corr = 1 exactly."""
    import dataclasses
    s = ki.config("c1", nt=8)
    fixed = oracle.Oracle(dataclasses.replace(s, n_corr=3))
    fixed.step(8)
    tiny = oracle.Oracle(dataclasses.replace(s, n_corr=3, corr_tol=1e-300))
    tiny.step(8)
    assert tiny.iterations().tolist() == [0] + [3] * 8
    one = oracle.Oracle(dataclasses.replace(s, n_corr=1))
    one.step(8)
    huge = oracle.Oracle(dataclasses.replace(s, n_corr=3, corr_tol=1e30))
    huge.step(8)
    assert huge.iterations().tolist() == [0] + [1] * 8
    for i in (1, 4, 8):
        for x in (0, 1):
            assert np.array_equal(tiny.row(i, x), fixed.row(i, x))
            assert np.array_equal(huge.row(i, x), one.row(i, x))


def test_corrector_tolerance_counts_follow_the_change():
    """with a moderate epsilon the number of passes varies from step to step, and
    tightening epsilon never removes a pass"""
    import dataclasses
    s = ki.config("c1", nt=24)
    runs = []
    for tol in (2e-10, 1.19e-10, 1e-12):
        o = oracle.Oracle(dataclasses.replace(s, n_corr=4, corr_tol=tol))
        o.step(24)
        runs.append(o.iterations())
    assert set(runs[1][1:].tolist()) == {3, 4}
    assert np.all(runs[0] <= runs[1]) and np.all(runs[1] <= runs[2])


@pytest.mark.parametrize("nb,nk", [(2, 3), (3, 2)])
def test_gregory_collision_integral_converges_at_fourth_order(nb, nk):
    """The Gregory weights against exact integrals of the same exponential
    histories as the trapezoid pin: columns j >= 2 and the first integral use
    rules exact for cubics, so their error falls ~16x per halving of dt; the
    column j = 1 (a single trapezoid panel) falls ~8x."""
    rng = np.random.default_rng(nb * 10 + nk + 7)
    gl = np.stack([_antiherm(rng, nb) for _ in range(nk)])
    gg = np.stack([_antiherm(rng, nb) for _ in range(nk)])
    sl = ki.random_blocks(rng, (nk, nb, nb))
    sg = ki.random_blocks(rng, (nk, nb, nb))
    alpha, beta, T = 1.7, -0.6, 2.0
    kappa = alpha - beta

    def F(t):
        return (np.exp(1j * kappa * t) - 1) / (1j * kappa)

    errs_hi, errs_1 = [], []
    for n in (20, 40):
        dt = T / n
        tri = [(i, j) for i in range(n + 1) for j in range(i + 1)]
        Hl = np.stack([gl * np.exp(-1j * beta * (i - j) * dt) for i, j in tri])
        Hg = np.stack([gg * np.exp(-1j * beta * (i - j) * dt) for i, j in tri])
        Sl = np.stack([sl * np.exp(-1j * alpha * (n - l) * dt) for l in range(n + 1)])
        Sg = np.stack([sg * np.exp(-1j * alpha * (n - l) * dt) for l in range(n + 1)])
        Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=1)
        t = n * dt
        e_hi = e_1 = 0.0
        for j in range(n + 1):
            tp = j * dt
            ph = np.exp(-1j * alpha * t + 1j * beta * tp)
            for I, g, s in ((Il, gl, sl), (Ig, gg, sg)):
                err = np.abs(I[j] - ph * ((sg - sl) @ g * F(t) + s @ (gl - gg) * F(tp))).max()
                if j == 1:
                    e_1 = max(e_1, err)
                elif j != 1:
                    e_hi = max(e_hi, err)
        errs_hi.append(e_hi)
        errs_1.append(e_1)
    assert 13 < errs_hi[0] / errs_hi[1] < 19, errs_hi
    assert 6.5 < errs_1[0] / errs_1[1] < 9.5, errs_1


def test_gregory_weights_integrate_cubics_exactly():
    """I^< of a history whose integrands are cubic in the memory time: every rule
    with m >= 2 nodes-1 is exact (Gregory, Simpson, Simpson 3/8, Boole)."""
    nb, nk, dt = 1, 1, 0.3
    for n in range(2, 9):
        c3 = lambda t: 0.5 - 1.1 * t + 0.7 * t ** 2 + 0.2 * t ** 3
        tri = [(i, j) for i in range(n + 1) for j in range(i + 1)]
        # G^<(l, j) = i (for every l, j: its adjoint image is also i), G^> = 0
        Hl = np.full((len(tri), nk, nb, nb), 1j)
        Hg = np.zeros_like(Hl)
        Sl = np.zeros((n + 1, nk, nb, nb), complex)
        Sg = np.stack([np.full((nk, nb, nb), c3(l * dt)) for l in range(n + 1)])
        Il, _ = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=1)
        T = n * dt
        exact = 1j * (0.5 * T - 1.1 * T ** 2 / 2 + 0.7 * T ** 3 / 3 + 0.2 * T ** 4 / 4)
        # j = 0: only the first integral; I^<(n, 0) = int_0^T (S^> - S^<) G^< = i int c3
        assert abs(Il[0][0, 0, 0] - exact) < 1e-13, (n, Il[0][0, 0, 0], exact)
