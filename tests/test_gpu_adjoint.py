"""Reverse mode through the C ABI (kbe_backward) against finite differences.

Loss L = sum_kb (n_kb(t_N) - n*_kb)^2 of the final-time occupations; the
library returns dL/dA_i for every Peierls sample and dL/dU.

* Against the oracle: its Richardson-extrapolated central differences
  (oracle/gradient.py, pinned by tests/test_oracle_gradient.py) on small
  systems, every A_i and U (or every U(t_i) sample), bar 1e-7 of the
  largest component. The oracle's
  forward is the same discrete map up to rounding (exact exponentials in
  place of the converged series), so the two derivatives agree to the
  differences' accuracy.
* Against the library's own forward: central differences with h = 1e-6 on
  c2's system (16 seeded A_i and U), normwise relative
  error <= 1e-5 (256 steps here; bench.py times the 512-step gradient).
"""
import ctypes
import dataclasses

import numpy as np
import pytest

import kbe_inputs as ki
from oracle import gradient as og

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu


def gpu_loss(sys, N, tgt, A=None, U=None, **over):
    s = dataclasses.replace(sys, A=sys.A if A is None else np.asarray(A, np.float64),
                            U=sys.U if U is None else float(U))
    g = kbe.KBE.from_system(s, nt_max=max(N, s.nt), **over)
    g.step(N)
    nkb, _ = g.observables(N)
    g.close()
    return float(((nkb - tgt) ** 2).sum())


def gpu_grad(sys, N, tgt, **over):
    g = kbe.KBE.from_system(sys, nt_max=max(N, sys.nt), **over)
    g.step(N)
    nkb, _ = g.observables(N)
    dA, dU = g.backward(2.0 * (nkb - tgt))
    g.close()
    return dA, dU


# dt ||h||_rowsum stays <= 1/4 (the unscaled propagator series the reverse mode needs)
SMALL = [
    # nb, L, nt, dt, U, n_corr, hf, paper_shift, band_velocity
    (2, (4, 1), 8, 0.05, 0.8, 2, 1, 1, 0.5),
    (3, (2, 3), 6, 0.03, 1.1, 1, 1, 0, 0.3),
    (2, (3, 2), 5, 0.04, 0.6, 0, 0, 0, 0.5),
    (4, (2, 2), 5, 0.02, 0.9, 2, 1, 0, 0.3),
]


@pytest.mark.parametrize("nb,L,nt,dt,U,nc,hf,shift,bv", SMALL)
def test_gradient_matches_oracle_reference(nb, L, nt, dt, U, nc, hf, shift, bv):
    sys = ki.small_system(nb, L, nt, dt, U, seed=7 + nb, drive_amp=0.6, n_corr=nc, hf=hf,
                          paper_shift=shift, band_velocity=bv)
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    dA, dU = gpu_grad(sys, nt, tgt)
    assert np.all(dA[nt:] == 0.0)
    rA, rU = og.gradient(sys, nt, tgt)
    scale = max(np.abs(rA).max(), abs(rU))
    assert np.abs(dA[:nt] - rA).max() < 1e-7 * scale, (dA[:nt], rA)
    assert abs(dU - rU) < 1e-7 * scale, (dU, rU)


def test_gradient_with_general_pair_pattern():
    """a general symmetric v_ab with a non-zero diagonal: a transposed or dropped
    v index in the Sigma or mean-field transposes would show here"""
    sys = ki.small_system(3, (3, 1), 5, 0.03, 0.9, seed=13, drive_amp=0.5, band_velocity=0.4)
    w = np.random.default_rng(13).uniform(0.2, 1.0, (3, 3))
    sys.v = w + w.T
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    dA, dU = gpu_grad(sys, 5, tgt)
    rA, rU = og.gradient(sys, 5, tgt)
    scale = max(np.abs(rA).max(), abs(rU))
    assert np.abs(dA[:5] - rA).max() < 1e-7 * scale, (dA[:5], rA)
    assert abs(dU - rU) < 1e-7 * scale, (dU, rU)


def test_asymmetric_pair_pattern_is_refused():
    sys = ki.small_system(3, (3, 1), 5, 0.03, 0.9, seed=13)
    g = kbe.KBE.from_system(sys)
    v = np.ones((3, 3)) - np.eye(3)
    v[0, 1] = 0.5
    with pytest.raises(kbe.KBEError) as ex:
        g.set_interaction(np.array([0.9]), v)
    assert ex.value.status == -1
    g.close()


def test_gradient_with_dipole_drive():
    """the dipole term of h carries no parameter but must be in the recomputed steps"""
    sys = ki.small_system(2, (4, 1), 6, 0.05, 0.7, seed=5, drive_amp=0.4, paper_shift=1,
                          band_velocity=0.3)
    sys.dipole_M = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sys.dipole_E = np.linspace(0.2, -0.3, 6)
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    dA, dU = gpu_grad(sys, 6, tgt)
    rA, rU = og.gradient(sys, 6, tgt)
    scale = max(np.abs(rA).max(), abs(rU))
    assert np.abs(dA[:6] - rA).max() < 1e-7 * scale
    assert abs(dU - rU) < 1e-7 * scale


def test_gradient_c2_system():
    """c2's system (N_b = 4, 8x8, dt = 0.02) over 256 steps, targets n* ~ U(0,1) seed 4:
    central differences of the library's forward, h = 1e-6, on U and 16 seeded A_i"""
    sys = ki.config("c2", nt=256)
    N = sys.nt
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    dA, dU = gpu_grad(sys, N, tgt)
    idx = np.sort(np.random.default_rng(4).choice(N, 16, replace=False))
    h = 1e-6
    fd, ad = [], []
    for i in idx:
        e = np.zeros(N)
        e[i] = h
        fd.append((gpu_loss(sys, N, tgt, A=sys.A + e) - gpu_loss(sys, N, tgt, A=sys.A - e)) / (2 * h))
        ad.append(dA[i])
    fd.append((gpu_loss(sys, N, tgt, U=sys.U + h) - gpu_loss(sys, N, tgt, U=sys.U - h)) / (2 * h))
    ad.append(dU)
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(ad - fd) <= 1e-5 * np.linalg.norm(fd), (ad, fd)
    assert np.all(np.isfinite(dA)) and np.abs(dA).max() > 0


def test_gradient_per_u_sample():
    """U(t) samples: dL/dU_i for every sample through Sigma (-U_n U_l) and the mean
    field (U_mid), against the oracle's reference; and a constant U equals the
    sum of the per-sample gradient at constant samples"""
    sys = ki.small_system(2, (4, 1), 6, 0.05, 0.8, seed=9, drive_amp=0.5, paper_shift=1, band_velocity=0.5)
    N = 6
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    Us = 0.8 * (1.0 + 0.3 * np.sin(np.arange(N + 1) * 0.9))
    g = kbe.KBE.from_system(sys, U=Us)
    g.step(N)
    nkb, _ = g.observables(N)
    dA, dU = g.backward(2.0 * (nkb - tgt))
    g.close()
    assert dU.shape == (N + 1,)
    rU = og.gradient_samples(sys, N, tgt, Us)
    scale = np.abs(rU).max()
    assert np.abs(dU[: N + 1] - rU).max() < 1e-7 * scale, (dU, rU)
    # constant samples: per-sample gradient sums to the scalar one
    c = kbe.KBE.from_system(sys, U=np.full(N + 1, sys.U))
    c.step(N)
    nkb, _ = c.observables(N)
    dA_s, dU_s = c.backward(2.0 * (nkb - tgt))
    c.close()
    dA_c, dU_c = gpu_grad(sys, N, tgt)
    assert abs(dU_s.sum() - dU_c) < 1e-12 * abs(dU_c)
    assert np.allclose(dA_s, dA_c, rtol=1e-12, atol=1e-16)


def test_backward_leaves_state_and_is_deterministic():
    sys = ki.small_system(3, (4, 4), 12, 0.025, 1.0, seed=2, drive_amp=0.5, band_velocity=0.4)
    tgt = ki.targets(sys.nk, sys.nb, seed=4)
    a = kbe.KBE.from_system(sys, nt_max=20)
    b = kbe.KBE.from_system(sys, nt_max=20)
    a.step(8)
    b.step(8)
    nkb, _ = a.observables(8)
    g1 = a.backward(2 * (nkb - tgt))
    g2 = a.backward(2 * (nkb - tgt))
    assert np.array_equal(g1[0], g2[0]) and g1[1] == g2[1]
    a.step(4)
    b.step(4)
    for i in (7, 8, 12):
        for x in (0, 1):
            assert np.array_equal(a.row(i, x), b.row(i, x)), (i, x)
    assert np.array_equal(a.observables_all()[0], b.observables_all()[0])


def test_backward_refusals():
    sys = ki.small_system(2, (4, 1), 4, 0.05, 0.5, seed=1, drive_amp=0.3)
    g = kbe.KBE.from_system(sys)
    z = np.zeros((sys.nk, sys.nb))
    with pytest.raises(kbe.KBEError) as ex:      # no step yet
        g.backward(z)
    assert ex.value.status == -4
    g.close()
    d = kbe.KBE.from_system(sys, precision=kbe.KBE_PREC_DF64)
    d.step(2)
    with pytest.raises(kbe.KBEError) as ex:
        d.backward(z)
    assert ex.value.status == -7
    d.close()
    # dt ||h|| > 1/4 needs the scaled-and-squared propagators: refused, handle still steps
    big = ki.small_system(2, (4, 1), 6, 0.3, 0.5, seed=1, drive_amp=0.3)
    b = kbe.KBE.from_system(big)
    b.step(2)
    with pytest.raises(kbe.KBEError) as ex:
        b.backward(z)
    assert ex.value.status == -7
    b.step(2)
    b.synchronize()
    assert b.n == 4
    b.close()


def test_autograd_function_matches_backward():
    sys = ki.small_system(2, (4, 1), 6, 0.05, 0.8, seed=9, drive_amp=0.5, paper_shift=1, band_velocity=0.5)
    tgt = torch.tensor(ki.targets(sys.nk, sys.nb, seed=4))
    A = torch.tensor(sys.A, requires_grad=True)
    U = torch.tensor(sys.U, dtype=torch.float64, requires_grad=True)
    n = kbe.occupations(sys, A, U, 6)
    L = ((n - tgt) ** 2).sum()
    L.backward()
    dA, dU = gpu_grad(sys, 6, tgt.numpy())
    assert np.allclose(A.grad.numpy(), dA[:6], rtol=0, atol=1e-15)
    assert abs(U.grad.item() - dU) < 1e-15
