"""Whole-step parity: KBE trajectories through the C-ABI handle API against
the FP64 oracle on the same seeded systems, every stored entry compared.

The FP64 bar is 1e-10 relative on every stored G entry, with a zero-entry
floor of 1e-4 x (largest |G^<| or |G^>| of that row): smaller entries, e.g.
those that vanish in exact arithmetic or carry Fermi factors near e^{-40}, are
compared absolutely at 1e-14 of the row maximum, which is what two FP64
eigen-solvers agree to. The scale is taken over both components because
G^>(t,t) = G^<(t,t) - i: a filled band has |G^>| ~ 1 - f, pure cancellation.
"""
import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import relerr

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu
TOL = 1e-10


def compare_trajectory(sys, nsteps, rows=None, U=None, **over):
    g = kbe.KBE.from_system(sys, U=U, **over)
    g.step(nsteps)
    g.synchronize()
    okw = {k: v for k, v in over.items() if k in ("n_corr", "hf", "paper_shift")}
    o = oracle.Oracle(sys, U=U, **okw)
    o.step(nsteps)
    worst = 0.0
    for i in (range(nsteps + 1) if rows is None else rows):
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            e_el, e_norm = relerr(g.row(i, x), ref[x], scale=scale)
            assert e_el < TOL, (i, x, e_el)
            worst = max(worst, e_el)
    nkb_g, sc_g = g.observables_all()
    for n in range(nsteps + 1):
        nkb_o, sc_o = o.observables(n)
        assert np.abs(nkb_g[n] - nkb_o).max() < TOL
        assert np.abs(sc_g[n] - sc_o).max() < TOL * max(1.0, np.abs(sc_o).max()), (n, sc_g[n], sc_o)
    g.close()
    return worst


def test_c1_full_trajectory_every_entry():
    s = ki.config("c1")
    compare_trajectory(s, s.nt)


def test_c2_system_prefix_every_entry():
    s = ki.config("c2")
    compare_trajectory(s, 20)


@pytest.mark.parametrize("nb,L,dim_drive,n_corr,hf,shift,nsteps", [
    (1, (6, 1), 0.4, 2, 1, 0, 12),
    (2, (5, 1), 0.0, 0, 1, 1, 10),
    (3, (3, 3), 0.5, 1, 0, 0, 14),
    (4, (7, 3), 0.3, 3, 1, 0, 9),
    (6, (2, 3), 0.2, 2, 1, 0, 6),
    (8, (3, 2), 0.0, 2, 1, 0, 5),
    (12, (2, 1), 0.1, 2, 1, 0, 4),
    (16, (1, 2), 0.0, 1, 1, 0, 3),
    (2, (1, 1), 0.0, 2, 1, 1, 8),
])
def test_small_systems_every_entry(nb, L, dim_drive, n_corr, hf, shift, nsteps):
    s = ki.small_system(nb, L, nsteps, 0.05, 0.8, seed=nb * 31 + L[0], drive_amp=dim_drive,
                        hf=hf, paper_shift=shift, n_corr=n_corr)
    compare_trajectory(s, nsteps)


def test_time_dependent_interaction_samples():
    s = ki.small_system(2, (6, 1), 12, 0.05, 1.0, seed=4, drive_amp=0.3)
    U = 1.0 + 0.3 * np.sin(np.arange(13) * 0.4)
    compare_trajectory(s, 12, U=U)


def test_nt_max_one_and_stepping_in_pieces():
    s = ki.small_system(2, (4, 1), 1, 0.05, 0.7, seed=2)
    compare_trajectory(s, 1)
    s = ki.small_system(3, (4, 1), 9, 0.05, 0.7, seed=3, drive_amp=0.2)
    g = kbe.KBE.from_system(s)
    for _ in range(3):
        g.step(3)
    o = oracle.Oracle(s)
    o.step(9)
    assert relerr(g.row(9, 0), o.row(9, 0))[0] < TOL


def test_errors_are_reported_not_fatal():
    s = ki.small_system(2, (4, 1), 3, 0.05, 0.7, seed=2)
    g = kbe.KBE(s.nb, s.dim, s.L, 3, s.dt, s.beta, s.mu)
    with pytest.raises(kbe.KBEError) as e:
        g.step(1)                       # before reset
    assert e.value.status == -4
    with pytest.raises(kbe.KBEError):
        g.reset()                       # no hamiltonian yet
    g.set_hamiltonian(s.hop_R, s.hop_T)
    g.reset()
    g.step(3)
    with pytest.raises(kbe.KBEError) as e:
        g.step(1)                       # past nt_max
    assert e.value.status == -4
    with pytest.raises(kbe.KBEError) as e:
        g.set_interaction(np.array([np.nan]))
    assert e.value.status == -5
    with pytest.raises(kbe.KBEError):
        g.set_interaction(np.ones(2))   # neither 1 nor nt_max+1 samples
    with pytest.raises(kbe.KBEError):
        g.row(7, 0)
    g.reset()                           # the handle stays usable
    g.step(2)
    g.synchronize()
    g.close()


def test_nonfinite_state_is_sticky_until_reset():
    s = ki.small_system(2, (4, 1), 6, 0.05, 0.7, seed=2)
    g = kbe.KBE.from_system(s)
    g.set_interaction(np.array([1e300]))     # finite input, overflowing dynamics
    g.step(2)
    with pytest.raises(kbe.KBEError) as e:
        g.synchronize()
    assert e.value.status == -5
    with pytest.raises(kbe.KBEError):
        g.step(1)
    g.set_interaction(np.array([0.7]))
    g.reset()
    g.step(2)
    g.synchronize()


def test_dipole_kick_paper_model_every_entry():
    """The paper's two-band model (Sec. 2) with the dipole kick of Eq. 4, on a
    16-site ring so that the oracle runs in seconds."""
    s = ki.config("paper", nt=32)
    s.L = (16, 1)
    compare_trajectory(s, 32)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_checkpoint_resume_is_exact(prec):
    s = ki.small_system(3, (3, 2), 14, 0.05, 0.8, seed=21, drive_amp=0.4)
    a = kbe.KBE.from_system(s, precision=prec)
    a.step(7)
    ck = a.checkpoint()
    a.step(7)
    b = kbe.KBE.from_system(s, precision=prec)
    b.step(2)                            # some other state, overwritten by the restore
    b.restore(ck)
    assert b.n == 7
    b.step(7)
    for i in (3, 7, 10, 14):
        for x in (0, 1):
            assert np.array_equal(a.row(i, x), b.row(i, x)), (i, x)
    assert np.array_equal(a.observables_all()[1], b.observables_all()[1])
    c = kbe.KBE(s.nb, s.dim, (2, 3), s.nt, s.dt, s.beta, s.mu, precision=prec)
    with pytest.raises(kbe.KBEError):
        c.restore(ck)                    # another mesh


@pytest.mark.parametrize("prec", [kbe.KBE_PREC_FP64, kbe.KBE_PREC_DF64, kbe.KBE_PREC_C64])
def test_device_getters_match_host_getters(prec):
    """kbe_get_row_dev / kbe_observables_all_dev write the same values as the
    host getters into caller-owned device tensors: stored rows (unpacked from
    the history's storage) and the two newest FP64 rows, both components"""
    s = ki.config("c2", nt=6)
    g = kbe.KBE.from_system(s, precision=prec)
    g.step(6)
    g.synchronize()
    dev = torch.device("cuda")
    for i in (0, 2, 5, 6):
        for x in (0, 1):
            out = torch.full((i + 1, s.nk, s.nb, s.nb), float("nan"), dtype=torch.complex128, device=dev)
            torch.cuda.synchronize()   # the fill is done before the handle's stream writes
            g.row_dev(i, x, out)
            g.synchronize()
            assert np.array_equal(out.cpu().numpy(), g.row(i, x)), (i, x)
    nkb = torch.empty((7, s.nk, s.nb), dtype=torch.float64, device=dev)
    sc = torch.empty((7, 6), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g.observables_all_dev(nkb, sc)
    g.synchronize()
    nkb_h, sc_h = g.observables_all()
    assert np.array_equal(nkb.cpu().numpy(), nkb_h) and np.array_equal(sc.cpu().numpy(), sc_h)
    g.close()
