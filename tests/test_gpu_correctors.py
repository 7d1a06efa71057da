"""Algorithm 1's corrector loop with its epsilon (kbe_config.corr_tol): at most
n_corr passes, ending once the largest change of the new G^< row is <= epsilon.
The decision is taken on the device (no host round trip inside a step); the
oracle takes it on the CPU from its own row. Both must take the same number of
passes at every step (the tolerance is chosen with >= 2.5 % margin to every
per-step decision, tests/test_oracle_pins.py), and the rows must agree to the
FP64 bar."""
import dataclasses

import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import relerr
from oracle import gradient as og

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu
TOL_C1 = 1.19e-10


def test_pass_counts_and_rows_match_the_oracle():
    s = dataclasses.replace(ki.config("c1", nt=24), n_corr=4, corr_tol=TOL_C1)
    g = kbe.KBE.from_system(s)
    g.step(24)
    o = oracle.Oracle(s)
    o.step(24)
    it_g, it_o = g.corrector_iterations(), o.iterations()
    assert it_g.tolist() == it_o.tolist()
    assert set(it_g[1:].tolist()) == {3, 4}
    for i in (5, 6, 7, 24):
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            e_el, _ = relerr(g.row(i, x), ref[x], scale=scale)
            assert e_el < 1e-10, (i, x, e_el)
    g.close()


def test_limits_reproduce_fixed_counts_bitwise():
    s = ki.config("c1", nt=10)
    runs = {}
    for name, nc, tol in (("fixed3", 3, 0.0), ("tiny", 3, 1e-300), ("one", 1, 0.0), ("huge", 3, 1e30)):
        g = kbe.KBE.from_system(dataclasses.replace(s, n_corr=nc, corr_tol=tol))
        g.step(10)
        runs[name] = (g.corrector_iterations(), [g.row(10, 0), g.row(10, 1)], g.observables_all()[1])
        g.close()
    assert runs["tiny"][0].tolist() == [0] + [3] * 10
    assert runs["huge"][0].tolist() == [0] + [1] * 10
    for a, b in (("tiny", "fixed3"), ("huge", "one")):
        for x in (0, 1):
            assert np.array_equal(runs[a][1][x], runs[b][1][x]), (a, b, x)
        assert np.array_equal(runs[a][2], runs[b][2])


@pytest.mark.parametrize("prec", ["df64", "c64"])
def test_reduced_forms_take_a_valid_number_of_passes(prec):
    s = dataclasses.replace(ki.config("c2", nt=12), n_corr=4, corr_tol=1e-9)
    g = kbe.KBE.from_system(s, precision=kbe.PRECISIONS[prec])
    g.step(12)
    it = g.corrector_iterations()
    assert it[0] == 0 and np.all((it[1:] >= 1) & (it[1:] <= 4))
    f = kbe.KBE.from_system(s)
    f.step(12)
    d = np.abs(g.observables_all()[0] - f.observables_all()[0]).max()
    assert d < (1e-12 if prec == "df64" else 1e-6), d
    g.close()
    f.close()


def test_gradient_replays_the_pass_counts():
    """kbe_backward differentiates the steps as they ran: the counts are fixed
    (piecewise constant in the parameters); dL/dU against the oracle's reference"""
    s = dataclasses.replace(ki.config("c1", nt=24), n_corr=4, corr_tol=TOL_C1)
    tgt = ki.targets(s.nk, s.nb, seed=4)
    g = kbe.KBE.from_system(s)
    g.step(24)
    nkb, _ = g.observables(24)
    _, dU = g.backward(2.0 * (nkb - tgt))
    g.close()
    rU = og.directional(s, 24, tgt, dU=1.0, h=1e-4)
    assert abs(dU - rU) < 1e-7 * abs(rU), (dU, rU)


def test_checkpoint_keeps_pass_counts():
    s = dataclasses.replace(ki.config("c1", nt=16), n_corr=4, corr_tol=TOL_C1)
    a = kbe.KBE.from_system(s)
    a.step(8)
    blob = a.checkpoint()
    b = kbe.KBE.from_system(s)
    b.restore(blob)
    a.step(8)
    b.step(8)
    assert a.corrector_iterations().tolist() == b.corrector_iterations().tolist()
    assert np.array_equal(a.row(16, 0), b.row(16, 0))
