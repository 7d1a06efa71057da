"""Fourth-order Gregory weights for the collision integrals (kbe_config.quadrature
= KBE_QUAD_GREGORY): whole trajectories against the oracle with the same weights
(FP64 bar: 1e-10 element-wise, as for the trapezoid runs), the reduced-storage
forms against the FP64 trajectory, and the reverse mode against the oracle's
reference gradient."""
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


@pytest.mark.parametrize("name,nt", [("c1", 24), ("c2", 12)])
def test_gregory_trajectory_matches_oracle(name, nt):
    s = dataclasses.replace(ki.config(name, nt=nt), quadrature=1)
    g = kbe.KBE.from_system(s)
    g.step(nt)
    o = oracle.Oracle(s)
    o.step(nt)
    for i in sorted({1, 2, 4, 5, 6, nt}):
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            e_el, _ = relerr(g.row(i, x), ref[x], scale=scale)
            assert e_el < 1e-10, (i, x, e_el)
    _, sc_g = g.observables_all()
    sc_o = np.stack([o.observables(i)[1] for i in range(nt + 1)])
    assert np.abs(sc_g - sc_o).max() < 1e-10 * np.abs(sc_o).max()
    # the rule matters: the trapezoid trajectory differs well above the bar
    t = kbe.KBE.from_system(dataclasses.replace(s, quadrature=0))
    t.step(nt)
    assert np.abs(t.row(nt, 0) - g.row(nt, 0)).max() > 1e-8
    g.close()
    t.close()


@pytest.mark.parametrize("prec,bar", [("df64", 1e-12), ("c64", 1e-5)])
def test_gregory_reduced_forms(prec, bar):
    s = dataclasses.replace(ki.config("c2", nt=16), quadrature=1)
    f = kbe.KBE.from_system(s)
    f.step(16)
    g = kbe.KBE.from_system(s, precision=kbe.PRECISIONS[prec])
    g.step(16)
    nf, sf = f.observables_all()
    ng, sg = g.observables_all()
    assert np.abs(ng - nf).max() < bar
    assert np.abs(sg[:, 5] - sf[:, 5]).max() < bar * np.abs(sf[:, 5]).max()
    f.close()
    g.close()


def test_gregory_gradient_matches_oracle_reference():
    s = dataclasses.replace(ki.small_system(2, (4, 1), 8, 0.05, 0.8, seed=9, drive_amp=0.5, paper_shift=1,
                                            band_velocity=0.5), quadrature=1)
    tgt = ki.targets(s.nk, s.nb, seed=4)
    g = kbe.KBE.from_system(s)
    g.step(8)
    nkb, _ = g.observables(8)
    dA, dU = g.backward(2.0 * (nkb - tgt))
    g.close()
    rA, rU = og.gradient(s, 8, tgt)
    scale = max(np.abs(rA).max(), abs(rU))
    assert np.abs(dA[:8] - rA).max() < 1e-7 * scale, (dA[:8], rA)
    assert abs(dU - rU) < 1e-7 * scale
