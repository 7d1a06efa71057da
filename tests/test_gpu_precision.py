"""The two reduced-storage forms of the history against the FP64 oracle.

DF64 (FP32 hi/lo pairs = 48-bit significands, double-float sweep on the FP32
pipe) is checked at its stated accuracy: 1e-12 normwise on every stored row,
5e-10 element-wise with the 1e-4 zero-entry floor, observables to 1e-11. (On
the c1 ring it reaches 1.0e-10 element-wise: a nearly filled band has
|G^>| ~ 1e-9 built from O(1) terms of I^> that cancel, and 2^-48 storage
leaves ~1e-14 of them; the FP64 form keeps ~1e-16.) C64 (complex64 history,
FP32 sweep with a compensated sum; everything else FP64) must meet the
mixed-precision bar: 1e-5 relative in density and energy.
"""
import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import from_dev_blocks, relerr, to_dev_blocks, tri

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def packed(prec, arr):
    """[m, 2, nb, nb, nk] FP64 (G^<, G^>) blocks -> packed (G^<, dG) storage"""
    src = dev(arr)
    nbytes = 8 if prec == kbe.KBE_PREC_C64 else 16
    dst = torch.empty(src.numel() * nbytes // 4, dtype=torch.float32, device="cuda")
    kbe.pack(prec, src, dst, arr.shape[0], arr[0, 0].size)
    return dst


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (2, 5e-6)])
@pytest.mark.parametrize("nb,L,n", [(1, (5, 1), 7), (2, (8, 1), 0), (2, (8, 1), 23), (3, (3, 3), 11),
                                    (4, (8, 8), 17), (6, (3, 1), 6), (8, (2, 3), 5), (16, (1, 3), 2)])
def test_collision_row_reduced_storage(prec, tol, nb, L, n):
    rng = np.random.default_rng(700 + nb * 13 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg)
    H = packed(prec, to_dev_blocks(Hl, Hg))
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    ws = kbe.collision_row_workspace(nb, L, n, prec)
    work = torch.empty(ws // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, precision=prec, work=work)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    # normwise bar, and element-wise: DF64 1e-10 above 1e-4 of the scale,
    # C64 1e-4 above 1e-2 of it (complex64 rounds every stored input at 6e-8)
    floor, el_bar = (1e-4, 1e-10) if prec == 1 else (1e-2, 1e-4)
    for got, ref in ((gl, Il), (gg, Ig)):
        el, nw = relerr(got, ref, floor_frac=floor)
        assert nw < tol and el < el_bar, (el, nw)


def _trajectory(sys, prec, nsteps):
    g = kbe.KBE.from_system(sys, precision=prec)
    g.step(nsteps)
    g.synchronize()
    o = oracle.Oracle(sys)
    o.step(nsteps)
    return g, o


DF64_EL, DF64_NORM, DF64_OBS = 5e-10, 1e-12, 1e-11


@pytest.mark.parametrize("name,nsteps", [("c1", 64), ("c2", 20)])
def test_df64_trajectory_every_entry(name, nsteps):
    s = ki.config(name)
    g, o = _trajectory(s, kbe.KBE_PREC_DF64, nsteps)
    for i in range(nsteps + 1):
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            el, nw = relerr(g.row(i, x), ref[x], scale=scale)
            assert el < DF64_EL and nw < DF64_NORM, (i, x, el, nw)
    nkb, sc = g.observables_all()
    for n in range(nsteps + 1):
        assert np.abs(sc[n] - o.observables(n)[1]).max() < DF64_OBS


@pytest.mark.parametrize("nb,L,drive", [(3, (3, 3), 0.5), (6, (2, 3), 0.2), (16, (1, 2), 0.0)])
def test_df64_small_systems(nb, L, drive):
    s = ki.small_system(nb, L, 8, 0.05, 0.8, seed=nb * 5, drive_amp=drive)
    g, o = _trajectory(s, kbe.KBE_PREC_DF64, 8)
    for i in (1, 4, 7, 8):
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            el, nw = relerr(g.row(i, x), ref[x], scale=scale)
            assert el < DF64_EL and nw < DF64_NORM, (i, x, el, nw)


@pytest.mark.parametrize("name,nsteps", [("c1", 64), ("c2", 40)])
def test_c64_density_and_energy_within_1e5(name, nsteps):
    s = ki.config(name)
    g, o = _trajectory(s, kbe.KBE_PREC_C64, nsteps)
    nkb, sc = g.observables_all()
    for n in range(nsteps + 1):
        nkb_o, sc_o = o.observables(n)
        assert np.abs(nkb[n] - nkb_o).max() <= 1e-5 * np.abs(nkb_o).max(), n
        # energies: relative to the total energy scale of the system
        escale = max(abs(sc_o[1]), abs(sc_o[5]))
        assert np.abs(sc[n][1:] - sc_o[1:]).max() <= 1e-5 * escale, (n, sc[n], sc_o)
        assert abs(sc[n][0] - sc_o[0]) <= 1e-5 * abs(sc_o[0])


def test_c64_tile_sweep_trajectory_matches_oracle():
    """c2's first 20 steps in the complex64 form with the single-read tile sweep
    forced on every row: density and energies within 1e-5 of the oracle"""
    s = ki.config("c2", nt=20)
    kbe.set_sweep_choice(s.nb, s.L, kbe.KBE_PREC_C64, -32)
    try:
        g = kbe.KBE.from_system(s, precision=kbe.KBE_PREC_C64)
        g.step(20)
        nkb, sc = g.observables_all()
        g.close()
    finally:
        kbe.set_sweep_choice(s.nb, s.L, kbe.KBE_PREC_C64, 0)
    o = oracle.Oracle(s)
    o.step(20)
    nkb_o = np.array([o.observables(i)[0] for i in range(21)])
    sc_o = np.array([o.observables(i)[1] for i in range(21)])
    assert np.abs(nkb - nkb_o).max() <= 1e-5 * np.abs(nkb_o).max()
    assert np.abs(sc[:, 1:] - sc_o[:, 1:]).max() <= 1e-5 * np.abs(sc_o[:, 5]).max()
