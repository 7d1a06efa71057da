"""The split-FP16 pair history (KBE_PREC_F16X2) and its tensor-core sweep
(tcgen05.mma) against the FP64 oracle.

The history keeps hi = fp16(4096 x), lo = fp16(4096 x - hi) per real part
(22-bit significand); the sweep multiplies the hi and lo parts on the tensor
cores with FP32 accumulation, the coefficient rows split the same way under a
power-of-two scale. Checked here:
  - the storage itself: the packed halves (per k, strips of column blocks,
    each holding its rows as consecutive slots), decoded on the host from the
    documented layout, give back every input to 2^-21 of the scale;
  - per-row collision integrals (Eq. 6) on random histories and self-energy
    rows, for several panels and strips, ragged n, both quadratures and every
    panel height, at the mixed form's bar (1e-5 normwise, 1e-4 element-wise
    above 1e-2 of the scale), bitwise repeatable over two calls;
  - whole trajectories: density and energies within 1e-5 of the oracle.
"""
import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import from_dev_blocks, relerr, to_dev_blocks, tri

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu
P = 3   # KBE_PREC_F16X2


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def packed_f16x2(arr, nb, L, n):
    """a triangle [ntri, 2, nb, nb, nk] of FP64 (G^<, G^>) blocks, rows 0..n ->
    split-FP16 storage (halves)"""
    src = dev(arr)
    dst = torch.empty(kbe.history_bytes(nb, L, n, P) // 2, dtype=torch.float16, device="cuda")
    kbe.pack(P, src, dst, arr.shape[0], arr[0, 0].size, nb=nb, L=L)
    return dst


def decode_f16x2(h, n, nb, nk):
    """host decode of the documented layout for a storage of rows 0..n: per k,
    strips s of TM columns, each holding rows s TM .. n as consecutive slots of
    8 nb^2 TM halves; within a slot [r / 4][part hi/lo][x][block][s][r % 4][re/im]
    -> (G^<, dG) as [ntri, 2, nb, nb, nk] ([x][r][s][k])"""
    tm = 16 if nb == 4 else 8
    slot = 8 * nb * nb * tm
    cap = n + 1
    nstrips = (cap - 1) // tm + 1
    colstart = [st * cap - tm * st * (st - 1) // 2 for st in range(nstrips + 1)]
    kslots = colstart[nstrips]
    assert h.size == nk * kslots * slot
    with np.errstate(invalid="ignore", over="ignore"):   # padding blocks are never written
        v = h.astype(np.float64)
    out = np.zeros(((n + 1) * (n + 2) // 2, 2, nb, nb, nk), np.complex128)
    for k in range(nk):
        for st in range(nstrips):
            for i in range(st * tm, cap):
                o = (k * kslots + colstart[st] + i - st * tm) * slot
                w = v[o:o + slot].reshape(nb // 4, 2, 2, tm, nb, 4, 2)   # [r/4][h][x][block][s][r%4][ri]
                z = (w[:, 0] + w[:, 1]) / 4096.0                          # [r/4][x][block][s][r%4][ri]
                c = (z[..., 0] + 1j * z[..., 1]).transpose(2, 1, 0, 4, 3).reshape(tm, 2, nb, nb)   # [block][x][r][s]
                for jj in range(tm):
                    j = st * tm + jj
                    if j <= i:
                        out[tri(i, j), :, :, :, k] = c[jj]
    return out


@pytest.mark.parametrize("nb,L,n", [(4, (3, 2), 18), (8, (2, 1), 9)])
def test_f16x2_storage_layout_and_accuracy(nb, L, n):
    rng = np.random.default_rng(40 + nb)
    nk = L[0] * L[1]
    m = tri(n, n) + 1
    Xl = ki.random_blocks(rng, (m, nk, nb, nb))
    Xg = ki.random_blocks(rng, (m, nk, nb, nb))
    Xl[0, 0, 0, 0] = 3e-9 + 2e-8j    # tiny entries keep an absolute error of 2^-25 / 4096
    arr = to_dev_blocks(Xl, Xg)
    h = packed_f16x2(arr, nb, L, n).cpu().numpy()
    got = decode_f16x2(h, n, nb, nk)
    want = np.stack([arr[:, 0], arr[:, 0] - arr[:, 1]], axis=1)   # (G^<, dG)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 2.0 ** -21 * scale
    assert abs(got[0, 0, 0, 0, 0] - want[0, 0, 0, 0, 0]) <= 2.0 ** -36


def _collision(nb, L, n, quad, TI, seed, reps=2):
    rng = np.random.default_rng(seed)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=quad)
    H = packed_f16x2(to_dev_blocks(Hl, Hg), nb, L, n)
    S = dev(to_dev_blocks(Sl, Sg))
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, P) // 4 + 1, dtype=torch.float32, device="cuda")
    if TI:
        kbe.set_sweep_choice(nb, L, P, -TI, quadrature=quad)
    try:
        outs = []
        for _ in range(reps):
            I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
            work.fill_(float("nan"))   # nothing may depend on stale scratch
            kbe.collision_row(nb, L, n, dt, H, S, I, precision=P, work=work, quadrature=quad)
            torch.cuda.synchronize()
            outs.append(I.cpu().numpy())
    finally:
        if TI:
            kbe.set_sweep_choice(nb, L, P, 0, quadrature=quad)
    return outs, Il, Ig


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,L,n,TI", [
    (4, (8, 8), 70, 32), (4, (6, 5), 45, 64), (4, (3, 1), 130, 128), (4, (2, 1), 0, 32),
    (4, (2, 1), 1, 32), (4, (2, 1), 6, 64), (4, (5, 1), 17, 16), (8, (4, 4), 40, 32),
    (8, (2, 3), 35, 64), (8, (3, 1), 9, 16), (8, (1, 1), 0, 32), (8, (2, 1), 71, 32),
    (4, (8, 8), 70, 33), (4, (3, 1), 130, 129), (8, (4, 4), 40, 33), (8, (2, 1), 71, 65),
])
def test_f16x2_collision_row_matches_oracle(nb, L, n, TI, quad):
    """several panels (TI rows) and strips, the diagonal strips, odd row counts
    (N_b = 4 pairs rows in one MMA), n below one strip, both copy paths (an odd
    choice TI + 1: loader warps); bitwise repeatable"""
    outs, Il, Ig = _collision(nb, L, n, quad, TI, 1300 + nb * 7 + n)
    assert np.array_equal(outs[0], outs[1])
    gl, gg = from_dev_blocks(outs[0])
    assert np.all(np.isfinite(gl)) and np.all(np.isfinite(gg))
    for got, ref in ((gl, Il), (gg, Ig)):
        el, nw = relerr(got, ref, floor_frac=1e-2)
        assert el < 1e-4 and nw < 1e-5, (el, nw)


def test_f16x2_rejected_where_it_does_not_apply():
    with pytest.raises(kbe.KBEError):
        kbe.KBE(nb=2, dim=1, L=(8, 1), nt_max=4, dt=0.05, beta=10.0, mu=0.0, precision=P)
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(4, (4, 4), P, -24)     # TI not a multiple of 16
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(8, (4, 4), P, -128)    # accumulators beyond tensor memory
    with pytest.raises(kbe.KBEError):
        kbe.pack(P, torch.zeros(2, dtype=torch.complex128, device="cuda"),
                 torch.zeros(8, dtype=torch.float16, device="cuda"), 0, 4)   # needs the mesh


@pytest.mark.parametrize("name,nsteps", [("c2", 40)])
def test_f16x2_density_and_energy_within_1e5(name, nsteps):
    s = ki.config(name, nt=nsteps)
    g = kbe.KBE.from_system(s, precision=P)
    g.step(nsteps)
    nkb, sc = g.observables_all()
    g.close()
    o = oracle.Oracle(s)
    o.step(nsteps)
    for n in range(nsteps + 1):
        nkb_o, sc_o = o.observables(n)
        assert np.abs(nkb[n] - nkb_o).max() <= 1e-5 * np.abs(nkb_o).max(), n
        escale = max(abs(sc_o[1]), abs(sc_o[5]))
        assert np.abs(sc[n][1:] - sc_o[1:]).max() <= 1e-5 * escale, (n, sc[n], sc_o)


@pytest.mark.parametrize("nb,L,drive", [(4, (3, 3), 0.5), (8, (2, 2), 0.3)])
def test_f16x2_small_systems_and_readback(nb, L, drive):
    """small driven systems: observables within 1e-5, and the stored history
    read back through kbe_get_row (host decode of the split pairs)"""
    s = ki.small_system(nb, L, 12, 0.05, 0.8, seed=nb * 11, drive_amp=drive)
    g = kbe.KBE.from_system(s, precision=P)
    g.step(12)
    o = oracle.Oracle(s)
    o.step(12)
    for i in (2, 6, 11):   # rows older than the two FP64 working rows come from the history
        ref = [o.row(i, 0), o.row(i, 1)]
        scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
        for x in (0, 1):
            _, nw = relerr(g.row(i, x), ref[x], scale=scale)
            assert nw < 1e-5, (i, x, nw)
    nkb, sc = g.observables_all()
    g.close()
    for n in range(13):
        nkb_o, sc_o = o.observables(n)
        assert np.abs(nkb[n] - nkb_o).max() <= 1e-5 * max(np.abs(nkb_o).max(), 1e-3), n
        escale = max(abs(sc_o[1]), abs(sc_o[5]))
        assert np.abs(sc[n][1:] - sc_o[1:]).max() <= 1e-5 * escale, (n, sc[n], sc_o)
