"""Per-row parity of the CUDA path with the FP64 oracle on seeded inputs.

Each test calls one stateless C-ABI operation (a1 Sigma row, a2 collision
row, a3 propagators, a4 row update) on device buffers and compares every
output element with the oracle on the same inputs. Sizes span several CTAs
and ragged tails (n_k not a multiple of the block, odd meshes, N_b in every
compiled value).
"""
import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import from_dev_blocks, from_dev_perk, relerr, to_dev_blocks, to_dev_perk, tri

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu
TOL = 1e-12   # FP64 vs FP64, different summation order: normwise, of the largest |ref|
EL_TOL = 1e-10   # element-wise, |d| / max(|ref|, 1e-4 of the largest |ref|)


def assert_close(got, ref, prec="fp64", norm=None):
    """element-wise and normwise bars of one output array against the oracle.
    FP64 / DF64: 1e-10 element-wise (floor 1e-4 of the array's scale) and the
    normwise bar; C64: 1e-4 element-wise above 1e-2 of the scale (complex64
    storage rounds each input at 6e-8) and 1e-5 normwise."""
    if prec == "c64":
        el, nw = relerr(got, ref, floor_frac=1e-2)
        assert el < 1e-4 and nw < (1e-5 if norm is None else norm), (el, nw)
    else:
        el, nw = relerr(got, ref)
        assert el < EL_TOL and nw < (TOL if norm is None else norm), (el, nw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nb,L,n,Uvar", [
    (2, (8, 1), 9, False), (4, (8, 8), 13, True), (3, (5, 3), 6, False), (1, (7, 1), 4, False),
    (6, (3, 2), 3, True), (8, (4, 4), 2, False), (12, (2, 2), 1, False), (16, (2, 1), 1, False),
    (2, (1, 1), 0, False), (4, (37, 1), 5, False),
])
def test_sigma_row_matches_oracle(nb, L, n, Uvar):
    rng = np.random.default_rng(100 + nb * 7 + n)
    nk = L[0] * L[1]
    Gl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Gg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    v = ki.pair_pattern(nb) if nb != 3 else rng.uniform(0, 1, (nb, nb))
    Un = 0.9
    Ul = rng.uniform(0.5, 1.5, n + 1) if Uvar else np.full(n + 1, Un)
    Grow = dev(to_dev_blocks(Gl, Gg))
    Sig = torch.empty_like(Grow)
    work = torch.empty(kbe.sigma_row_workspace(nb, L, n) // 16 + 1, dtype=torch.complex128, device="cuda")
    kbe.sigma_row(nb, L, v, n, Un, Grow, Sig, work, Ul=dev(Ul) if Uvar else None)
    torch.cuda.synchronize()
    Sl, Sg = from_dev_blocks(Sig.cpu().numpy())
    for l in range(n + 1):
        ol, og = oracle.sigma_pair(nb, L, v, Un * Ul[l], Gl[l], Gg[l])
        assert_close(Sl[l], ol)
        assert_close(Sg[l], og)


@pytest.mark.parametrize("nb,L,n", [
    (1, (5, 1), 7), (2, (8, 1), 0), (2, (8, 1), 1), (2, (8, 1), 23), (3, (3, 3), 11),
    (4, (8, 8), 17), (4, (7, 5), 9), (6, (3, 1), 6), (8, (2, 3), 5), (12, (2, 1), 3), (16, (1, 3), 2),
])
def test_collision_row_matches_oracle(nb, L, n):
    rng = np.random.default_rng(200 + nb * 13 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg)
    H64 = dev(to_dev_blocks(Hl, Hg))
    H = torch.empty_like(H64)
    kbe.pack(kbe.KBE_PREC_FP64, H64, H, ntri, nb * nb * nk)
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    work = torch.empty(kbe.collision_row_workspace(nb, L, n) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, work=work)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    assert_close(gl, Il)
    assert_close(gg, Ig)


@pytest.mark.parametrize("prec", ["fp64", "df64", "c64"])
@pytest.mark.parametrize("nb,L,n", [(2, (8, 1), 1), (2, (8, 1), 2), (3, (3, 3), 4), (4, (8, 8), 5),
                                    (4, (7, 5), 23), (2, (8, 1), 40)])
def test_gregory_collision_row_matches_oracle(nb, L, n, prec):
    """the Gregory weights (start rules for n <= 4, end corrections beyond) in all
    three arithmetic forms; the l range is split over CTAs at the larger n"""
    rng = np.random.default_rng(300 + nb * 13 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=1)
    p = kbe.PRECISIONS[prec]
    H64 = dev(to_dev_blocks(Hl, Hg))
    esz = 8 if prec == "c64" else 16
    H = torch.empty(H64.numel() * esz // 4, dtype=torch.float32, device="cuda")
    kbe.pack(p, H64, H, ntri, nb * nb * nk)
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, p) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, precision=p, work=work, quadrature=1)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    assert_close(gl, Il, prec)
    assert_close(gg, Ig, prec)


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,L,n", [(8, (2, 3), 9), (8, (5, 2), 6), (16, (1, 6), 4), (4, (2, 3), 7),
                                    (4, (13, 2), 12), (8, (4, 4), 40)])
def test_c64_staged_sweep_ragged_tiles(nb, L, n, quad):
    """the staged C64 sweep (N_b >= 4, n_k even) with k-tiles that run past n_k
    (zero-filled copies) and with split l ranges, against the oracle"""
    rng = np.random.default_rng(400 + nb * 7 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=quad)
    p = kbe.KBE_PREC_C64
    H64 = dev(to_dev_blocks(Hl, Hg))
    H = torch.empty(H64.numel() * 2, dtype=torch.float32, device="cuda")
    kbe.pack(p, H64, H, ntri, nb * nb * nk)
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, p) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, precision=p, work=work, quadrature=quad)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    assert np.all(np.isfinite(gl)) and np.all(np.isfinite(gg))
    assert_close(gl, Il, "c64")
    assert_close(gg, Ig, "c64")


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,L,n", [(1, (7, 1), 5), (2, (8, 1), 0), (2, (129, 1), 9), (2, (3, 3), 1),
                                    (2, (300, 1), 40), (1, (131, 1), 33)])
def test_c64_blocked_sweep_small_nb(nb, L, n, quad):
    """the register-blocked C64 sweep (N_b <= 2, one thread per k owning every
    (a, b)): odd n_k leave the last CTA ragged, and the larger rows split the l
    range over CTAs; against the oracle at the mixed form's bar"""
    rng = np.random.default_rng(500 + nb * 7 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=quad)
    p = kbe.KBE_PREC_C64
    H64 = dev(to_dev_blocks(Hl, Hg))
    H = torch.empty(H64.numel() * 2, dtype=torch.float32, device="cuda")
    kbe.pack(p, H64, H, ntri, nb * nb * nk)
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, p) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, precision=p, work=work, quadrature=quad)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    assert np.all(np.isfinite(gl)) and np.all(np.isfinite(gg))
    assert_close(gl, Il, "c64")
    assert_close(gg, Ig, "c64")


def _herm_batch(rng, nk, nb, scale=1.5):
    a = ki.random_blocks(rng, (nk, nb, nb), scale)
    return 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))


@pytest.mark.parametrize("nb,nk,dt,scale", [(1, 3, 0.02, 1.5), (2, 65, 0.02, 1.5), (4, 64, 0.02, 1.5),
                                         (6, 7, 0.02, 1.5), (8, 33, 0.05, 3.0), (12, 5, 0.02, 1.5),
                                         (16, 3, 0.02, 1.5), (4, 9, 0.7, 4.0), (3, 5, 2.5, 8.0)])
def test_propagators_match_oracle(nb, nk, dt, scale):
    """U, V against the oracle's eigen-decomposition route; the last two cases
    have dt ||h|| >> 1 and exercise the doublings."""
    rng = np.random.default_rng(300 + nb)
    h = _herm_batch(rng, nk, nb, scale)
    h[0] = np.diag(np.linspace(-1, 1, nb))                     # already diagonal
    if nb >= 2:
        h[1] = np.diag(np.r_[np.zeros(nb - 1), 0.7])           # degenerate zero eigenvalues
    U, V, W, lam = oracle.propagators(nb, nk, dt, h)
    L = (nk, 1)
    hd = dev(to_dev_perk(h))
    Ud, Vd = torch.empty_like(hd), torch.empty_like(hd)
    kbe.propagators(nb, L, dt, hd, Ud, Vd)
    torch.cuda.synchronize()
    Ug, Vg = (from_dev_perk(x.cpu().numpy()) for x in (Ud, Vd))
    tol = 1e-13 * max(1.0, dt * scale * nb)
    assert np.abs(Ug - U).max() < tol
    assert np.abs(Vg - V).max() < tol * max(dt, 1.0)


@pytest.mark.parametrize("nb,nk,n,theta,dt", [(2, 8, 1, 0.0, 0.04), (2, 8, 9, 0.5, 0.04),
                                              (4, 64, 6, 0.5, 0.04), (3, 9, 4, 0.0, 0.04),
                                              (8, 5, 3, 0.5, 0.04), (16, 2, 2, 0.5, 0.04),
                                              (4, 7, 3, 0.5, 0.9)])
def test_update_row_matches_oracle(nb, nk, n, theta, dt):
    rng = np.random.default_rng(400 + nb + n)
    h = _herm_batch(rng, nk, nb)
    U, V, W, lam = oracle.propagators(nb, nk, dt, h)
    Gpl = ki.random_blocks(rng, (n, nk, nb, nb))
    Gpg = ki.random_blocks(rng, (n, nk, nb, nb))
    Ipl = ki.random_blocks(rng, (n, nk, nb, nb))
    Ipg = ki.random_blocks(rng, (n, nk, nb, nb))
    Icl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Icg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    ol, og = oracle.update_row(nb, nk, n, dt, theta, U, V, W, lam, Gpl, Gpg, Ipl, Ipg, Icl, Icg)
    L = (nk, 1)
    out = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    kbe.update_row(nb, L, n, dt, theta, dev(to_dev_perk(h)), dev(to_dev_perk(U)), dev(to_dev_perk(V)),
                   dev(to_dev_blocks(Gpl, Gpg)), dev(to_dev_blocks(Ipl, Ipg)), dev(to_dev_blocks(Icl, Icg)),
                   out)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(out.cpu().numpy())
    assert_close(gl, ol, norm=1e-13)
    assert_close(gg, og, norm=1e-13)


@pytest.mark.parametrize("prec", ["fp64", "df64", "c64"])
def test_collision_row_paper_shape(prec):
    """the paper's two-band ring extent, n_k = 1024 (N_b = 2, the C64 form's
    register-blocked kernel and the per-element FP64 / DF64 kernels), at row
    n = 64 with the l range split over CTAs, on random history"""
    nb, L, n, dt = 2, (1024, 1), 64, 0.02
    rng = np.random.default_rng(600)
    nk = L[0] * L[1]
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg)
    p = kbe.PRECISIONS[prec]
    H64 = dev(to_dev_blocks(Hl, Hg))
    esz = 8 if prec == "c64" else 16
    H = torch.empty(H64.numel() * esz // 4, dtype=torch.float32, device="cuda")
    kbe.pack(p, H64, H, ntri, nb * nb * nk)
    del H64
    S = dev(to_dev_blocks(Sl, Sg))
    I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, p) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.collision_row(nb, L, n, dt, H, S, I, precision=p, work=work)
    torch.cuda.synchronize()
    gl, gg = from_dev_blocks(I.cpu().numpy())
    assert_close(gl, Il, prec)
    assert_close(gg, Ig, prec)


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,L,n,TI", [(4, (8, 8), 70, 32), (4, (6, 5), 45, 64), (8, (4, 4), 40, 32),
                                       (8, (2, 3), 35, 128), (2, (64, 1), 70, 32), (2, (30, 1), 33, 128),
                                       (4, (2, 1), 0, 32), (4, (2, 1), 1, 32), (4, (2, 1), 6, 32)])
def test_c64_tile_sweep_matches_oracle(nb, L, n, TI, quad):
    """the single-read tile sweep (each stored block read once, both uses from
    shared memory; kbe_set_sweep_choice forces it on every row): several column
    strips and row chunks, k-tiles that run past n_k, the diagonal and end
    nodes, both quadratures; against the oracle at the mixed form's bar, and
    bitwise repeatable (the partial sums are added in a fixed order)"""
    rng = np.random.default_rng(900 + nb * 7 + n)
    nk = L[0] * L[1]
    dt = 0.03
    ntri = tri(n, n) + 1
    Hl = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Hg = ki.random_blocks(rng, (ntri, nk, nb, nb))
    Sl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Sg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Il, Ig = oracle.collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=quad)
    p = kbe.KBE_PREC_C64
    H64 = dev(to_dev_blocks(Hl, Hg))
    H = torch.empty(H64.numel() * 2, dtype=torch.float32, device="cuda")
    kbe.pack(p, H64, H, ntri, nb * nb * nk)
    S = dev(to_dev_blocks(Sl, Sg))
    work = torch.empty(kbe.collision_row_workspace(nb, L, n, p) // 4 + 1, dtype=torch.float32, device="cuda")
    kbe.set_sweep_choice(nb, L, p, -TI, quadrature=quad)
    try:
        outs = []
        for _ in range(2):
            I = torch.full((n + 1, 2, nb, nb, nk), float("nan"), dtype=torch.complex128, device="cuda")
            work.fill_(float("nan"))   # nothing may depend on stale scratch
            kbe.collision_row(nb, L, n, dt, H, S, I, precision=p, work=work, quadrature=quad)
            torch.cuda.synchronize()
            outs.append(I.cpu().numpy())
    finally:
        kbe.set_sweep_choice(nb, L, p, 0, quadrature=quad)
    assert np.array_equal(outs[0], outs[1])
    gl, gg = from_dev_blocks(outs[0])
    assert np.all(np.isfinite(gl)) and np.all(np.isfinite(gg))
    assert_close(gl, Il, "c64")
    assert_close(gg, Ig, "c64")


def test_c64_tile_sweep_rejected_where_it_does_not_apply():
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(3, (4, 4), kbe.KBE_PREC_C64, -32)      # N_b = 3
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(4, (5, 3), kbe.KBE_PREC_C64, -32)      # odd n_k
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(4, (4, 4), kbe.KBE_PREC_FP64, -32)     # FP64 history
    with pytest.raises(kbe.KBEError):
        kbe.set_sweep_choice(4, (4, 4), kbe.KBE_PREC_C64, -16)      # TI below 32
