"""Batched independent systems of uneven N_b, n_k and N_t (kbe_batch_*):
every system of the batch must match its own oracle run entry by entry, each
system stops at its own nt_max, and admission follows the memory budget. The
persistent mode (the sweeps of all systems in one launch per N_b class, steps
enqueued stage-major) must give the stream-ordered batch's rows bit for bit."""
import dataclasses

import numpy as np
import pytest

import kbe_inputs as ki
import oracle
from layout import relerr

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu


def uneven_batch():
    specs = [(1, (5, 1), 5, 0.4), (2, (8, 1), 12, 0.0), (3, (3, 3), 8, 0.5), (4, (4, 3), 6, 0.3),
             (8, (2, 2), 4, 0.2), (2, (1, 1), 9, 0.0)]
    return [ki.small_system(nb, L, nt, 0.05, 0.9, seed=40 + i, drive_amp=amp)
            for i, (nb, L, nt, amp) in enumerate(specs)]


@pytest.mark.parametrize("prec,el_tol", [(0, 1e-10), (1, 5e-10)])
def test_batch_matches_oracle_per_system(prec, el_tol):
    systems = uneven_batch()
    b = kbe.KBEBatch(systems, precision=prec)
    assert all(b.admitted)
    b.reset()
    b.step(7)
    b.step(10)            # systems with nt_max < 17 stop at their own end
    b.synchronize()
    for s, g in zip(systems, b.systems):
        assert g.n == s.nt
        o = oracle.Oracle(s)
        o.step(s.nt)
        for i in (1, s.nt // 2, s.nt):
            ref = [o.row(i, 0), o.row(i, 1)]
            scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
            for x in (0, 1):
                assert relerr(g.row(i, x), ref[x], scale=scale)[0] < el_tol, (s.name, i, x)
        nkb, sc = g.observables_all()
        assert np.abs(sc[s.nt] - o.observables(s.nt)[1]).max() < 1e-10
    b.close()


def test_batch_admission_by_memory_budget():
    systems = uneven_batch()
    need = [kbe.memory_bytes(kbe.system_config(s)) for s in systems]
    budget = need[0] + need[1] + need[2] // 2          # the third does not fit
    b = kbe.KBEBatch(systems, budget_bytes=budget)
    assert b.admitted[:2] == [True, True] and not b.admitted[2]
    assert b.systems[2] is None
    b.reset()
    b.step(3)
    b.synchronize()
    assert b.systems[0].n == 3 and b.systems[1].n == 3
    b.close()


def test_batch_graphs_match_eager_bitwise():
    """graph mode (one replayed graph per system and call) runs the same kernels
    with the same arguments: rows equal the stream-ordered batch bit for bit,
    also across a second reset and an uneven stop"""
    systems = uneven_batch()
    a = kbe.KBEBatch(systems)
    g = kbe.KBEBatch(systems)
    g.set_graphs(True)
    for rep in range(2):
        a.reset()
        g.reset()
        for k in (5, 9):
            a.step(k)
            g.step(k)
        a.synchronize()
        g.synchronize()
        for s, x, y in zip(systems, a.systems, g.systems):
            assert x.n == y.n == min(14, s.nt)
            for i in (1, x.n // 2, x.n):
                for c in (0, 1):
                    assert np.array_equal(x.row(i, c), y.row(i, c)), (rep, s.name, i, c)
    a.close()
    g.close()


def test_batch_wide_graph_on_a_stream_matches_eager_bitwise():
    """on a non-default stream the whole batch step is one captured graph:
    rows equal the stream-ordered batch bit for bit, across resets, uneven
    stops, and a drive changed on one system between calls (which must drop
    the captured graph)"""
    systems = uneven_batch()
    st = torch.cuda.Stream()
    a = kbe.KBEBatch(systems, stream=st)
    g = kbe.KBEBatch(systems, stream=st)
    g.set_graphs(True)
    for rep in range(3):
        if rep == 2:   # new drive samples on system 0 (a driven one) of both batches
            assert systems[0].A is not None
            for bb in (a, g):
                bb.systems[0].set_drive(np.asarray(systems[0].A) * 0.5)
        a.reset()
        g.reset()
        for k in (5, 9):
            a.step(k)
            g.step(k)
        a.synchronize()
        g.synchronize()
        st.synchronize()
        for s, x, y in zip(systems, a.systems, g.systems):
            assert x.n == y.n == min(14, s.nt)
            for i in (1, x.n // 2, x.n):
                for c in (0, 1):
                    assert np.array_equal(x.row(i, c), y.row(i, c)), (rep, s.name, i, c)
    a.close()
    g.close()


def persistent_batch():
    """the uneven batch with a 4-corrector system, a Gregory-weighted one and an
    early-converging one (Algorithm 1's epsilon: skipped passes), plus the
    N_b = 6, 12, 16 classes of the uneven draw"""
    base = uneven_batch()
    base[1] = dataclasses.replace(base[1], n_corr=3)
    base[2] = dataclasses.replace(base[2], quadrature=1)
    base[3] = dataclasses.replace(base[3], n_corr=4, corr_tol=1e-9)
    extra = [ki.small_system(6, (2, 2), 6, 0.05, 0.9, seed=50, drive_amp=0.3),
             ki.small_system(12, (2, 1), 5, 0.05, 0.7, seed=51),
             ki.small_system(16, (1, 1), 4, 0.05, 0.6, seed=52, drive_amp=0.2)]
    return base + extra


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_persistent_matches_stream_ordered_bitwise(graphs):
    """every stored row of every system equals the stream-ordered batch's bit
    for bit (the batched launch runs each system's blocks with the same split
    and arithmetic), across a reset and uneven stops, eager and captured"""
    systems = persistent_batch()
    st = torch.cuda.Stream()
    a = kbe.KBEBatch(systems, stream=st)
    p = kbe.KBEBatch(systems, stream=st)
    p.set_persistent(True)
    if graphs:
        p.set_graphs(True)
    for rep in range(2):
        a.reset()
        p.reset()
        for k in (5, 9):
            a.step(k)
            p.step(k)
        a.synchronize()
        p.synchronize()
        st.synchronize()
        for s, x, y in zip(systems, a.systems, p.systems):
            assert x.n == y.n == min(14, s.nt)
            for i in range(1, x.n + 1):
                for c in (0, 1):
                    assert np.array_equal(x.row(i, c), y.row(i, c)), (rep, s.name, i, c)
            assert np.array_equal(x.corrector_iterations(), y.corrector_iterations())
            assert np.array_equal(x.observables_all()[1], y.observables_all()[1])
    if graphs:
        assert p.sweep_launches() == 0          # replayed, not enqueued eagerly
    else:
        # at most one launch per N_b class (f64m: 1, 2, 3, 4, 6, 8; plain: 12, 16) and
        # quadrature per cut; 14 steps of at most n_corr + 1 = 5 cuts per call
        assert 0 < p.sweep_launches() <= 2 * 14 * 5 * 9
    a.close()
    p.close()


def test_batch_persistent_matches_oracle_per_system():
    systems = persistent_batch()
    b = kbe.KBEBatch(systems)
    b.set_persistent(True)
    b.reset()
    b.step(7)
    b.step(10)
    b.synchronize()
    for s, g in zip(systems, b.systems):
        assert g.n == s.nt
        o = oracle.Oracle(s)
        o.step(s.nt)
        for i in (1, s.nt // 2, s.nt):
            ref = [o.row(i, 0), o.row(i, 1)]
            scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
            for x in (0, 1):
                assert relerr(g.row(i, x), ref[x], scale=scale)[0] < 1e-10, (s.name, i, x)
        nkb, sc = g.observables_all()
        assert np.abs(sc[s.nt] - o.observables(s.nt)[1]).max() < 1e-10
    b.close()


def test_batch_persistent_needs_fp64_histories():
    systems = uneven_batch()[:2]
    b = kbe.KBEBatch(systems, precision=1)
    with pytest.raises(kbe.KBEError):
        b.set_persistent(True)
    b.close()
