"""Graph replay of kbe_step (kbe_set_graphs): the captured and replayed steps
give the same bits as the ordinary launches, across resets, odd step counts,
input changes (which drop the graphs), the tolerance-driven correctors and a
restored checkpoint."""
import dataclasses

import numpy as np
import pytest

import kbe_inputs as ki

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu


def run(s, nsteps, graphs, stream, chunks=None, **over):
    g = kbe.KBE.from_system(s, stream=stream, **over)
    g.set_graphs(graphs)
    out = []
    for rep in range(2):   # the second pass replays the captured graphs
        g.reset()
        for k in (chunks or [nsteps]):
            g.step(k)
        out.append((g.row(nsteps, 0), g.row(nsteps, 1), g.observables_all()[1]))
    g.close()
    return out


@pytest.mark.parametrize("name,nsteps,chunks", [("c1", 24, None), ("c1", 23, [7, 9, 7]), ("c2", 12, [5, 7])])
def test_graph_replay_is_bitwise_identical(name, nsteps, chunks):
    s = ki.config(name, nt=nsteps)
    st = torch.cuda.Stream()
    ref = run(s, nsteps, False, st, chunks)
    got = run(s, nsteps, True, st, chunks)
    for r in (0, 1):
        for a, b in zip(ref[r], got[r]):
            assert np.array_equal(a, b)


def test_graphs_follow_input_changes_and_checkpoints():
    s = ki.small_system(2, (6, 1), 10, 0.05, 0.8, seed=3, drive_amp=0.4, band_velocity=0.3)
    st = torch.cuda.Stream()
    g = kbe.KBE.from_system(s, stream=st)
    g.set_graphs(True)
    g.step(10)
    first = g.row(10, 0)
    g.set_drive(s.A * 1.5, s.direction)        # drops the graphs
    g.reset()
    g.step(10)
    h = kbe.KBE.from_system(dataclasses.replace(s, A=s.A * 1.5), stream=st)
    h.step(10)
    assert np.array_equal(g.row(10, 0), h.row(10, 0))
    assert not np.array_equal(first, g.row(10, 0))
    # checkpoint at row 4, restore, replay the rest through graphs
    g.reset()
    g.step(4)
    blob = g.checkpoint()
    g.step(6)
    end = g.row(10, 1)
    g.restore(blob)
    g.step(6)
    assert np.array_equal(g.row(10, 1), end)
    g.close()
    h.close()


def test_graphs_with_tolerance_correctors():
    s = dataclasses.replace(ki.config("c1", nt=24), n_corr=4, corr_tol=1.19e-10)
    st = torch.cuda.Stream()
    ref = run(s, 24, False, st)
    got = run(s, 24, True, st)
    for a, b in zip(ref[1], got[1]):
        assert np.array_equal(a, b)
