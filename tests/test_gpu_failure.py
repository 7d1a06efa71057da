"""Failure detection without a GPU fault: a one-shot injection makes one CTA of
the staged C64 sweep omit its first node's TMA copies. Its waits on the
stage's mbarrier are bounded (one second of device time), so the kernel marks
a timeout and returns; the host reports KBE_ERR_TIMEOUT (sticky), and after
kbe_reset the handle steps again with results identical to a fresh handle."""
import numpy as np
import pytest

import kbe_inputs as ki

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu


def test_lost_copy_times_out_and_the_handle_recovers():
    s = ki.config("c2", nt=8)    # N_b = 4, n_k = 64: the staged C64 sweep
    g = kbe.KBE.from_system(s, precision=kbe.KBE_PREC_C64)
    g.step(3)
    g.synchronize()
    g.debug_inject(1)
    g.step(1)
    with pytest.raises(kbe.KBEError) as ex:
        g.synchronize()
    assert ex.value.status == -6            # KBE_ERR_TIMEOUT
    with pytest.raises(kbe.KBEError):       # sticky until reset
        g.step(1)
    g.reset()
    g.step(6)
    g.synchronize()
    f = kbe.KBE.from_system(s, precision=kbe.KBE_PREC_C64)
    f.step(6)
    for x in (0, 1):
        assert np.array_equal(g.row(6, x), f.row(6, x))
    g.close()
    f.close()


def test_injection_needs_the_staged_form():
    s = ki.config("c1", nt=4)      # N_b = 2: no staged sweep
    g = kbe.KBE.from_system(s, precision=kbe.KBE_PREC_C64)
    with pytest.raises(kbe.KBEError) as ex:
        g.debug_inject(1)
    assert ex.value.status == -7
    g.close()
