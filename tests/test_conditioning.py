"""How sensitive the c2 trajectory is to rounding-level changes (CPU oracle).

This sets what "agreement" can mean between two FP64 programs that round
differently: a one-ulp change of the interaction U moves the oracle's own
G row by ~1e-14 of its scale within 32 steps (5e-14 by step 100 and ~1e-12 by
the end of the driven c2 run, as measured once on 8 cores). Parity bars on
long runs are therefore stated above a floor of 1e-2 of the row scale.
"""
import numpy as np

import kbe_inputs as ki
import oracle


def test_one_ulp_of_U_moves_the_trajectory_by_1e14():
    s = ki.config("c2")
    nt = 24
    a = oracle.Oracle(s, nt_max=nt)
    a.step(nt)
    b = oracle.Oracle(s, nt_max=nt, U=np.array([s.U * (1 + 2.0 ** -52)]))
    b.step(nt)
    drift = [np.abs(a.row(i, 0) - b.row(i, 0)).max() / np.abs(a.row(i, 0)).max() for i in (8, 24)]
    assert drift[0] > 1e-15 and drift[1] > drift[0] * 0.9
    assert drift[1] < 1e-12
