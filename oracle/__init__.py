"""FP64 CPU oracle for the Kadanoff-Baym time stepping (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import this package. It shares no code with
the CUDA library; the two meet only in ``kbe_inputs`` (seeded inputs).
Block layout on this side is [k][a][b] (band indices fastest).

Parity status of each function (what pins it) is listed in ``PINS`` below and
checked by ``tests/test_oracle_pins.py``.
"""
from .oracle import (Oracle, build, sigma_pair, sigma_pair_literal, collision_row, evaluate_row_on,
                     propagators, update_row, library_path)
from . import gradient

PINS = {
    "sigma_pair": "direct Eq. 7 sum (N_b=2 bar form, general v); ED O(U^2) at N_b=2 and, "
                  "for v = 1 - delta and a random symmetric v, at N_b=3 (U^2 coefficient)",
    "sigma_pair_literal": "Eq. 7 as printed (bar convention) on random G; a hand-summed element",
    "collision_row": "analytic integrals of exponentials (trapezoid error O(dt^2); Gregory "
                     "O(dt^4), exact for cubics); I^>(n,n) = I^<(n,n); number conservation",
    "propagators": "unitarity, closed form at U = 0, h V = U - 1",
    "update_row": "U = 0 closed form (driven and undriven)",
    "Oracle.step": "U = 0 closed form; particle number; energy drift O(dt^2); "
                   "exact diagonalisation through O(U^2); time-step order 2; the full-grid "
                   "mode's right-equation column equals -G(t_n, t_j)^+ (Eq. 6 as printed, limit t')",
    "gradient.directional": "U = 0: Frechet derivative of the exact one-step propagators "
                            "(drive samples and U through the mean field and shift)",
}
