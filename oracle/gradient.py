"""Reference gradient of the occupation loss from the FP64 oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path). It differentiates the oracle's own forward (Algorithm 1 as
oracle/kbe_oracle.c implements it) numerically, so it shares nothing with
the library's hand-written reverse mode.

Loss (the reverse-mode workload): L = sum_kb (n_kb(t_N) - n*_kb)^2, with
n_kb = Im G^<_bb(k; t_N, t_N) the occupations of the oracle's trajectory.

The derivative along a parameter direction e (Peierls samples A and/or the
constant U) is taken by central differences with one Richardson step,
    D(h) = [L(p + h e) - L(p - h e)] / 2h,   R = [4 D(h/2) - D(h)] / 3,
which cancels the h^2 term of D: the error is O(h^4) from truncation plus
O(eps |L| / h) from rounding, about 1e-11 relative at h = 1e-3 for the
small systems used.

Pinned in tests/test_oracle_gradient.py: at U = 0 the trajectory is a
product of exact one-step propagators, and the gradient follows from the
Frechet derivative of the matrix exponential (scipy), computed there
independently of this module and of the oracle.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .oracle import Oracle


def occupations(sys, N: int, A: Optional[np.ndarray] = None, U=None) -> np.ndarray:
    """n_kb(t_N) [nk][nb] of the oracle's trajectory with drive A and U: a
    constant, or samples U(t_i) (len >= max(N, sys.nt) + 1)."""
    samples = U is not None and np.ndim(U) > 0
    s = dataclasses.replace(sys, A=sys.A if A is None else np.asarray(A, np.float64).copy(),
                            U=sys.U if (U is None or samples) else float(U))
    nt_max = max(N, s.nt)
    o = Oracle(s, nt_max=nt_max, U=np.asarray(U, np.float64)[: nt_max + 1] if samples else None)
    o.step(N)
    nkb, _ = o.observables(N)
    o.close()
    return nkb


def loss(sys, N: int, target: np.ndarray, A=None, U=None) -> float:
    return float(((occupations(sys, N, A, U) - target) ** 2).sum())


def directional(sys, N: int, target: np.ndarray, dA: Optional[np.ndarray] = None, dU: float = 0.0,
                h: float = 1e-3) -> float:
    """dL along (dA, dU) at (sys.A, sys.U), Richardson-extrapolated central differences."""
    A0 = np.zeros(N) if sys.A is None else np.asarray(sys.A, np.float64)
    dA = np.zeros_like(A0) if dA is None else np.asarray(dA, np.float64)

    def D(step):
        lp = loss(sys, N, target, A0 + step * dA, sys.U + step * dU)
        lm = loss(sys, N, target, A0 - step * dA, sys.U - step * dU)
        return (lp - lm) / (2 * step)

    return (4.0 * D(h / 2) - D(h)) / 3.0


def gradient_samples(sys, N: int, target: np.ndarray, U: np.ndarray, which=None, h: float = 1e-3):
    """dL/dU_i for samples U(t_i) (i in which, default 0..N), at the drive sys.A"""
    U = np.asarray(U, np.float64)

    def D(i, step):
        e = np.zeros_like(U)
        e[i] = step
        return (loss(sys, N, target, U=U + e) - loss(sys, N, target, U=U - e)) / (2 * step)

    idx = range(N + 1) if which is None else which
    return np.array([(4.0 * D(i, h / 2) - D(i, h)) / 3.0 for i in idx])


def gradient(sys, N: int, target: np.ndarray, which_A=None, with_U: bool = True, h: float = 1e-3):
    """(dL/dA_i for i in which_A, dL/dU): each a directional derivative above"""
    A0 = np.zeros(N) if sys.A is None else np.asarray(sys.A, np.float64)
    idx = range(N) if which_A is None else which_A
    gA = []
    for i in idx:
        e = np.zeros_like(A0)
        e[i] = 1.0
        gA.append(directional(sys, N, target, dA=e, h=h))
    gU = directional(sys, N, target, dU=1.0, h=h) if with_U else None
    return np.array(gA), gU
