"""ctypes binding of ``kbe_oracle.c`` (test infrastructure, see package doc)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libkbe_oracle.so")
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, FP64, no contraction into FMA)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fcx-limited-range", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [i, i, i, i, i, d, d, d, i, i, i]
            lib.orc_destroy.argtypes = [P]
            lib.orc_set_hamiltonian.argtypes = [P, i, P, P]
            lib.orc_set_interaction.argtypes = [P, i, P, P]
            lib.orc_set_drive.argtypes = [P, i, P, P]
            lib.orc_set_dipole.argtypes = [P, i, P, P]
            lib.orc_reset.argtypes = [P]
            lib.orc_step.argtypes = [P, i]
            lib.orc_current.argtypes = [P]
            lib.orc_get_block.argtypes = [P, i, i, i, P]
            lib.orc_get_irow.argtypes = [P, i, P]
            lib.orc_observables.argtypes = [P, i, P, P]
            lib.orc_sigma_pair.argtypes = [i, i, i, P, d, P, P, P, P]
            lib.orc_sigma_pair_literal.argtypes = [i, i, i, P, d, P, P, P, P]
            lib.orc_collision_row.argtypes = [i, i, i, d, P, P, P, P, P, P]
            lib.orc_propagators.argtypes = [i, i, d, P, P, P, P, P]
            lib.orc_update_row.argtypes = [i, i, i, d, d, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_set_corr_tol.argtypes = [P, d]
            lib.orc_set_quadrature.argtypes = [P, i]
            lib.orc_collision_row_q.argtypes = [i, i, i, d, i, P, P, P, P, P, P]
            lib.orc_get_iters.argtypes = [P, P]
            lib.orc_set_threads.argtypes = [i]
            lib.orc_threads.restype = i
            lib.orc_enable_full.argtypes = [P, i]
            lib.orc_evaluate_row_on.argtypes = [i, i, i, P, d, i, d, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_threads())


def sigma_pair(nb, L, v, UnUl, Gl, Gg):
    """Sigma^<, Sigma^> (n,l) from G^<, G^> (n,l), each [nk, nb, nb] (Eqs. 7-9)."""
    lib = _load()
    Gl, Gg = _c128(Gl), _c128(Gg)
    v = np.ascontiguousarray(v, dtype=np.float64)
    Sl, Sg = np.empty_like(Gl), np.empty_like(Gg)
    lib.orc_sigma_pair(nb, L[0], L[1], _ptr(v), float(UnUl), _ptr(Gl), _ptr(Gg), _ptr(Sl), _ptr(Sg))
    return Sl, Sg


def sigma_pair_literal(nb, L, v, UnUl, Gl, Gg):
    """Eq. 7 as an O(n_k^3) sum; v=None selects the paper's bar form (N_b=2)."""
    lib = _load()
    Gl, Gg = _c128(Gl), _c128(Gg)
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    Sl, Sg = np.empty_like(Gl), np.empty_like(Gg)
    lib.orc_sigma_pair_literal(nb, L[0], L[1], _ptr(vv), float(UnUl), _ptr(Gl), _ptr(Gg), _ptr(Sl), _ptr(Sg))
    return Sl, Sg


def collision_row(nb, nk, n, dt, Hl, Hg, Sl, Sg, quadrature=0):
    """I^<, I^> (n, j), j=0..n. H*: triangle [(n+1)(n+2)/2, nk, nb, nb];
    S*: [n+1, nk, nb, nb]. Returns two [n+1, nk, nb, nb] arrays. quadrature:
    0 trapezoid (the paper's rule), 1 fourth-order Gregory."""
    lib = _load()
    Hl, Hg, Sl, Sg = map(_c128, (Hl, Hg, Sl, Sg))
    Il = np.empty((n + 1, nk, nb, nb), np.complex128)
    Ig = np.empty_like(Il)
    lib.orc_collision_row_q(nb, nk, n, float(dt), int(quadrature), _ptr(Hl), _ptr(Hg), _ptr(Sl), _ptr(Sg),
                            _ptr(Il), _ptr(Ig))
    return Il, Ig


def evaluate_row_on(nb, L, v, U, n, dt, Hl, Hg):
    """One row evaluation as the stepper performs it (Sigma row n of the
    triangle's row n, then the collision row) on caller arrays: Hl, Hg hold a
    triangle with at least rows 0..n ([ntri, nk, nb, nb] complex128). Returns
    (Sl, Sg, Il, Ig), each [n+1, nk, nb, nb]. For timing sampled rows."""
    lib = _load()
    nk = L[0] * L[1]
    v = np.ascontiguousarray(v, dtype=np.float64)
    S = [np.empty((n + 1, nk, nb, nb), np.complex128) for _ in range(4)]
    lib.orc_evaluate_row_on(nb, L[0], L[1], _ptr(v), float(U), int(n), float(dt), _ptr(Hl), _ptr(Hg),
                            *(_ptr(x) for x in S))
    return tuple(S)


def propagators(nb, nk, dt, h):
    """U, V, W, lam per k from h [nk, nb, nb]."""
    lib = _load()
    h = _c128(h)
    U, V, W = np.empty_like(h), np.empty_like(h), np.empty_like(h)
    lam = np.empty((nk, nb), np.float64)
    lib.orc_propagators(nb, nk, float(dt), _ptr(h), _ptr(U), _ptr(V), _ptr(W), _ptr(lam))
    return U, V, W, lam


def update_row(nb, nk, n, dt, theta, U, V, W, lam, Gpl, Gpg, Ipl, Ipg, Icl=None, Icg=None):
    """Row n of G^<, G^> ([n+1, nk, nb, nb]) from row n-1 (n blocks)."""
    lib = _load()
    U, V, W, Gpl, Gpg, Ipl, Ipg = map(_c128, (U, V, W, Gpl, Gpg, Ipl, Ipg))
    Icl = None if Icl is None else _c128(Icl)
    Icg = None if Icg is None else _c128(Icg)
    lam = np.ascontiguousarray(lam, np.float64)
    outl = np.empty((n + 1, nk, nb, nb), np.complex128)
    outg = np.empty_like(outl)
    lib.orc_update_row(nb, nk, n, float(dt), float(theta), _ptr(U), _ptr(V), _ptr(W), _ptr(lam),
                       _ptr(Gpl), _ptr(Gpg), _ptr(Ipl), _ptr(Ipg), _ptr(Icl), _ptr(Icg),
                       _ptr(outl), _ptr(outg))
    return outl, outg


class Oracle:
    """Stateful FP64 stepper (Algorithm 1) on one kbe_inputs.System."""

    def __init__(self, sys, nt_max: Optional[int] = None, n_corr: Optional[int] = None,
                 hf: Optional[int] = None, paper_shift: Optional[int] = None,
                 U: Optional[np.ndarray] = None, full_grid: bool = False,
                 right_limit_printed: bool = False):
        """full_grid: propagate the upper triangle G(t_j, t_n) with the right
        equation (Eq. 6 as printed, G * Sigma) instead of mirroring the lower
        one; tiny grids only (Eq. 7 is summed directly, O(n_k^3) per pair).
        right_limit_printed: in that mode, end the second integral of Eq. 6 at
        t as printed instead of t'."""
        lib = _load()
        self.sys = sys
        self.nb, self.nk, self.L = sys.nb, sys.nk, sys.L
        self.nt_max = sys.nt if nt_max is None else nt_max
        self._h = lib.orc_create(sys.nb, sys.dim, sys.L[0], sys.L[1], self.nt_max, sys.dt,
                                 sys.beta, sys.mu, sys.n_corr if n_corr is None else n_corr,
                                 sys.hf if hf is None else hf,
                                 sys.paper_shift if paper_shift is None else paper_shift)
        if not self._h:
            raise MemoryError("oracle: create failed")
        R = np.ascontiguousarray(sys.hop_R, np.int32)
        T = _c128(sys.hop_T)
        lib.orc_set_hamiltonian(self._h, R.shape[0], _ptr(R), _ptr(T))
        Us = np.array([sys.U], np.float64) if U is None else np.ascontiguousarray(U, np.float64)
        v = np.ascontiguousarray(sys.v, np.float64)
        rc = lib.orc_set_interaction(self._h, len(Us), _ptr(Us), _ptr(v))
        if rc != 0:
            raise ValueError("oracle: v must be symmetric" if rc == -2 else "oracle: bad interaction samples")
        d = np.array(sys.direction, np.float64)
        if sys.A is not None:
            A = np.ascontiguousarray(sys.A, np.float64)
            lib.orc_set_drive(self._h, len(A), _ptr(A), _ptr(d))
        else:
            lib.orc_set_drive(self._h, 0, None, _ptr(d))
        self._keep = (R, T, Us, v, d)
        if getattr(sys, "dipole_E", None) is not None:
            E = np.ascontiguousarray(sys.dipole_E, np.float64)
            M = _c128(sys.dipole_M)
            lib.orc_set_dipole(self._h, len(E), _ptr(E), _ptr(M))
            self._keep = self._keep + (E, M)
        lib.orc_set_corr_tol(self._h, float(getattr(sys, "corr_tol", 0.0)))
        lib.orc_set_quadrature(self._h, int(getattr(sys, "quadrature", 0)))
        if full_grid and lib.orc_enable_full(self._h, int(bool(right_limit_printed))) != 0:
            raise MemoryError("oracle: full-grid storage")
        if lib.orc_reset(self._h) != 0:
            raise RuntimeError("oracle: reset failed")

    def close(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return int(_load().orc_current(self._h))

    def step(self, nsteps: int = 1) -> None:
        rc = _load().orc_step(self._h, int(nsteps))
        if rc != 0:
            raise RuntimeError(f"oracle: step failed ({rc})")

    def block(self, i: int, j: int, which: int = 0) -> np.ndarray:
        out = np.empty((self.nk, self.nb, self.nb), np.complex128)
        if _load().orc_get_block(self._h, i, j, which, _ptr(out)) != 0:
            raise IndexError((i, j))
        return out

    def row(self, i: int, which: int = 0) -> np.ndarray:
        return np.stack([self.block(i, j, which) for j in range(i + 1)])

    def iterations(self) -> np.ndarray:
        """corrector passes run at steps 0..n"""
        out = np.empty(self.n + 1, np.int32)
        _load().orc_get_iters(self._h, _ptr(out))
        return out

    def irow(self, which: int = 0) -> np.ndarray:
        out = np.empty((self.n + 1, self.nk, self.nb, self.nb), np.complex128)
        _load().orc_get_irow(self._h, which, _ptr(out))
        return out

    def observables(self, step: int):
        nkb = np.empty((self.nk, self.nb), np.float64)
        sc = np.empty(6, np.float64)
        if _load().orc_observables(self._h, step, _ptr(nkb), _ptr(sc)) != 0:
            raise IndexError(step)
        return nkb, sc
