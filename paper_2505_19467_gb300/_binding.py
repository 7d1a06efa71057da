"""ctypes binding of libkbe (include/kbe.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts numpy /
torch arguments to pointers and status codes to exceptions. There is no CPU
fallback: if libkbe.so cannot be loaded, importing the handle API raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libkbe.so")

KBE_PREC_FP64 = 0
KBE_PREC_DF64 = 1
KBE_PREC_C64 = 2
KBE_PREC_F16X2 = 3
PRECISIONS = {"fp64": KBE_PREC_FP64, "df64": KBE_PREC_DF64, "c64": KBE_PREC_C64, "f16x2": KBE_PREC_F16X2}

STATUS = {
    0: "KBE_OK", -1: "KBE_ERR_ARG", -2: "KBE_ERR_OOM", -3: "KBE_ERR_CUDA", -4: "KBE_ERR_STATE",
    -5: "KBE_ERR_NONFINITE", -6: "KBE_ERR_TIMEOUT", -7: "KBE_ERR_UNSUPPORTED", -8: "KBE_ERR_INTERNAL",
}

# every function declared in include/kbe.h (checked against the header by the tests)
EXPORTS = [
    "kbe_create", "kbe_destroy", "kbe_set_hamiltonian", "kbe_set_interaction", "kbe_set_drive",
    "kbe_reset", "kbe_step", "kbe_synchronize", "kbe_current_step", "kbe_observables",
    "kbe_observables_all", "kbe_get_row", "kbe_profile_enable", "kbe_profile_read",
    "kbe_last_error", "kbe_op_sigma_row_workspace", "kbe_op_sigma_row", "kbe_op_collision_row",
    "kbe_op_propagators", "kbe_op_update_row", "kbe_op_sigma_row_noalloc",
    "kbe_op_collision_row_workspace", "kbe_op_pack", "kbe_memory_bytes", "kbe_batch_create",
    "kbe_batch_destroy", "kbe_batch_system", "kbe_batch_reset", "kbe_batch_step",
    "kbe_batch_synchronize", "kbe_checkpoint_bytes", "kbe_checkpoint_save", "kbe_checkpoint_load",
    "kbe_set_dipole", "kbe_backward", "kbe_backward_memory_bytes", "kbe_corrector_iterations",
    "kbe_op_collision_row_quad", "kbe_set_graphs", "kbe_autotune", "kbe_debug_inject", "kbe_batch_set_graphs",
    "kbe_observables_all_dev", "kbe_get_row_dev", "kbe_device_info", "kbe_measure_fma_peaks",
    "kbe_set_sweep_choice", "kbe_op_pack_mesh", "kbe_history_bytes", "kbe_batch_set_persistent",
    "kbe_batch_sweep_launches",
]


class KBEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class kbe_config(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("dim", ctypes.c_int), ("L", ctypes.c_int * 2),
                ("nt_max", ctypes.c_int), ("dt", ctypes.c_double), ("beta", ctypes.c_double),
                ("mu", ctypes.c_double), ("precision", ctypes.c_int), ("n_corr", ctypes.c_int),
                ("hf", ctypes.c_int), ("paper_shift", ctypes.c_int), ("corr_tol", ctypes.c_double),
                ("quadrature", ctypes.c_int)]


class kbe_mesh(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("L", ctypes.c_int * 2)]


class kbe_profile_stats(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_int), ("sweep_ms", ctypes.c_double),
                ("sweep_flops", ctypes.c_double), ("sweep_flops_executed", ctypes.c_double),
                ("sweep_bytes", ctypes.c_double),
                ("launches", ctypes.c_int), ("backward_ms", ctypes.c_double * 4),
                ("backward_sweep_flops", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libkbe.so; raises if it is missing (build with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libkbe.so not found at {path}: run __graft_entry__.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pcfg, pmesh = ctypes.POINTER(kbe_config), ctypes.POINTER(kbe_mesh)
    sig = {
        "kbe_create": (I, [pcfg, P, ctypes.POINTER(P)]),
        "kbe_destroy": (I, [P]),
        "kbe_set_hamiltonian": (I, [P, I, P, P]),
        "kbe_set_interaction": (I, [P, I, P, P]),
        "kbe_set_drive": (I, [P, I, P, P]),
        "kbe_reset": (I, [P]),
        "kbe_step": (I, [P, I]),
        "kbe_synchronize": (I, [P]),
        "kbe_current_step": (I, [P, ctypes.POINTER(I)]),
        "kbe_observables": (I, [P, I, P, P]),
        "kbe_observables_all": (I, [P, P, P]),
        "kbe_get_row": (I, [P, I, I, P]),
        "kbe_profile_enable": (I, [P, I]),
        "kbe_profile_read": (I, [P, ctypes.POINTER(kbe_profile_stats)]),
        "kbe_last_error": (ctypes.c_char_p, [P]),
        "kbe_op_sigma_row_workspace": (S, [pmesh, I]),
        "kbe_op_sigma_row": (I, [pmesh, P, I, D, P, P, P, P, S, P]),
        "kbe_op_collision_row": (I, [pmesh, I, D, I, P, P, P, P, S, P]),
        "kbe_op_collision_row_workspace": (S, [pmesh, I, I]),
        "kbe_op_pack": (I, [I, P, P, S, S, P]),
        "kbe_op_pack_mesh": (I, [pmesh, I, P, P, S, P]),
        "kbe_history_bytes": (S, [pmesh, I, I]),
        "kbe_op_propagators": (I, [pmesh, D, P, P, P, P]),
        "kbe_op_update_row": (I, [pmesh, I, D, D, P, P, P, P, P, P, P, P]),
        "kbe_op_sigma_row_noalloc": (I, [pmesh, P, I, D, P, P, P, P]),
        "kbe_memory_bytes": (S, [pcfg]),
        "kbe_checkpoint_bytes": (S, [P]),
        "kbe_set_dipole": (I, [P, I, P, P]),
        "kbe_checkpoint_save": (I, [P, P, S]),
        "kbe_checkpoint_load": (I, [P, P, S]),
        "kbe_batch_create": (I, [I, pcfg, P, S, ctypes.POINTER(P), P]),
        "kbe_batch_destroy": (I, [P]),
        "kbe_batch_system": (P, [P, I]),
        "kbe_batch_reset": (I, [P]),
        "kbe_batch_step": (I, [P, I]),
        "kbe_batch_synchronize": (I, [P]),
        "kbe_backward": (I, [P, P, P, P]),
        "kbe_backward_memory_bytes": (S, [pcfg]),
        "kbe_corrector_iterations": (I, [P, P]),
        "kbe_set_graphs": (I, [P, I]),
        "kbe_autotune": (I, [P, P]),
        "kbe_debug_inject": (I, [P, I]),
        "kbe_batch_set_graphs": (I, [P, I]),
        "kbe_batch_set_persistent": (I, [P, I]),
        "kbe_batch_sweep_launches": (ctypes.c_long, [P]),
        "kbe_op_collision_row_quad": (I, [pmesh, I, D, I, I, P, P, P, P, S, P]),
        "kbe_observables_all_dev": (I, [P, P, P]),
        "kbe_get_row_dev": (I, [P, I, I, P]),
        "kbe_device_info": (I, [P, P]),
        "kbe_measure_fma_peaks": (I, [P, P]),
        "kbe_set_sweep_choice": (I, [pmesh, I, I, I, I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, handle=None) -> None:
    if rc != 0:
        msg = load().kbe_last_error(handle)
        raise KBEError(rc, msg.decode() if msg else "")


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _tptr(t):
    """Device pointer of a torch tensor (or None)."""
    return None if t is None else t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def mesh(nb: int, L) -> kbe_mesh:
    m = kbe_mesh()
    m.nb = nb
    m.L[0], m.L[1] = int(L[0]), int(L[1])
    return m


def make_config(nb, dim, L, nt_max, dt, beta, mu, precision=KBE_PREC_FP64, n_corr=2, hf=1,
                paper_shift=0, corr_tol=0.0, quadrature=0) -> kbe_config:
    cfg = kbe_config()
    cfg.nb, cfg.dim = nb, dim
    cfg.L[0], cfg.L[1] = int(L[0]), int(L[1])
    cfg.nt_max, cfg.dt, cfg.beta, cfg.mu = nt_max, dt, beta, mu
    cfg.precision, cfg.n_corr, cfg.hf, cfg.paper_shift = precision, n_corr, hf, paper_shift
    cfg.corr_tol = corr_tol
    cfg.quadrature = quadrature
    return cfg


def system_config(sys, nt_max=None, precision=KBE_PREC_FP64) -> kbe_config:
    return make_config(sys.nb, sys.dim, sys.L, sys.nt if nt_max is None else nt_max, sys.dt, sys.beta,
                       sys.mu, precision, sys.n_corr, sys.hf, sys.paper_shift, sys.corr_tol, sys.quadrature)


def memory_bytes(cfg: kbe_config) -> int:
    return int(load().kbe_memory_bytes(ctypes.byref(cfg)))


def backward_memory_bytes(cfg: kbe_config) -> int:
    """device bytes the first KBE.backward of a handle with cfg allocates"""
    return int(load().kbe_backward_memory_bytes(ctypes.byref(cfg)))


class KBE:
    """One Kadanoff-Baym system on the GPU (handle API of include/kbe.h)."""

    def __init__(self, nb: int, dim: int, L, nt_max: int, dt: float, beta: float, mu: float,
                 precision: int = KBE_PREC_FP64, n_corr: int = 2, hf: int = 1,
                 paper_shift: int = 0, stream=None, _borrow=None, corr_tol: float = 0.0,
                 quadrature: int = 0):
        lib = load()
        self.nb, self.nk, self.nt_max = nb, int(L[0]) * int(L[1]), nt_max
        self._u_len = 1
        self._owned = _borrow is None
        if _borrow is not None:      # a handle owned by a batch
            self._h = ctypes.c_void_p(_borrow)
            return
        cfg = make_config(nb, dim, L, nt_max, dt, beta, mu, precision, n_corr, hf, paper_shift, corr_tol,
                          quadrature)
        self._h = ctypes.c_void_p()
        self._stream = _stream_ptr(stream)
        _check(lib.kbe_create(ctypes.byref(cfg), self._stream, ctypes.byref(self._h)), None)

    @classmethod
    def from_system(cls, sys, nt_max=None, precision=KBE_PREC_FP64, stream=None, U=None, **over):
        """Build and initialise from a kbe_inputs.System (reset included)."""
        kw = dict(n_corr=sys.n_corr, hf=sys.hf, paper_shift=sys.paper_shift, corr_tol=sys.corr_tol,
                  quadrature=sys.quadrature)
        kw.update(over)
        k = cls(sys.nb, sys.dim, sys.L, sys.nt if nt_max is None else nt_max, sys.dt, sys.beta,
                sys.mu, precision=precision, stream=stream, **kw)
        k.set_hamiltonian(sys.hop_R, sys.hop_T)
        k.set_interaction(np.array([sys.U]) if U is None else U, sys.v)
        k.set_drive(sys.A, sys.direction)
        if getattr(sys, "dipole_E", None) is not None:
            k.set_dipole(sys.dipole_E, sys.dipole_M)
        k.reset()
        return k

    def close(self):
        if getattr(self, "_h", None) and self._h.value and getattr(self, "_owned", True):
            load().kbe_destroy(self._h)
        self._h = ctypes.c_void_p()

    def load_inputs(self, sys, U=None):
        """hoppings, interaction and drive of a kbe_inputs.System"""
        self.set_hamiltonian(sys.hop_R, sys.hop_T)
        self.set_interaction(np.array([sys.U]) if U is None else U, sys.v)
        self.set_drive(sys.A, sys.direction)
        if getattr(sys, "dipole_E", None) is not None:
            self.set_dipole(sys.dipole_E, sys.dipole_M)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hamiltonian(self, R, T):
        R = np.ascontiguousarray(R, np.int32)
        T = np.ascontiguousarray(T, np.complex128)
        _check(load().kbe_set_hamiltonian(self._h, R.shape[0], _np_ptr(R), _np_ptr(T)), self._h)

    def set_interaction(self, U, v=None):
        U = np.ascontiguousarray(np.atleast_1d(U), np.float64)
        self._u_len = len(U)
        v = None if v is None else np.ascontiguousarray(v, np.float64)
        _check(load().kbe_set_interaction(self._h, len(U), _np_ptr(U), _np_ptr(v)), self._h)

    def set_drive(self, A, direction=(1.0, 0.0)):
        d = np.ascontiguousarray(direction, np.float64)
        if A is None:
            _check(load().kbe_set_drive(self._h, 0, None, _np_ptr(d)), self._h)
        else:
            A = np.ascontiguousarray(A, np.float64)
            _check(load().kbe_set_drive(self._h, len(A), _np_ptr(A), _np_ptr(d)), self._h)

    def set_dipole(self, E, M=None):
        """dipole drive E_i M (Eq. 4); E None removes it"""
        if E is None:
            _check(load().kbe_set_dipole(self._h, 0, None, None), self._h)
            return
        E = np.ascontiguousarray(E, np.float64)
        M = np.ascontiguousarray(M, np.complex128)
        _check(load().kbe_set_dipole(self._h, len(E), _np_ptr(E), _np_ptr(M)), self._h)

    def reset(self):
        _check(load().kbe_reset(self._h), self._h)

    def step(self, nsteps: int = 1):
        _check(load().kbe_step(self._h, int(nsteps)), self._h)

    def synchronize(self):
        _check(load().kbe_synchronize(self._h), self._h)

    @property
    def n(self) -> int:
        x = ctypes.c_int()
        _check(load().kbe_current_step(self._h, ctypes.byref(x)), self._h)
        return x.value

    def observables(self, step: int):
        nkb = np.empty((self.nk, self.nb), np.float64)
        sc = np.empty(6, np.float64)
        _check(load().kbe_observables(self._h, int(step), _np_ptr(nkb), _np_ptr(sc)), self._h)
        return nkb, sc

    def observables_all(self, nkb_out=None, scalars_out=None):
        n = self.n
        nkb = nkb_out if nkb_out is not None else np.empty((n + 1, self.nk, self.nb), np.float64)
        sc = scalars_out if scalars_out is not None else np.empty((n + 1, 6), np.float64)
        _check(load().kbe_observables_all(self._h, _np_ptr(nkb), _np_ptr(sc)), self._h)
        return nkb, sc

    def row(self, i: int, which: int = 0) -> np.ndarray:
        out = np.empty((i + 1, self.nk, self.nb, self.nb), np.complex128)
        _check(load().kbe_get_row(self._h, int(i), int(which), _np_ptr(out)), self._h)
        return out

    def row_dev(self, i: int, which: int, out) -> None:
        """row i of G^which into a caller-owned device tensor (complex128,
        [(i+1), nk, nb, nb], contiguous), enqueued on the handle's stream"""
        _check(load().kbe_get_row_dev(self._h, int(i), int(which), _tptr(out)), self._h)

    def observables_all_dev(self, nkb_out=None, scalars_out=None) -> None:
        """n_kb [(n+1), nk, nb] and scalars [(n+1), 6] (float64 device tensors,
        either may be None), enqueued on the handle's stream"""
        _check(load().kbe_observables_all_dev(self._h, None if nkb_out is None else _tptr(nkb_out),
                                              None if scalars_out is None else _tptr(scalars_out)), self._h)

    def checkpoint(self) -> bytes:
        """The state after the current row, as bytes (history rows 0..n etc.)."""
        nbytes = int(load().kbe_checkpoint_bytes(self._h))
        buf = np.empty(nbytes, np.uint8)
        _check(load().kbe_checkpoint_save(self._h, _np_ptr(buf), nbytes), self._h)
        return buf.tobytes()

    def restore(self, data: bytes):
        buf = np.frombuffer(data, np.uint8)
        _check(load().kbe_checkpoint_load(self._h, _np_ptr(np.ascontiguousarray(buf)), len(buf)), self._h)

    def debug_inject(self, fault: int):
        """one-shot fault injection for the failure-path test (kbe_debug_inject)"""
        _check(load().kbe_debug_inject(self._h, int(fault)), self._h)

    def autotune(self) -> np.ndarray:
        """time the sweep's split candidates and keep the fastest (kbe_autotune);
        returns the choice per row bucket (0 = not tuned)"""
        out = np.zeros(17, np.int32)
        _check(load().kbe_autotune(self._h, _np_ptr(out)), self._h)
        return out

    def set_graphs(self, enable: bool = True):
        """replay captured CUDA graphs for repeated kbe_step calls (kbe_set_graphs)"""
        _check(load().kbe_set_graphs(self._h, int(enable)), self._h)

    def corrector_iterations(self) -> np.ndarray:
        """corrector passes run at each step 0..n (kbe_corrector_iterations)"""
        out = np.empty(self.n + 1, np.int32)
        _check(load().kbe_corrector_iterations(self._h, _np_ptr(out)), self._h)
        return out

    def backward(self, dL_dn):
        """(dL/dA [nt_max], dL/dU) for the cotangent dL_dn [nk][nb] of the
        current row's occupations (kbe_backward). dL/dU is a float for a
        constant U, an array [nt_max + 1] (per sample) for U(t) samples."""
        g = np.ascontiguousarray(dL_dn, np.float64).reshape(self.nk, self.nb)
        dA = np.empty(self.nt_max, np.float64)
        dU = np.empty(self.nt_max + 1, np.float64)
        _check(load().kbe_backward(self._h, _np_ptr(g), _np_ptr(dA), _np_ptr(dU)), self._h)
        return dA, (float(dU[0]) if self._u_len == 1 else dU)

    def profile(self, enable: bool = True):
        _check(load().kbe_profile_enable(self._h, int(enable)), self._h)

    def profile_read(self) -> dict:
        s = kbe_profile_stats()
        _check(load().kbe_profile_read(self._h, ctypes.byref(s)), self._h)
        return dict(sweep_launches=s.sweep_launches, sweep_ms=s.sweep_ms, sweep_flops=s.sweep_flops,
                    sweep_flops_executed=s.sweep_flops_executed, sweep_bytes=s.sweep_bytes,
                    launches=s.launches, backward_ms=list(s.backward_ms),
                    backward_sweep_flops=s.backward_sweep_flops)


# ---- stateless ops on torch device tensors (GPU layout, see include/kbe.h) ----

def _c(t):
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def sigma_row(nb, L, v, n, Un, Grow, Sigma, work, Ul=None, stream=None):
    m = mesh(nb, L)
    v = np.ascontiguousarray(v, np.float64)
    _check(load().kbe_op_sigma_row(ctypes.byref(m), _np_ptr(v), int(n), float(Un),
                                   None if Ul is None else _c(Ul), _c(Grow), _c(Sigma), _c(work),
                                   work.numel() * work.element_size(), _stream_ptr(stream)))


def sigma_row_workspace(nb, L, n) -> int:
    m = mesh(nb, L)
    return int(load().kbe_op_sigma_row_workspace(ctypes.byref(m), int(n)))


def collision_row_workspace(nb, L, n, precision=KBE_PREC_FP64) -> int:
    m = mesh(nb, L)
    return int(load().kbe_op_collision_row_workspace(ctypes.byref(m), int(n), int(precision)))


def collision_row(nb, L, n, dt, H, Sigma, I, precision=KBE_PREC_FP64, work=None, stream=None,
                  quadrature=0):
    """H: history triangle in the precision's storage (see pack); quadrature
    0 trapezoid, 1 Gregory (kbe_op_collision_row_quad)."""
    m = mesh(nb, L)
    wb = 0 if work is None else work.numel() * work.element_size()
    if quadrature == 0:
        _check(load().kbe_op_collision_row(ctypes.byref(m), int(n), float(dt), int(precision), _c(H),
                                           _c(Sigma), _c(I), None if work is None else _c(work), wb,
                                           _stream_ptr(stream)))
    else:
        _check(load().kbe_op_collision_row_quad(ctypes.byref(m), int(n), float(dt), int(precision),
                                                int(quadrature), _c(H), _c(Sigma), _c(I),
                                                None if work is None else _c(work), wb, _stream_ptr(stream)))


def history_bytes(nb, L, n, precision) -> int:
    """bytes of a history triangle with rows 0..n in `precision`'s storage
    (kbe_history_bytes)"""
    m = mesh(nb, L)
    return int(load().kbe_history_bytes(ctypes.byref(m), int(n), int(precision)))


def pack(precision, src, dst, nblocks, block_elems, stream=None, nb=None, L=None):
    """FP64 (G^<, G^>) blocks [nblocks][2][nb][nb][nk] -> history storage of
    `precision`, (G^<, dG) per block (dst bytes: 16 per complex for FP64 and
    DF64, 8 for C64 and F16X2). With the mesh (nb, L) it calls
    kbe_op_pack_mesh, which every precision accepts (F16X2 requires it)."""
    if nb is not None:
        m = mesh(nb, L)
        _check(load().kbe_op_pack_mesh(ctypes.byref(m), int(precision), _c(src), _c(dst), int(nblocks),
                                       _stream_ptr(stream)))
        return
    _check(load().kbe_op_pack(int(precision), _c(src), _c(dst), int(nblocks), int(block_elems),
                              _stream_ptr(stream)))


def propagators(nb, L, dt, h, U, V, stream=None):
    m = mesh(nb, L)
    _check(load().kbe_op_propagators(ctypes.byref(m), float(dt), _c(h), _c(U), _c(V), _stream_ptr(stream)))


def update_row(nb, L, n, dt, theta, h, U, V, Gprev, Iprev, Icur, out, stream=None):
    m = mesh(nb, L)
    _check(load().kbe_op_update_row(ctypes.byref(m), int(n), float(dt), float(theta), _c(h), _c(U), _c(V),
                                    _c(Gprev), _c(Iprev), None if Icur is None else _c(Icur), _c(out),
                                    _stream_ptr(stream)))


def sigma_row_noalloc(nb, L, v, n, Un, Grow, Sigma, Ul=None, stream=None):
    """Sigma row with the library's built-in scratch (no device allocation);
    for callers that cannot allocate. Rows needing more than
    KBE_NOALLOC_SCRATCH_BYTES of scratch raise KBEError (KBE_ERR_ARG)."""
    m = mesh(nb, L)
    v = np.ascontiguousarray(v, np.float64)
    _check(load().kbe_op_sigma_row_noalloc(ctypes.byref(m), _np_ptr(v), int(n), float(Un),
                                           None if Ul is None else _c(Ul), _c(Grow), _c(Sigma),
                                           _stream_ptr(stream)))


NOALLOC_SCRATCH_BYTES = 64 << 20   # KBE_NOALLOC_SCRATCH_BYTES in include/kbe.h


class KBEBatch:
    """Independent systems advanced together (kbe_batch_* of include/kbe.h)."""

    def __init__(self, systems, precision=KBE_PREC_FP64, nt_max=None, budget_bytes=0, stream=None):
        lib = load()
        n = len(systems)
        cfgs = (kbe_config * n)(*[system_config(s, None if nt_max is None else nt_max[i], precision)
                                  for i, s in enumerate(systems)])
        adm = (ctypes.c_int * n)()
        self._b = ctypes.c_void_p()
        _check(lib.kbe_batch_create(n, cfgs, _stream_ptr(stream), int(budget_bytes),
                                    ctypes.byref(self._b), adm), None)
        self.admitted = [bool(a) for a in adm]
        self.systems = []
        for i, s in enumerate(systems):
            if not self.admitted[i]:
                self.systems.append(None)
                continue
            h = lib.kbe_batch_system(self._b, i)
            k = KBE(s.nb, s.dim, s.L, cfgs[i].nt_max, s.dt, s.beta, s.mu, _borrow=h)
            k.load_inputs(s)
            self.systems.append(k)

    def reset(self):
        _check(load().kbe_batch_reset(self._b))

    def step(self, nsteps: int):
        _check(load().kbe_batch_step(self._b, int(nsteps)))

    def set_graphs(self, enable: bool = True):
        """graph mode: one captured graph per batch step call on a non-default
        stream, per-system graphs on the default one (kbe_batch_set_graphs)"""
        _check(load().kbe_batch_set_graphs(self._b, int(enable)))

    def set_persistent(self, enable: bool = True):
        """stage-major steps with the sweeps of the systems in one persistent
        launch per (N_b, quadrature, form) and lane; FP64 histories (kbe_batch_set_persistent)"""
        _check(load().kbe_batch_set_persistent(self._b, int(enable)))

    def sweep_launches(self) -> int:
        """persistent sweep launches enqueued eagerly so far (kbe_batch_sweep_launches)"""
        return int(load().kbe_batch_sweep_launches(self._b))

    def synchronize(self):
        _check(load().kbe_batch_synchronize(self._b))

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            for k in self.systems:
                if k is not None:
                    k._h = ctypes.c_void_p()
            load().kbe_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_info():
    """(binary version the kernels were built for, SM count of the current device)"""
    bv, sm = ctypes.c_int(), ctypes.c_int()
    _check(load().kbe_device_info(ctypes.byref(bv), ctypes.byref(sm)))
    return bv.value, sm.value


def measure_fma_peaks():
    """(FP64, FP32) FMA throughput of the current device in GFLOP/s (measured)"""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().kbe_measure_fma_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def set_sweep_choice(nb, L, precision, choice, quadrature=0, bucket=-1):
    """the sweep's launch choice for a shape (kbe_set_sweep_choice): > 0 the
    per-column sweep's CTAs per SM, < 0 the single-read tile sweep with -choice
    rows per work item, 0 the default"""
    m = mesh(nb, L)
    _check(load().kbe_set_sweep_choice(ctypes.byref(m), int(precision), int(quadrature), int(bucket), int(choice)))
