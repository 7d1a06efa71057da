"""Seeded synthetic inputs for the Kadanoff-Baym (KBE) time stepping.

This module is shared by both sides of every parity check: the FP64 CPU oracle
(``oracle/``) and the CUDA library (``paper_2505_19467_gb300``). It holds only
the *description* of each workload -- hopping tables, interaction samples,
drive-pulse samples and random test tensors -- drawn from numpy's PCG64
generator with fixed seeds. It contains none of the method's arithmetic
(no Green's functions, self-energies, collision integrals or propagators), so
neither side can borrow the other's numerics through it.

Workloads (the paper's model, Sec. 2, Eqs. 2-4, generalised to N_b bands and a
Peierls drive):

* ``c1``  N_b=2, 1-D ring L=8, eps_b(k) = -2 cos(k + b pi/2) + 0.5 b, U=0.5,
          beta=10, mu=0, no drive, N_t=64, dt=0.05, seed 0.
* ``c2``  N_b=4, 8x8 mesh, eps_b(k) = -2(cos kx + cos ky) + 0.4 b plus a seeded
          k-independent Hermitian inter-band coupling (re, im ~ N(0, 0.1)),
          U=1.0, beta=20, mu=0, Peierls pulse A0=0.3, t0=5, sigma=1.5, omega=2
          along x, N_t=512, dt=0.02, seed 1.
* ``c3``  N_b=8, 16x16 mesh, offsets 0.25 b, U=1.5, A0=0.5, otherwise as c2,
          seed 2.
* ``c4``  64 independent systems of uneven size (seed 3), see ``batched``.
* ``c5``  c2's system with seeded target occupations (seed 4), see ``targets``.
* ``paper`` the paper's own model problem shape (Sec. 2, Sec. 6): two bands on a
          1-D ring of n_k = 1024, eps_v = -2(1 - cos k) - E_g/2,
          eps_c = 2(1 - cos k) + E_g/2, E_g = 1, dipole kick E(t) = I delta(t - 0.5)
          with d_k = 1, N_t = 500. The paper gives no U, I, dt or temperature;
          this workload takes U = 0.5, I = 0.1, dt = 0.02, beta = 10, mu = 0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass
class System:
    """One lattice system and its run parameters (plain data, no numerics)."""

    name: str
    nb: int                       # number of bands N_b
    dim: int                      # 1 or 2
    L: Tuple[int, int]            # mesh (L0, L1); L1 = 1 for dim = 1
    nt: int                       # number of time steps N_t
    dt: float
    U: float                      # on-site inter-band interaction U (constant)
    beta: float
    mu: float
    hop_R: np.ndarray             # int32 [nhop, 2]  lattice vectors R
    hop_T: np.ndarray             # complex128 [nhop, nb, nb]  t_ab(R)
    v: np.ndarray                 # float64 [nb, nb]  band pairing pattern v_ab
    A: Optional[np.ndarray]       # float64 [nt] Peierls samples at t_{i+1/2}, or None
    direction: Tuple[float, float]
    hf: int = 1                   # Hartree-Fock mean field on
    paper_shift: int = 0          # the -U n_c one-body term of Eq. 2 (N_b = 2)
    n_corr: int = 2               # corrector iterations, P(EC)^n_corr E
    seed: int = 0
    dipole_E: Optional[np.ndarray] = None   # float64 [nt] dipole field samples (Eq. 4), or None
    dipole_M: Optional[np.ndarray] = None   # complex128 [nb, nb] Hermitian dipole coupling
    corr_tol: float = 0.0         # Algorithm 1's epsilon (0: always n_corr corrector passes)
    quadrature: int = 0           # collision-integral weights: 0 trapezoid, 1 Gregory

    @property
    def nk(self) -> int:
        return self.L[0] * self.L[1]


def pair_pattern(nb: int) -> np.ndarray:
    """v_ab = 1 - delta_ab: every pair of distinct bands interacts on site."""
    return np.ones((nb, nb)) - np.eye(nb)


def ring_hoppings_c1(nb: int = 2) -> Tuple[np.ndarray, np.ndarray]:
    """Hoppings giving eps_b(k) = -2 cos(k + b pi/2) + 0.5 b on a 1-D ring."""
    R = np.array([[0, 0], [1, 0], [-1, 0]], dtype=np.int32)
    T = np.zeros((3, nb, nb), dtype=np.complex128)
    for b in range(nb):
        phase = b * math.pi / 2
        T[0, b, b] = 0.5 * b
        T[1, b, b] = -np.exp(1j * phase)
        T[2, b, b] = -np.exp(-1j * phase)
    return R, T


def square_hoppings(nb: int, offset: float, sigma: float,
                    rng: np.random.Generator) -> Tuple[np.ndarray, np.ndarray]:
    """Nearest-neighbour square-lattice bands plus seeded R=0 couplings.

    eps_b(k) = -2 (cos kx + cos ky) + b * offset on the diagonal; for a < b the
    R = 0 entry t_ab gets re, im ~ N(0, sigma) (drawn in row-major a<b order,
    re then im) and t_ba = conj(t_ab).
    """
    R = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1]], dtype=np.int32)
    T = np.zeros((5, nb, nb), dtype=np.complex128)
    for b in range(nb):
        T[0, b, b] = b * offset
        for r in range(1, 5):
            T[r, b, b] = -1.0
    for a in range(nb):
        for b in range(a + 1, nb):
            re, im = rng.normal(0.0, sigma, size=2)
            T[0, a, b] = re + 1j * im
            T[0, b, a] = re - 1j * im
    return R, T


def pulse(nt: int, dt: float, A0: float, t0: float = 5.0, sigma: float = 1.5,
          omega: float = 2.0) -> np.ndarray:
    """A(t) = A0 exp(-(t-t0)^2 / 2 sigma^2) cos(omega t) at t_{i+1/2}, i < nt."""
    t = (np.arange(nt) + 0.5) * dt
    return A0 * np.exp(-(t - t0) ** 2 / (2 * sigma ** 2)) * np.cos(omega * t)


def config(name: str, nt: Optional[int] = None) -> System:
    """The named workload; ``nt`` truncates (or extends) the number of steps."""
    if name == "c1":
        R, T = ring_hoppings_c1(2)
        s = System("c1", 2, 1, (8, 1), 64, 0.05, 0.5, 10.0, 0.0, R, T,
                   pair_pattern(2), None, (1.0, 0.0), hf=1, paper_shift=1, seed=0)
    elif name == "c2":
        rng = np.random.default_rng(1)
        R, T = square_hoppings(4, 0.4, 0.1, rng)
        s = System("c2", 4, 2, (8, 8), 512, 0.02, 1.0, 20.0, 0.0, R, T,
                   pair_pattern(4), pulse(512, 0.02, 0.3), (1.0, 0.0), seed=1)
    elif name == "c3":
        rng = np.random.default_rng(2)
        R, T = square_hoppings(8, 0.25, 0.1, rng)
        s = System("c3", 8, 2, (16, 16), 512, 0.02, 1.5, 20.0, 0.0, R, T,
                   pair_pattern(8), pulse(512, 0.02, 0.5), (1.0, 0.0), seed=2)
    elif name == "paper":
        R, T = paper_hoppings(1.0)
        dt, n_t = 0.02, 500
        s = System("paper", 2, 1, (1024, 1), n_t, dt, 0.5, 10.0, 0.0, R, T, pair_pattern(2), None,
                   (1.0, 0.0), hf=1, paper_shift=1, seed=5)
        s.dipole_M = np.array([[0, 1], [1, 0]], dtype=np.complex128)
        s.dipole_E = kick(n_t, dt, 0.5, 0.1)
    else:
        raise KeyError(name)
    if nt is not None:
        s.nt = nt
        if s.A is not None:
            s.A = pulse(nt, s.dt, _pulse_amp(name))
        if s.dipole_E is not None:
            s.dipole_E = kick(nt, s.dt, 0.5, 0.1)
    return s


def paper_hoppings(Eg: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """eps_v(k) = -2(1 - cos k) - Eg/2, eps_c(k) = 2(1 - cos k) + Eg/2 as hoppings"""
    R = np.array([[0, 0], [1, 0], [-1, 0]], dtype=np.int32)
    T = np.zeros((3, 2, 2), dtype=np.complex128)
    T[0, 0, 0], T[1, 0, 0], T[2, 0, 0] = -2 - Eg / 2, 1.0, 1.0
    T[0, 1, 1], T[1, 1, 1], T[2, 1, 1] = 2 + Eg / 2, -1.0, -1.0
    return R, T


def kick(nt: int, dt: float, t_p: float, intensity: float) -> np.ndarray:
    """I delta(t - t_p) as step-averaged samples: I / dt in the step containing t_p"""
    E = np.zeros(nt)
    i = int(np.floor(t_p / dt + 1e-9))
    if 0 <= i < nt:
        E[i] = intensity / dt
    return E


def _pulse_amp(name: str) -> float:
    return {"c2": 0.3, "c3": 0.5}[name]


def batched(n_sys: int = 64, seed: int = 3) -> List[System]:
    """Uneven batch: N_b in {2,4,6,8,12,16}, L^2 in {16,36,64,100,144},
    N_t ~ U{256..1024}, U ~ U(0.2, 2), A0 ~ U(0, 0.5); drawn in that order
    per system from one PCG64 stream, couplings drawn after A0."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sys):
        nb = int(rng.choice([2, 4, 6, 8, 12, 16]))
        L = int(rng.choice([4, 6, 8, 10, 12]))
        nt = int(rng.integers(256, 1025))
        U = float(rng.uniform(0.2, 2.0))
        A0 = float(rng.uniform(0.0, 0.5))
        R, T = square_hoppings(nb, 0.4, 0.1, rng)
        out.append(System(f"c4.{s}", nb, 2, (L, L), nt, 0.02, U, 20.0, 0.0, R, T,
                          pair_pattern(nb), pulse(nt, 0.02, A0), (1.0, 0.0), seed=seed))
    return out


def targets(nk: int, nb: int, seed: int = 4) -> np.ndarray:
    """Target occupations n*_kb ~ U(0, 1) for the adjoint loss."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(nk, nb))


def small_system(nb: int, L: Tuple[int, int], nt: int, dt: float, U: float,
                 seed: int, drive_amp: float = 0.0, beta: float = 10.0,
                 mu: float = 0.0, hf: int = 1, paper_shift: int = 0,
                 n_corr: int = 2, band_velocity: float = 0.0) -> System:
    """A seeded test system of arbitrary size (square-lattice bands).

    band_velocity s scales the R != 0 hoppings of band b by (1 + s b), so that
    the bands disperse differently and a Peierls drive changes occupations
    even without interaction (equal dispersions only add a phase).
    """
    rng = np.random.default_rng(seed)
    dim = 1 if L[1] == 1 else 2
    R, T = square_hoppings(nb, 0.3, 0.1, rng)
    if dim == 1:
        keep = [0, 1, 2]
        R, T = R[keep].copy(), T[keep].copy()
    for b in range(nb):
        T[1:, b, b] *= 1.0 + band_velocity * b
    A = pulse(nt, dt, drive_amp, t0=nt * dt / 3, sigma=nt * dt / 8, omega=2.0) if drive_amp else None
    return System(f"small{nb}x{L}", nb, dim, L, nt, dt, U, beta, mu, R, T,
                  pair_pattern(nb), A, (1.0, 0.0), hf=hf, paper_shift=paper_shift,
                  n_corr=n_corr, seed=seed)


def random_blocks(rng: np.random.Generator, shape, scale: float = 1.0) -> np.ndarray:
    """Complex normal test tensor (re, im ~ N(0, scale^2 / 2))."""
    z = rng.normal(0.0, scale / math.sqrt(2), size=tuple(shape) + (2,))
    return z[..., 0] + 1j * z[..., 1]
