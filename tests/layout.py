"""Layout conversion between the oracle ([m][k][a][b] per component) and the
CUDA library's device layout ([m][x][a][b][k]); test-side only."""
import numpy as np


def to_dev_blocks(Xl: np.ndarray, Xg: np.ndarray) -> np.ndarray:
    """two [m, nk, nb, nb] arrays -> [m, 2, nb, nb, nk] complex128"""
    return np.ascontiguousarray(np.stack([Xl, Xg], axis=1).transpose(0, 1, 3, 4, 2))


def from_dev_blocks(D: np.ndarray):
    """[m, 2, nb, nb, nk] -> (lesser, greater) each [m, nk, nb, nb]"""
    X = D.transpose(0, 1, 4, 2, 3)
    return np.ascontiguousarray(X[:, 0]), np.ascontiguousarray(X[:, 1])


def to_dev_perk(M: np.ndarray) -> np.ndarray:
    """[nk, nb, nb] -> [nb, nb, nk]"""
    return np.ascontiguousarray(M.transpose(1, 2, 0))


def from_dev_perk(M: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(M.transpose(2, 0, 1))


def tri(i, j):
    return i * (i + 1) // 2 + j


def relerr(a, b, floor_frac=1e-4, scale=None):
    """max |a-b| / max(|b|, 1e-4 * scale) (zero-entry floor) and the normwise
    max|a-b| / scale, scale = max|b| unless given."""
    a, b = np.asarray(a), np.asarray(b)
    scale = np.abs(b).max() if scale is None else scale
    if scale == 0:
        return float(np.abs(a).max()), float(np.abs(a).max())
    den = np.maximum(np.abs(b), floor_frac * scale)
    return float((np.abs(a - b) / den).max()), float(np.abs(a - b).max() / scale)
