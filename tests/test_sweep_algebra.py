"""The algebra the collision-sweep kernels and their transposes rely on,
checked on the CPU against the oracle's collision row (Eq. 6 summed as written).

* (I^<, I^> - I^<) form: with C1 = w^(n)_l (S^> - S^<), C2 = dt S^<,
  C3 = dt S^> - C1 and f = w^(j)_l / dt, the kernels accumulate
  X(j) = sum_l C1 X_lj + sum_{l<=j} f C2 D_lj and
  Y(j) = -sum_{l>j} C1 D_lj + sum_{l<=j} (f (C3 - C2) + (f - 1) C1) D_lj,
  skipping Y at the interior nodes of [0, t_j], where both quadratures weigh
  the node dt. I^< = X, I^> = X + Y must equal the oracle's row.
* The reverse mode's transposes of that form (lam of the Sigma row, lam of
  every stored block) must pass a dot-product test against the oracle's
  forward, which is linear in the history for a fixed Sigma row and linear
  in the Sigma row for a fixed history.

Trapezoid and fourth-order Gregory weights; the models below are plain loops
over blocks, written from those formulas."""
import numpy as np
import pytest

import oracle


def omega(quad, m, l):
    """w^(m)_l / dt: trapezoid; Gregory with the end weights 3/8, 7/6, 23/24
    (Newton-Cotes rules for m <= 4)"""
    if m == 0:
        return 0.0
    if quad == 0 or m == 1:
        return 0.5 if l in (0, m) else 1.0
    if m == 2:
        return [1 / 3, 4 / 3, 1 / 3][l]
    if m == 3:
        return [3 / 8, 9 / 8, 9 / 8, 3 / 8][l]
    if m == 4:
        return [14 / 45, 64 / 45, 24 / 45, 64 / 45, 14 / 45][l]
    e = min(l, m - l)
    return [3 / 8, 7 / 6, 23 / 24][e] if e <= 2 else 1.0


def tri(i, j):
    return i * (i + 1) // 2 + j


def cT(a):
    return np.conj(np.swapaxes(a, -1, -2))


def interior(quad, j, l):
    return (0 < l < j) if quad == 0 else (3 <= l <= j - 3)


def xy_row(n, dt, Hl, dG, Sl, Sg, quad):
    C1 = np.array([dt * omega(quad, n, l) * (Sg[l] - Sl[l]) for l in range(n + 1)])
    C2, C3 = dt * Sl, dt * Sg - C1
    X = np.zeros_like(Sl)
    Y = np.zeros_like(Sl)
    for j in range(n + 1):
        for l in range(n + 1):
            if l >= j:
                G, D = Hl[tri(l, j)], dG[tri(l, j)]
            else:
                G, D = -cT(Hl[tri(j, l)]), -cT(dG[tri(j, l)])
            X[j] += C1[l] @ G
            if l > j or j == 0:
                Y[j] -= C1[l] @ D
            elif interior(quad, j, l):
                X[j] += C2[l] @ D
            else:
                f = omega(quad, j, l)
                X[j] += f * C2[l] @ D
                Y[j] += (f * (C3[l] - C2[l]) + (f - 1) * C1[l]) @ D
    return X, X + Y


def adj_sigma(n, dt, Hl, dG, LL, LG, quad):
    LX, LY = LL + LG, LG
    out_l, out_g = np.zeros_like(LL), np.zeros_like(LL)
    for l in range(n + 1):
        wn = dt * omega(quad, n, l)
        jb = l + 1 if quad == 0 else max(l + 3, 5)
        t1, t2, t3, s3, s4 = (np.zeros_like(LL[0]) for _ in range(5))
        for j in range(n + 1):
            if j < l:
                t1 += LX[j] @ cT(Hl[tri(l, j)])
                t2 += LY[j] @ cT(dG[tri(l, j)])
            elif j == l or j < jb:
                G, D = (Hl[tri(l, l)], dG[tri(l, l)]) if j == l else (Hl[tri(j, l)], dG[tri(j, l)])
                sgn = 1 if j == l else -1
                t1 += sgn * (LX[j] @ (cT(G) if j == l else G))
                P = sgn * (LX[j] @ (cT(D) if j == l else D))
                Q = sgn * (LY[j] @ (cT(D) if j == l else D))
                wj = dt * omega(quad, j, l)
                s3 += wj * P
                s4 += (wj - wn) * Q
            else:
                t1 -= LX[j] @ Hl[tri(j, l)]
                t3 -= LX[j] @ dG[tri(j, l)]
        ld = wn * (t1 - t2) + s4
        out_g[l] = ld
        out_l[l] = s3 + wn * t3 - ld
    return out_l, out_g


def adj_history(n, dt, Sl, Sg, LL, LG, quad):
    LX, LY = LL + LG, LG
    Delta = Sg - Sl
    w = lambda m, l: dt * omega(quad, m, l)
    C1 = np.array([w(n, l) * Delta[l] for l in range(n + 1)])
    ntri = tri(n, n) + 1
    lam_l = np.zeros((ntri,) + LL.shape[1:], complex)
    lam_g = np.zeros_like(lam_l)
    for i in range(n + 1):
        for jp in range(i + 1):
            if jp < i:
                gl = cT(C1[i]) @ LX[jp] - cT(cT(C1[jp]) @ LX[i])
                gd = -(cT(C1[i]) @ LY[jp]) - cT(w(i, jp) * (cT(Sl[jp]) @ LX[i])
                                               + (w(i, jp) - w(n, jp)) * (cT(Delta[jp]) @ LY[i]))
            else:
                gl = cT(C1[i]) @ LX[i]
                gd = w(i, i) * (cT(Sl[i]) @ LX[i]) + (w(i, i) - w(n, i)) * (cT(Delta[i]) @ LY[i])
            lam_l[tri(i, jp)] = gl + gd
            lam_g[tri(i, jp)] = -gd
    return lam_l, lam_g


CASES = [(2, 3, 7), (3, 2, 9), (1, 2, 4), (2, 2, 1), (2, 1, 12)]


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,nk,n", CASES)
def test_xy_form_equals_the_collision_row(nb, nk, n, quad):
    rng = np.random.default_rng(11 * nb + n)
    cz = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    ntri = tri(n, n) + 1
    Hl, Hg = cz(ntri, nk, nb, nb), cz(ntri, nk, nb, nb)
    Sl, Sg = cz(n + 1, nk, nb, nb), cz(n + 1, nk, nb, nb)
    Il, Ig = oracle.collision_row(nb, nk, n, 0.05, Hl, Hg, Sl, Sg, quadrature=quad)
    Xl, Xg = xy_row(n, 0.05, Hl, Hl - Hg, Sl, Sg, quad)
    scale = max(np.abs(Il).max(), np.abs(Ig).max())
    assert np.abs(Xl - Il).max() < 1e-13 * scale
    assert np.abs(Xg - Ig).max() < 1e-13 * scale


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("nb,nk,n", CASES)
def test_xy_transposes_pass_the_dot_product_test(nb, nk, n, quad):
    rng = np.random.default_rng(7 * nb + n)
    cz = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    ip = lambda a, b: np.real(np.vdot(a, b))
    ntri = tri(n, n) + 1
    Hl, Hg = cz(ntri, nk, nb, nb), cz(ntri, nk, nb, nb)
    Sl, Sg = cz(n + 1, nk, nb, nb), cz(n + 1, nk, nb, nb)
    LL, LG = cz(n + 1, nk, nb, nb), cz(n + 1, nk, nb, nb)
    dSl, dSg = cz(n + 1, nk, nb, nb), cz(n + 1, nk, nb, nb)
    dHl, dHg = cz(ntri, nk, nb, nb), cz(ntri, nk, nb, nb)
    F = lambda hl, hg, sl, sg: oracle.collision_row(nb, nk, n, 0.05, hl, hg, sl, sg, quadrature=quad)
    # linear in the Sigma row for a fixed history
    Il, Ig = F(Hl, Hg, dSl, dSg)
    aL, aG = adj_sigma(n, 0.05, Hl, Hl - Hg, LL, LG, quad)
    lhs, rhs = ip(LL, Il) + ip(LG, Ig), ip(aL, dSl) + ip(aG, dSg)
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)
    # linear in the history for a fixed Sigma row
    Il, Ig = F(dHl, dHg, Sl, Sg)
    hL, hG = adj_history(n, 0.05, Sl, Sg, LL, LG, quad)
    lhs, rhs = ip(LL, Il) + ip(LG, Ig), ip(hL, dHl) + ip(hG, dHg)
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_a_dropped_y_term_fails():
    """the interior skip is only valid where both weights are dt: applying it
    at an end node (here l = 0 of the trapezoid) must break the equality"""
    rng = np.random.default_rng(5)
    cz = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    nb, nk, n = 2, 2, 6
    ntri = tri(n, n) + 1
    Hl, Hg = cz(ntri, nk, nb, nb), cz(ntri, nk, nb, nb)
    Sl, Sg = cz(n + 1, nk, nb, nb), cz(n + 1, nk, nb, nb)
    Il, Ig = oracle.collision_row(nb, nk, n, 0.05, Hl, Hg, Sl, Sg, quadrature=0)
    global interior
    keep = interior
    try:
        interior = lambda quad, j, l: 0 <= l < j   # wrongly treats l = 0 as interior
        Xl, Xg = xy_row(n, 0.05, Hl, Hl - Hg, Sl, Sg, 0)
    finally:
        interior = keep
    assert np.abs(Xl - Il).max() > 1e-6 * np.abs(Il).max()
