"""Pins of the oracle's scalar GMLS stencils (Sec. 2.1 and 2.5).

Each check comes from outside the oracle: textbook finite differences, a
square system solved by numpy, exact polynomial reproduction (Sec. 2.1: the
approximation is exact on pi_m), the weighted least-squares projection
property, and the normal equations (Eqs. matrix-A, matrix-B, vector-c) solved
in 50-digit arithmetic.  Together, reproduction (P^T w = lambda^T) and the
projection property (W^{-1} w in col P) determine w uniquely.
"""
import itertools
from math import factorial

import mpmath
import numpy as np
import pytest

import oracle
from paper_2104_14447_gb300 import inputs
from tests import _poly


def _fixed_k(idx):
    nt, k = idx.shape
    return np.arange(0, nt * k + 1, k, dtype=np.int64), idx.reshape(-1)


def _monomials(dim, m):
    out = []
    for s in range(m + 1):
        for a in itertools.product(range(s + 1), repeat=dim):
            if sum(a) == s:
                out.append(tuple(a) + (0,) * (3 - dim))
    return out


@pytest.mark.parametrize("m,second,first", [
    (2, [1, -2, 1], [-1, 0, 1]),
    (4, [-1, 16, -30, 16, -1], [1, -8, 0, 8, -1]),
])
def test_1d_square_case_is_central_difference(m, second, first):
    """k = m + 1 collinear points: the unique interpolant gives the classical
    central differences (h^2 f'' = [1,-2,1], [-1,16,-30,16,-1]/12 ...)."""
    h = 0.125
    half = m // 2
    xs = np.array([[(i - half) * h for i in range(m + 1)]]) + 0.5
    t = half
    idx, eps = oracle.knn(xs, np.array([t], np.int32), m + 1, 1.5)
    off, flat = _fixed_k(idx)
    w2, _, _ = oracle.stencils(xs, [t], off, flat, eps, "scalar", m, "laplacian")
    w1, _, _ = oracle.stencils(xs, [t], off, flat, eps, "scalar", m, "grad")
    by_index2 = np.zeros(m + 1)
    by_index1 = np.zeros(m + 1)
    by_index2[idx[0]] = w2[0, 0, :, 0]
    by_index1[idx[0]] = w1[0, 0, :, 0]
    denom2 = 1.0 if m == 2 else 12.0
    denom1 = 2.0 if m == 2 else 12.0
    np.testing.assert_allclose(by_index2 * h * h * denom2, second, atol=1e-11)
    np.testing.assert_allclose(by_index1 * h * denom1, first, atol=1e-11)


@pytest.mark.parametrize("dim,m", [(2, 2), (2, 3), (3, 2)])
def test_square_case_matches_numpy_solve(dim, m):
    """k*1 = Q: w = P^{-T} lambda^T, independent of the weights (interpolatory)."""
    x = inputs.jittered_grid(dim, 7 if dim == 2 else 5, seed=11)
    mons = _monomials(dim, m)
    Q = len(mons)
    tg = np.array([x.shape[1] // 2 + 1], np.int32)
    idx, eps = oracle.knn(x, tg, Q, 1.5)
    off, flat = _fixed_k(idx)
    t = tg[0]
    d = x[:, idx[0]] - x[:, t:t + 1]
    P = np.stack([np.prod([d[c] ** a[c] for c in range(dim)], axis=0) for a in mons], axis=1)  # k x Q
    for name, lam_of in (("laplacian", lambda a: 2.0 * sum(a[c] == 2 and sum(a) == 2 for c in range(dim))),
                         ("grad", None)):
        w, _, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name)
        if name == "laplacian":
            lam = np.array([[lam_of(a) for a in mons]])
        else:
            lam = np.array([[1.0 if a == tuple(int(c == r) for c in range(3)) else 0.0 for a in mons]
                            for r in range(dim)])
        want = np.linalg.solve(P.T, lam.T).T
        np.testing.assert_allclose(w[0, :, :, 0], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
        # changing the weight exponent does not change an interpolatory stencil
        w6, _, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name, wpow=6.0)
        np.testing.assert_allclose(w6, w, rtol=1e-9, atol=1e-9 * np.abs(w).max())


def _exact(poly, name, dim):
    if name == "laplacian":
        return [_poly.laplacian(poly, dim).get((0, 0, 0), 0.0)]
    return [_poly.deriv(poly, k).get((0, 0, 0), 0.0) for k in range(dim)]


@pytest.mark.parametrize("dim,m,k", [(2, 2, 12), (2, 3, 20), (2, 4, 36), (3, 2, 20), (3, 3, 40), (3, 4, 84)])
@pytest.mark.parametrize("name", ["grad", "laplacian"])
def test_polynomial_reproduction(dim, m, k, name):
    """Sec. 2.1: exact on pi_m, so sum_j w_j q(x_j) = (L q)(x_T) for deg q <= m."""
    rng = np.random.default_rng(100 * dim + m)
    x = inputs.jittered_grid(dim, 16 if dim == 2 else 8, seed=m)
    tg = np.arange(0, x.shape[1], 9, dtype=np.int32)[:30]
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    w, _, diag = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name)
    for q, t in enumerate(tg):
        poly = _poly.random_poly(rng, dim, m)
        vals = _poly.evaluate(poly, x[:, idx[q]] - x[:, t:t + 1])
        got = w[q, :, :, 0] @ vals
        want = np.array(_exact(poly, name, dim))
        scale = np.abs(w[q, :, :, 0]) @ np.abs(vals)
        assert np.all(np.abs(got - want) <= 1e-12 * scale + 1e-12), (q, got, want)
    # a wrong degree would break this: a degree m+1 monomial is not reproduced
    bad = {(m + 1, 0, 0): 1.0, (m - 1, 2, 0) if dim > 1 else (m + 1, 0, 0): 1.0}
    vals = _poly.evaluate(bad, x[:, idx[0]] - x[:, tg[0]:tg[0] + 1])
    assert not np.allclose(w[0, :, :, 0] @ vals, _exact(bad, name, dim), atol=1e-6) or m + 1 > 4


@pytest.mark.parametrize("dim,m,k", [(2, 2, 12), (2, 4, 36), (3, 3, 40)])
def test_projection_property(dim, m, k):
    """w = W P y for some y (Eq. vector-c: w^T = lambda A^{-1} P^T W), i.e.
    W^{-1} w lies in the column space of P; the weight is (1 - r/eps)_+^4."""
    x = inputs.jittered_grid(dim, 14 if dim == 2 else 7, seed=4)
    tg = np.arange(3, x.shape[1], 17, dtype=np.int32)[:20]
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    w, _, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, "laplacian")
    mons = _monomials(dim, m)
    for q, t in enumerate(tg):
        d = x[:, idx[q]] - x[:, t:t + 1]
        r = np.sqrt(np.sum(d * d, axis=0))
        W = np.clip(1.0 - r / eps[q], 0.0, None) ** 4
        P = np.stack([np.prod([d[c] ** a[c] for c in range(dim)], axis=0) for a in mons], axis=1)
        u = w[q, 0, :, 0] / W
        y, *_ = np.linalg.lstsq(P, u, rcond=None)
        assert np.linalg.norm(P @ y - u) <= 1e-9 * np.linalg.norm(u)


@pytest.mark.parametrize("dim,m,k", [(2, 2, 12), (2, 3, 16), (3, 2, 14)])
def test_extended_precision_normal_equations(dim, m, k):
    """w = W P (P^T W P)^{-1} lambda^T evaluated in 50-digit arithmetic with
    unscaled monomials (x - x_T)^alpha (a different basis of the same span)."""
    mpmath.mp.dps = 50
    x = inputs.jittered_grid(dim, 8 if dim == 2 else 5, seed=9)
    tg = np.arange(5, x.shape[1], 23, dtype=np.int32)[:6]
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    mons = _monomials(dim, m)
    for name in ("grad", "laplacian"):
        w, _, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name)
        for q, t in enumerate(tg):
            rows = []
            ws = []
            for j in idx[q]:
                d = [mpmath.mpf(float(x[c, j])) - mpmath.mpf(float(x[c, t])) for c in range(dim)]
                r = mpmath.sqrt(sum(di * di for di in d))
                Wj = (1 - r / mpmath.mpf(float(eps[q]))) ** 4
                ws.append(Wj)
                row = []
                for a in mons:
                    v = mpmath.mpf(1)
                    for c in range(dim):
                        v *= d[c] ** a[c]
                    row.append(v)
                rows.append(row)
            P = mpmath.matrix(rows)
            Wm = mpmath.diag(ws)
            A = P.T * Wm * P
            if name == "laplacian":
                lam = [[2.0 if (sum(a) == 2 and max(a) == 2) else 0.0 for a in mons]]
            else:
                lam = [[1.0 if a == tuple(int(c == rr) for c in range(3)) else 0.0 for a in mons] for rr in range(dim)]
            for rr, lrow in enumerate(lam):
                yv = mpmath.lu_solve(A, mpmath.matrix(lrow))
                wmp = Wm * P * yv
                want = np.array([float(v) for v in wmp])
                got = w[q, rr, :, 0]
                assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), (name, q, rr)


def test_householder_qr_matches_numpy():
    rng = np.random.default_rng(0)
    A0 = rng.standard_normal((30, 12))
    A, tau = oracle.qr(A0)
    R = np.triu(A[:12, :12])
    Rn = np.linalg.qr(A0, mode="r")
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rn)), rtol=1e-12)
    np.testing.assert_allclose(R.T @ R, A0.T @ A0, rtol=1e-11, atol=1e-11)
    # Q [R; 0] reproduces A column by column
    for j in range(12):
        z = np.zeros(30)
        z[:12] = R[:, j]
        np.testing.assert_allclose(oracle.apply_q(A, tau, z), A0[:, j], atol=1e-12)
