"""Pins of the oracle's Neumann-constrained GMLS (Sec. 2.3).

The constrained problem (Eqs. neumann-optimization-1..3) reproduces every
q in pi_m that satisfies its own constraint, so for all q of degree <= m:
    sum_j w_j q(x_j) + beta * (n . grad q)(x_T) = (L q)(x_T),
where beta is the coefficient of h (R_uh applied by the functional, the
paper's beta_I for the Laplacian, Eq. grad-pressure-stencil-1).  The weights
are also compared with the saddle-point system of Eq.
(neumann-saddle-point-system) solved directly in 50-digit arithmetic.
"""
import itertools

import mpmath
import numpy as np
import pytest

import oracle
from paper_2104_14447_gb300 import inputs
from tests import _poly


def _fixed_k(idx):
    nt, k = idx.shape
    return np.arange(0, nt * k + 1, k, dtype=np.int64), idx.reshape(-1)


def _boundary_case(dim, seed):
    x = inputs.jittered_grid(dim, 14 if dim == 2 else 7, seed=seed)
    n = x.shape[1]
    tg = np.arange(0, n, 29, dtype=np.int32)[:12]
    nrm = inputs.unit_vectors(seed, 3, len(tg), dim).T.copy()
    return x, tg, nrm


@pytest.mark.parametrize("dim,m,k", [(2, 2, 12), (2, 4, 36), (3, 3, 40)])
@pytest.mark.parametrize("name", ["laplacian", "grad"])
def test_constrained_reproduction(dim, m, k, name):
    rng = np.random.default_rng(7 * m + dim)
    x, tg, nrm = _boundary_case(dim, 21)
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    bflag = np.ones(len(tg), np.uint8)
    w, beta, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name, bflag=bflag, normals=nrm)
    for q, t in enumerate(tg):
        poly = _poly.random_poly(rng, dim, m)
        d = x[:, idx[q]] - x[:, t:t + 1]
        vals = _poly.evaluate(poly, d)
        h = sum(nrm[q, c] * _poly.deriv(poly, c).get((0, 0, 0), 0.0) for c in range(dim))
        if name == "laplacian":
            want = np.array([_poly.laplacian(poly, dim).get((0, 0, 0), 0.0)])
        else:
            want = np.array([_poly.deriv(poly, c).get((0, 0, 0), 0.0) for c in range(dim)])
        got = w[q, :, :, 0] @ vals + beta[q] * h
        scale = np.abs(w[q, :, :, 0]) @ np.abs(vals) + np.abs(beta[q] * h)
        assert np.all(np.abs(got - want) <= 1e-11 * scale + 1e-11), (q, got, want)
    # unconstrained targets in the same call are untouched by the constraint
    w0, beta0, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name)
    bmix = (np.arange(len(tg)) % 2).astype(np.uint8)
    wm, betam, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, name, bflag=bmix, normals=nrm)
    np.testing.assert_array_equal(wm[bmix == 0], w0[bmix == 0])
    np.testing.assert_array_equal(wm[bmix == 1], w[bmix == 1])
    assert np.all(betam[bmix == 0] == 0.0)


def _monomials(dim, m):
    out = []
    for s in range(m + 1):
        for a in itertools.product(range(s + 1), repeat=dim):
            if sum(a) == s:
                out.append(tuple(a) + (0,) * (3 - dim))
    return out


@pytest.mark.parametrize("dim,m,k", [(2, 2, 12), (3, 2, 16)])
def test_kkt_extended_precision(dim, m, k):
    """[[P^T W P, F], [F^T, 0]] z = [lambda^T; 0]  =>  w = W P z_c, beta = z_mu."""
    mpmath.mp.dps = 50
    x, tg, nrm = _boundary_case(dim, 5)
    tg, nrm = tg[:5], nrm[:5]
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    w, beta, _ = oracle.stencils(x, tg, off, flat, eps, "scalar", m, "laplacian", bflag=np.ones(len(tg), np.uint8),
                                 normals=nrm)
    mons = _monomials(dim, m)
    Q = len(mons)
    for q, t in enumerate(tg):
        rows, ws = [], []
        for j in idx[q]:
            d = [mpmath.mpf(float(x[c, j])) - mpmath.mpf(float(x[c, t])) for c in range(dim)]
            r = mpmath.sqrt(sum(di * di for di in d))
            ws.append((1 - r / mpmath.mpf(float(eps[q]))) ** 4)
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
        # F = grad p(x_T)^T n: d/dx_c of (x - x_T)^alpha at x_T is 1 for alpha = e_c
        F = [mpmath.mpf(float(nrm[q, a.index(1)])) if sum(a) == 1 else mpmath.mpf(0) for a in mons]
        K = mpmath.zeros(Q + 1, Q + 1)
        for i in range(Q):
            for j in range(Q):
                K[i, j] = A[i, j]
            K[i, Q] = F[i]
            K[Q, i] = F[i]
        lam = [2.0 if (sum(a) == 2 and max(a) == 2) else 0.0 for a in mons] + [0.0]
        z = mpmath.lu_solve(K, mpmath.matrix(lam))
        zc = mpmath.matrix([z[i] for i in range(Q)])
        wmp = np.array([float(v) for v in Wm * P * zc])
        assert np.max(np.abs(w[q, 0, :, 0] - wmp)) <= 1e-11 * np.max(np.abs(wmp))
        assert abs(beta[q, 0] - float(z[Q])) <= 1e-11 * max(1.0, abs(float(z[Q])))
