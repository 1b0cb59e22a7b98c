"""Pins of the oracle's staggered GMLS (Sec. 2.4).

* The line integrals of Eq. vector-xi, taken by quadrature in the oracle,
  equal the closed form eps xi_c xi^alpha / (alpha! (|alpha| + 1)) for the
  scaled vector monomials phi = e_c xi^alpha / alpha!.
* Their span: the monomials of degree 1..m+1, so rank(Xi) = C(m+1+d, d) - 1,
  below the d C(m+d, d) columns (the dependent columns are why the oracle
  solves with a pseudo-inverse).
* Exactness: q_h = grad p for every p of degree <= m+1 (grad p is in pi_m^v),
  so the Laplacian and gradient stencils reproduce them; constants are
  annihilated.
* A second formulation, written independently: the stencil equals the scalar
  GMLS of degree m+1 without the constant (C oracle, custom basis table) on
  the differences p_j - p(x_T), with the target's own weight minus the sum.
* Convergence on a smooth field at rate m (second derivatives of a degree
  m+1 reconstruction).
"""
from math import comb, factorial

import numpy as np
import pytest

import oracle
from oracle import basis as obasis
from paper_2104_14447_gb300 import inputs
from tests import _poly


def _case(dim, na, k, seed=0):
    x = inputs.jittered_grid(dim, na, seed=seed)
    n = x.shape[1]
    tg = np.arange(0, n, max(1, n // 40), dtype=np.int32)
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off = np.arange(0, len(tg) * k + 1, k)
    return x, tg, idx, eps, off


@pytest.mark.parametrize("dim,m", [(2, 1), (2, 3), (3, 2)])
def test_line_integrals_closed_form(dim, m):
    rng = np.random.default_rng(dim * 10 + m)
    dx = rng.uniform(-1, 1, (7, dim)) * 0.1
    eps = 0.23
    Xi = oracle.staggered_xi(dx, eps, dim, m)
    alphas = obasis.graded_exponents(dim, m)
    col = 0
    for c in range(dim):
        for a in alphas:
            xi = dx / eps
            mono = np.prod([xi[:, k] ** a[k] for k in range(dim)], axis=0)
            fact = np.prod([factorial(v) for v in a[:dim]])
            ref = eps * xi[:, c] * mono / (fact * (sum(a) + 1))
            assert np.allclose(Xi[:, col], ref, rtol=1e-13, atol=1e-16)
            col += 1


@pytest.mark.parametrize("dim,m,k", [(2, 2, 24), (2, 4, 48), (3, 2, 40)])
def test_rank_is_the_span_of_degree_1_to_m_plus_1(dim, m, k):
    x, tg, idx, eps, off = _case(dim, 14 if dim == 2 else 8, k)
    _, ranks = oracle.staggered_stencils(x, tg, off, idx.reshape(-1), eps, m, "laplacian")
    assert np.all(ranks == comb(m + 1 + dim, dim) - 1)
    assert comb(m + 1 + dim, dim) - 1 < dim * comb(m + dim, dim)


@pytest.mark.parametrize("dim,m,k", [(2, 2, 24), (2, 3, 36), (2, 4, 48), (3, 2, 40)])
@pytest.mark.parametrize("name", ["laplacian", "grad"])
def test_polynomials_of_degree_m_plus_1_are_reproduced(dim, m, k, name):
    rng = np.random.default_rng(3 * m + dim)
    x, tg, idx, eps, off = _case(dim, 14 if dim == 2 else 8, k)
    w, _ = oracle.staggered_stencils(x, tg, off, idx.reshape(-1), eps, m, name)
    for _ in range(3):
        p = _poly.random_poly(rng, dim, m + 1)
        vals = _poly.evaluate(p, x)
        if name == "laplacian":
            exact_all = _poly.evaluate(_poly.laplacian(p, dim), x)[None, :]
        else:
            exact_all = np.stack([_poly.evaluate(_poly.deriv(p, c), x) for c in range(dim)])
        for q, t in enumerate(tg):
            nb = idx[q]
            approx = w[q, :, :, 0] @ vals[nb]
            exact = exact_all[:, t]
            scale = np.abs(w[q, :, :, 0]) @ np.abs(vals[nb]) + 1.0
            assert np.all(np.abs(approx - exact) <= 1e-10 * scale)
    assert np.allclose(w.sum(axis=2), 0.0, atol=1e-9 * np.abs(w).sum(axis=2).max())


@pytest.mark.parametrize("dim,m,k", [(2, 2, 24), (2, 4, 48), (3, 2, 40)])
def test_equals_interpolating_scalar_gmls(dim, m, k):
    x, tg, idx, eps, off = _case(dim, 14 if dim == 2 else 8, k)
    w, _ = oracle.staggered_stencils(x, tg, off, idx.reshape(-1), eps, m, "laplacian")
    table = obasis.basis_table(obasis.taylor_basis(dim, m + 1)[1:], 1)  # no constant
    w2, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, "scalar", m + 1, "laplacian", basis_table=table)
    for q, t in enumerate(tg):
        v = w2[q, 0, :, 0].copy()
        s = int(np.flatnonzero(idx[q] == t)[0])
        v[s] = 0.0
        v[s] = -v.sum()
        assert np.allclose(w[q, 0, :, 0], v, rtol=1e-9, atol=1e-9 * np.abs(v).max())


def test_convergence_rate():
    errs, hs = [], []
    m, k = 2, 24
    for na in (16, 24, 36):
        x = inputs.jittered_grid(2, na, seed=1)
        n = x.shape[1]
        # interior targets only (one-sided stencils converge at the same rate
        # with larger constants)
        inner = np.flatnonzero(np.all((x > 0.25) & (x < 0.75), axis=0)).astype(np.int32)
        idx, eps = oracle.knn(x, inner, k, 1.5, method="grid")
        off = np.arange(0, len(inner) * k + 1, k)
        w, _ = oracle.staggered_stencils(x, inner, off, idx.reshape(-1), eps, m, "laplacian")
        f = np.sin(2 * x[0]) * np.cos(3 * x[1])
        lap = -13.0 * f
        approx = np.einsum("tk,tk->t", w[:, 0, :, 0], f[idx])
        errs.append(np.abs(approx - lap[inner]).max())
        hs.append(1.0 / na)
    rate = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert rate > m - 0.5, (rate, errs)
