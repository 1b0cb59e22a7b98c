"""Pins of the oracle's divergence-free vector GMLS (Sec. 2.2, Sec. 3.1).

* every basis function has exactly zero divergence (rational arithmetic);
* the basis spans the whole kernel of div on (pi_m)^d, whose dimension is
  computed here by exact rank of the divergence map;
* for d = 2, m = 2 the span equals the nine functions printed in Sec. 2.2;
* vector stencils reproduce divergence-free polynomial fields, among them the
  paper's manufactured velocities (Sec. 4.1), whose Laplacians are fixtures;
* curl curl = -Laplacian on divergence-free fields (vector identity of
  Sec. 3.1), and the divergence functional vanishes on the basis.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import basis
from paper_2104_14447_gb300 import inputs
from tests import _poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixed_k(idx):
    nt, k = idx.shape
    return np.arange(0, nt * k + 1, k, dtype=np.int64), idx.reshape(-1)


def _vec(func, dim):
    """basis function -> dict {(comp, gamma): Fraction}"""
    out = {}
    for c in range(dim):
        for coef, g in func[c]:
            out[(c, g)] = out.get((c, g), 0) + Fraction(coef)
    return {k: v for k, v in out.items() if v != 0}


def _rank(vecs):
    return basis._rank(vecs)


def _div(vec, dim):
    out = {}
    for (c, g), v in vec.items():
        if g[c] == 0:
            continue
        h = list(g)
        h[c] -= 1
        out[tuple(h)] = out.get(tuple(h), 0) + v * g[c]
    return {k: v for k, v in out.items() if v != 0}


def _kernel_dim(dim, m):
    """dim ker(div: (pi_m)^d -> pi_{m-1}) = d*dim(pi_m) - rank(div)."""
    mons = basis.graded_exponents(dim, m)
    images = [_div({(c, a): Fraction(1)}, dim) for c in range(dim) for a in mons]
    return dim * len(mons) - _rank([im for im in images if im] or [{}])


@pytest.mark.parametrize("dim,m", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_divfree_basis_is_exact_and_complete(dim, m):
    funcs = basis.divfree_basis(dim, m)
    vecs = [_vec(f, dim) for f in funcs]
    for v in vecs:
        assert _div(v, dim) == {}
        assert all(sum(g) <= m for (_, g) in v)
    assert _rank(vecs) == len(vecs)  # linearly independent
    assert len(vecs) == _kernel_dim(dim, m) == basis.divfree_dimension(dim, m)
    if dim == 2:
        assert len(vecs) == (m + 1) * (m + 4) // 2


def test_span_equals_paper_2d_m2_example():
    paper = []
    with open(os.path.join(GOLDEN, "divfree_2d_m2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            vx, vy = line.split(";")
            vec = {}
            for c, part in enumerate((vx, vy)):
                for g, coef in _poly.parse_terms(part).items():
                    if coef != 0:
                        vec[(c, g)] = Fraction(coef)
            paper.append(vec)
    assert len(paper) == 9
    for v in paper:
        assert _div(v, 2) == {}
    ours = [_vec(f, 2) for f in basis.divfree_basis(2, 2)]
    assert _rank(paper) == 9 and _rank(ours) == 9 and _rank(paper + ours) == 9


def _load_manufactured():
    fields = {}
    with open(os.path.join(GOLDEN, "manufactured_3d.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, v, lap = (s.strip() for s in line.split("|"))
            fields[name] = ([_poly.parse_terms(p) for p in v.split(";")],
                            [_poly.parse_terms(p) for p in lap.split(";")])
    return fields


def test_manufactured_fixture_is_divergence_free_and_laplacian_consistent():
    for v, lap in _load_manufactured().values():
        div = _poly.add(*[_poly.deriv(v[c], c) for c in range(3)])
        assert all(abs(c) < 1e-14 for c in div.values())
        for c in range(3):
            mine = _poly.laplacian(v[c], 3)
            keys = set(mine) | set(lap[c])
            assert all(abs(mine.get(k, 0) - lap[c].get(k, 0)) < 1e-14 for k in keys)


def _vector_apply(w, x, nbr, field):
    """sum_{j, c} w[r, j, c] v_c(x_j)"""
    vals = np.stack([_poly.evaluate(field[c], x[:, nbr]) for c in range(len(field))], axis=1)  # k x nc
    return np.einsum("rjc,jc->r", w, vals), np.einsum("rjc,jc->r", np.abs(w), np.abs(vals))


@pytest.mark.parametrize("name,m,k", [("quadratic", 2, 42), ("quartic", 3, 80), ("quartic", 4, 136)])
def test_paper_manufactured_velocity_is_reproduced(name, m, k):
    v, lap = _load_manufactured()[name]
    x = inputs.jittered_grid(3, 9, seed=6) * 2.0 - 1.0  # the paper's bi-unit cube
    tg = np.array([364, 300, 420], dtype=np.int32)
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    wl, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", m, "vec_laplacian")
    wc, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", m, "curlcurl")
    wd, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", m, "div")
    for q, t in enumerate(tg):
        got, scale = _vector_apply(wl[q], x, idx[q], v)
        want = np.array([_poly.evaluate(lap[c], x[:, t:t + 1])[0] for c in range(3)])
        assert np.all(np.abs(got - want) <= 1e-11 * scale + 1e-11), (got, want)
        np.testing.assert_allclose(wc[q], -wl[q], atol=1e-10 * np.abs(wl[q]).max())
        assert np.abs(wd[q]).max() <= 1e-10 * np.abs(wl[q]).max() * eps[q]


@pytest.mark.parametrize("m,k", [(2, 22), (3, 34), (4, 48)])
def test_2d_stream_function_fields_are_reproduced(m, k):
    """v = (d_y s, -d_x s) for a random polynomial s of degree m+1 is
    divergence-free of degree m; its vector Laplacian must be reproduced."""
    rng = np.random.default_rng(m)
    x = inputs.jittered_grid(2, 20, seed=8)
    tg = np.arange(21, 400, 37, dtype=np.int32)
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    w, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", m, "vec_laplacian")
    for q, t in enumerate(tg):
        s = _poly.random_poly(rng, 2, m + 1)
        field = [_poly.deriv(s, 1), _poly.add(_poly.deriv(s, 0), scale=[-1])]
        d = x[:, idx[q]] - x[:, t:t + 1]
        vals = np.stack([_poly.evaluate(f, d) for f in field], axis=1)
        got = np.einsum("rjc,jc->r", w[q], vals)
        scale = np.einsum("rjc,jc->r", np.abs(w[q]), np.abs(vals))
        want = np.array([_poly.laplacian(f, 2).get((0, 0, 0), 0.0) for f in field])
        assert np.all(np.abs(got - want) <= 1e-11 * scale + 1e-11)


def _paper_basis_2d_m2():
    """The paper's nine div-free functions of degree <= 2 (Sec. 2.2) as
    [x-component poly, y-component poly] in unscaled offsets."""
    out = []
    with open(os.path.join(GOLDEN, "divfree_2d_m2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            vx, vy = line.split(";")
            out.append([_poly.parse_terms(vx), _poly.parse_terms(vy)])
    return out


def _rref_style_basis(dim, m):
    """A basis of pi^div_m written out here, independently of oracle.basis:
    e_c p_g - e_0 p_(g - e_c + e_0) for c >= 1 (second term when g_c >= 1),
    and e_0 p_g for g_0 = 0, with p_g = x^g / g! (d/dx_k p_g = p_(g - e_k))."""
    from math import factorial

    mons = [a for a in basis.graded_exponents(dim, m)]

    def p(g):
        return {g: 1.0 / (factorial(g[0]) * factorial(g[1]) * factorial(g[2]))}

    out = []
    for c in range(1, dim):
        for g in mons:
            f = [{} for _ in range(dim)]
            f[c] = p(g)
            if g[c] >= 1:
                h = list(g)
                h[c] -= 1
                h[0] += 1
                f[0] = {k: -v for k, v in p(tuple(h)).items()}
            out.append(f)
    for g in mons:
        if g[0] == 0:
            f = [{} for _ in range(dim)]
            f[0] = p(g)
            out.append(f)
    return out


def _vector_tile(funcs, d):
    """P[(j, c), i] = phi_i^c(d_j) for offsets d (dim, k), rows (j, c)."""
    dim, k = d.shape
    P = np.zeros((k * dim, len(funcs)))
    for i, f in enumerate(funcs):
        for c in range(dim):
            P[c::dim, i] = _poly.evaluate(f[c], d)
    return P


@pytest.mark.parametrize("dim,m,k", [(2, 2, 22), (2, 4, 48), (3, 2, 42), (3, 3, 80)])
def test_projection_property_vector(dim, m, k):
    """w = W P y for some y (Sec. 2.2 with the weighted least squares of
    Sec. 2.1): W^{-1} w, over the (neighbour, component) rows, lies in the
    column space of a basis of pi^div_m built here (the paper's nine
    functions for d = 2, m = 2; an independent explicit basis otherwise).
    Together with reproduction of div-free fields this fixes w uniquely."""
    x = inputs.jittered_grid(dim, 14 if dim == 2 else 7, seed=5)
    tg = np.arange(4, x.shape[1], 29, dtype=np.int32)[:12]
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    funcs = _paper_basis_2d_m2() if (dim, m) == (2, 2) else _rref_style_basis(dim, m)
    assert len(funcs) == basis.divfree_dimension(dim, m)
    for name in ("vec_laplacian", "curlcurl"):
        w, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", m, name)
        for q, t in enumerate(tg):
            d = x[:, idx[q]] - x[:, t:t + 1]
            r = np.sqrt(np.sum(d * d, axis=0))
            W = np.repeat(np.clip(1.0 - r / eps[q], 0.0, None) ** 4, dim)  # rows (j, c)
            P = _vector_tile(funcs, d)
            for row in range(w.shape[1]):
                u = w[q, row].reshape(-1) / W
                y, *_ = np.linalg.lstsq(P, u, rcond=None)
                assert np.linalg.norm(P @ y - u) <= 1e-9 * np.linalg.norm(u), (name, q, row)
    # a planted slip: dropping one function from the span breaks the property
    w, _, _ = oracle.stencils(x, tg[:1], off[:2], flat[:k], eps[:1], "divfree", m, "vec_laplacian")
    d = x[:, idx[0]] - x[:, tg[0]:tg[0] + 1]
    W = np.repeat(np.clip(1.0 - np.sqrt(np.sum(d * d, axis=0)) / eps[0], 0.0, None) ** 4, dim)
    P = _vector_tile(funcs[:-1], d)
    resid = [np.linalg.norm(P @ np.linalg.lstsq(P, w[0, r].reshape(-1) / W, rcond=None)[0] - w[0, r].reshape(-1) / W)
             / np.linalg.norm(w[0, r].reshape(-1) / W) for r in range(w.shape[1])]
    assert max(resid) > 1e-6


def test_extended_precision_normal_equations_vector():
    """w = W P (P^T W P)^{-1} lambda^T in 50-digit arithmetic on a tiny 2D
    cloud, P from the paper's nine div-free functions of degree 2 (Sec. 2.2)
    in unscaled offsets, lambda_i = Laplacian of component l of function i
    at the target; the oracle (its own scaled curl basis, Householder QR)
    must agree to 1e-12 relative."""
    import mpmath

    mpmath.mp.dps = 50
    funcs = _paper_basis_2d_m2()
    x = inputs.jittered_grid(2, 7, seed=12)
    tg = np.array([16, 24, 32], dtype=np.int32)
    k = 14
    idx, eps = oracle.knn(x, tg, k, 1.5)
    off, flat = _fixed_k(idx)
    w, _, _ = oracle.stencils(x, tg, off, flat, eps, "divfree", 2, "vec_laplacian")
    lap = [[_poly.laplacian(f[c], 2).get((0, 0, 0), 0.0) for f in funcs] for c in range(2)]
    for q, t in enumerate(tg):
        rows, ws = [], []
        for j in idx[q]:
            dd = [mpmath.mpf(float(x[c, j])) - mpmath.mpf(float(x[c, t])) for c in range(2)]
            Wj = (1 - mpmath.sqrt(dd[0] ** 2 + dd[1] ** 2) / mpmath.mpf(float(eps[q]))) ** 4
            for c in range(2):
                row = []
                for f in funcs:
                    v = mpmath.mpf(0)
                    for (a0, a1, _), coef in f[c].items():
                        v += mpmath.mpf(coef) * dd[0] ** a0 * dd[1] ** a1
                    row.append(v)
                rows.append(row)
                ws.append(Wj)
        P = mpmath.matrix(rows)
        Wm = mpmath.diag(ws)
        A = P.T * Wm * P
        for l in range(2):
            yv = mpmath.lu_solve(A, mpmath.matrix(lap[l]))
            want = np.array([float(v) for v in Wm * P * yv]).reshape(k, 2)
            got = w[q, l]
            assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), (q, l)
