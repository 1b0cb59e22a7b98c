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
