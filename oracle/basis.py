"""Polynomial bases and target functionals for the oracle, as exact term tables.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  Nothing here is
shared with the CUDA path, which builds its own tables differently.

A basis function psi_i (scalar, or a vector with ``nc`` components) is a sum of
terms ``coef * xi^gamma`` in the scaled offset ``xi = (x - x_T) / eps``.

* Scalar Taylor basis -- Eq. (basis-functions-1d) / (basis-functions-3d):
  ``p_alpha = prod_k xi_k^alpha_k / alpha_k!`` for all ``|alpha| <= m``; the
  span is pi_m(R^d) (Sec. 2.1) and Q = C(m+d, d).
* Divergence-free vector basis -- Sec. 2.2: a basis of
  pi^div_m(R^d) = {v in (pi_m)^d : div v = 0}.  The oracle spans it with curls
  of monomials: in 2D ``curl(xi^alpha e_z) = (d_y f, -d_x f)`` for
  ``1 <= |alpha| <= m+1`` (all independent); in 3D ``curl(xi^alpha e_c)`` for
  ``1 <= |alpha| <= m+1`` and c = x, y, z, reduced to a basis by exact rational
  rank.  Stencils do not depend on which basis of the span is used, so the CUDA
  path is free to use another one.

A functional row is a list of terms ``(coef, component, beta)`` meaning
``lambda(psi) = sum coef * D^beta psi_component (x_T)`` (Sec. 2.5, Eq.
polynomial-approximation-derivative).
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial

import numpy as np


def graded_exponents(dim: int, m: int) -> list[tuple[int, int, int]]:
    """All exponents alpha with |alpha| <= m, degree ascending (padded to 3)."""
    out = []
    for s in range(m + 1):
        if dim == 1:
            out.append((s, 0, 0))
        elif dim == 2:
            for ay in range(s + 1):
                out.append((s - ay, ay, 0))
        else:
            for az in range(s + 1):
                for ay in range(s - az + 1):
                    out.append((s - ay - az, ay, az))
    return out


def taylor_basis(dim: int, m: int):
    """Scalar scaled Taylor monomials xi^alpha / alpha! (one term each)."""
    terms = []
    for a in graded_exponents(dim, m):
        coef = Fraction(1, factorial(a[0]) * factorial(a[1]) * factorial(a[2]))
        terms.append([[(coef, a)]])  # one component
    assert len(terms) == comb(m + dim, dim)
    return terms


def _curl_of_monomial(alpha, c):
    """curl(xi^alpha e_c) component by component: (grad f x e_c)_i = eps_ijc d_j f."""
    comps = []
    for i in range(3):
        poly = {}
        for j in range(3):
            # Levi-Civita eps_{i j c}
            if len({i, j, c}) < 3:
                continue
            sign = 1 if (i, j, c) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)) else -1
            if alpha[j] == 0:
                continue
            g = list(alpha)
            g[j] -= 1
            g = tuple(g)
            poly[g] = poly.get(g, 0) + sign * alpha[j]
        comps.append({k: v for k, v in poly.items() if v != 0})
    return comps


def _rank(rows):
    """Exact rank of a list of dict-vectors (Fraction Gaussian elimination)."""
    keys = sorted({k for r in rows for k in r})
    mat = [[Fraction(r.get(k, 0)) for k in keys] for r in rows]
    rank = 0
    ncol = len(keys)
    for col in range(ncol):
        piv = None
        for r in range(rank, len(mat)):
            if mat[r][col] != 0:
                piv = r
                break
        if piv is None:
            continue
        mat[rank], mat[piv] = mat[piv], mat[rank]
        for r in range(len(mat)):
            if r != rank and mat[r][col] != 0:
                f = mat[r][col] / mat[rank][col]
                mat[r] = [a - f * b for a, b in zip(mat[r], mat[rank])]
        rank += 1
    return rank


def divfree_dimension(dim: int, m: int) -> int:
    """dim of pi^div_m(R^d): (m+1)(m+4)/2 in 2D, 3 C(m+3,3) - C(m+2,3) in 3D."""
    if dim == 2:
        return (m + 1) * (m + 4) // 2
    if dim == 3:
        return 3 * comb(m + 3, 3) - comb(m + 2, 3)
    raise ValueError("divergence-free basis needs d = 2 or 3")


def divfree_basis(dim: int, m: int):
    """Curls of monomials spanning pi^div_m(R^d); each entry: per component a
    list of (coef, gamma) terms with integer coefficients."""
    if dim == 2:
        funcs = []
        for a in graded_exponents(2, m + 1):
            if sum(a) == 0:
                continue
            comps = _curl_of_monomial(a, 2)  # f(x, y) e_z -> (d_y f, -d_x f, 0)
            funcs.append([[(Fraction(v), k) for k, v in sorted(comps[i].items())] for i in range(2)])
        assert len(funcs) == divfree_dimension(2, m)
        return funcs
    if dim != 3:
        raise ValueError("divergence-free basis needs d = 2 or 3")
    target = divfree_dimension(3, m)
    chosen, chosen_vecs = [], []
    for a in graded_exponents(3, m + 1):
        if sum(a) == 0:
            continue
        for c in range(3):
            comps = _curl_of_monomial(a, c)
            vec = {(i,) + k: v for i in range(3) for k, v in comps[i].items()}
            if not vec:
                continue
            if _rank(chosen_vecs + [vec]) > len(chosen_vecs):
                chosen_vecs.append(vec)
                chosen.append([[(Fraction(v), k) for k, v in sorted(comps[i].items())] for i in range(3)])
            if len(chosen) == target:
                return chosen
    raise AssertionError("curl candidates did not reach the expected dimension")


def basis_table(funcs, nc: int):
    """Flatten a term list into (nb, nc, off int32, coef float64, expo int32[.,3])."""
    off, coef, expo = [0], [], []
    for f in funcs:
        assert len(f) == nc
        for comp in f:
            for c, g in comp:
                coef.append(float(c))
                expo.append(g)
            off.append(len(coef))
    return (
        len(funcs),
        nc,
        np.asarray(off, dtype=np.int32),
        np.asarray(coef if coef else [0.0], dtype=np.float64),
        np.asarray(expo if expo else [(0, 0, 0)], dtype=np.int32).reshape(-1, 3),
    )


def _e(k, times=1):
    b = [0, 0, 0]
    b[k] += times
    return tuple(b)


def functional_terms(name: str, dim: int):
    """Rows of a target functional as (coef, component, beta) lists.

    grad           d rows, d/dx_k of a scalar           (Sec. 2.5)
    laplacian      1 row, sum_k d^2/dx_k^2 of a scalar  (Eq. laplacian-pressure-stencil)
    vec_laplacian  d rows, (Laplacian v)_c              (Sec. 3.1)
    curlcurl       d rows, (curl curl v)_c = d_c div v - (Laplacian v)_c
                   (vector identity of Sec. 3.1, Eq. curl-vector-stencil)
    div            1 row, sum_k d v_k / dx_k
    """
    if name == "grad":
        return [[(1.0, 0, _e(k))] for k in range(dim)]
    if name == "laplacian":
        return [[(1.0, 0, _e(k, 2)) for k in range(dim)]]
    if name == "vec_laplacian":
        return [[(1.0, c, _e(k, 2)) for k in range(dim)] for c in range(dim)]
    if name == "curlcurl":
        rows = []
        for c in range(dim):
            terms = []
            for k in range(dim):
                b = list(_e(c))
                b[k] += 1
                terms.append((1.0, k, tuple(b)))
            terms += [(-1.0, c, _e(k, 2)) for k in range(dim)]
            rows.append(terms)
        return rows
    if name == "div":
        return [[(1.0, k, _e(k)) for k in range(dim)]]
    raise ValueError(f"unknown functional {name!r}")


def functional_table(rows):
    off, coef, comp, beta = [0], [], [], []
    for r in rows:
        for c, k, b in r:
            coef.append(c)
            comp.append(k)
            beta.append(b)
        off.append(len(coef))
    return (
        len(rows),
        np.asarray(off, dtype=np.int32),
        np.asarray(coef, dtype=np.float64),
        np.asarray(comp, dtype=np.int32),
        np.asarray(beta, dtype=np.int32).reshape(-1, 3),
    )
