"""Pins of the oracle's Stokes collocation system (Sec. 3.2, Eq.
stokes-block-system) on the unit square with Dirichlet velocity and the
Neumann pressure condition at the outermost lattice layer.

* Polynomial exactness: for a divergence-free polynomial velocity of degree
  <= m and a polynomial pressure of degree <= m, every stencil reproduces its
  functional exactly, and the Neumann-constrained Laplacian reproduces the
  Laplacian once beta times the exact normal derivative is added.  Hence
  A x - b vanishes (up to rounding) on every row but the zero-mean row, for
  any viscosity.  A sign slip in the coupling of the boundary pressure rows,
  a missing nu or beta, or a mis-placed block fails this.
* Consistency on the manufactured trigonometric field: the residual decays
  like h^(m-1) on interior rows (second-derivative stencils) and h^(m-2) on
  boundary pressure rows (beta ~ 1/eps multiplies an O(h^(m-1)) error).
* Structure: Dirichlet rows are unit rows, every pressure row couples to the
  multiplier, the last row sums the pressures, columns ascend.
* The same three checks, and the solve, with the staggered Laplacian of
  degree m - 1 (Sec. 2.4; exact for pressures of degree <= m) on the interior
  pressure rows, as Sec. 3.2 prescribes for points inside the domain.
"""
import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

import oracle
from paper_2104_14447_gb300 import inputs

M = 4
MS = 3  # staggered interior pressure Laplacian: exact to degree MS + 1 = M, rate MS = M - 1
KV, KP = 48, 36


def _system(na, nu, seed=0, staggered=False):
    x = inputs.jittered_grid(2, na, seed=seed)
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(2, na)
    tg = np.arange(n, dtype=np.int32)
    iv, ev = oracle.knn(x, tg, KV, 1.5, method="grid")
    ip, ep = oracle.knn(x, tg, KP, 1.5, method="grid")
    offv = np.arange(0, n * KV + 1, KV)
    offp = np.arange(0, n * KP + 1, KP)
    wcc, _, _ = oracle.stencils(x, tg, offv, iv.reshape(-1), ev, "divfree", M, "curlcurl")
    wg, _, _ = oracle.stencils(x, tg, offp, ip.reshape(-1), ep, "scalar", M, "grad", bflag=bflag, normals=nrm.T)
    wl, bl, _ = oracle.stencils(x, tg, offp, ip.reshape(-1), ep, "scalar", M, "laplacian", bflag=bflag,
                                normals=nrm.T)
    pint = None
    if staggered:
        ws, _ = oracle.staggered_stencils(x, tg, offp, ip.reshape(-1), ep, MS, "laplacian")
        pint = (offp, ip.reshape(-1), ws)
    A = oracle.stokes_system(2, n, bflag, nrm, (offv, iv.reshape(-1), wcc),
                             (offp, ip.reshape(-1), wg, wl, bl[:, 0]), nu, pres_int=pint)
    return x, n, bflag, nrm, A, bl[:, 0]


def _polynomial_fields(x, nu):
    X, Y = sympy.symbols("x y")
    psi = X ** 3 * Y ** 2 - 2 * X * Y ** 4 + X ** 2 * Y - 3 * X * Y ** 3 + Y ** 5 / 5  # degree 5: v of degree 4
    v = [sympy.diff(psi, Y), -sympy.diff(psi, X)]
    p = X ** 4 - 2 * X ** 2 * Y ** 2 + 3 * X * Y ** 3 - Y + 1
    omega = sympy.diff(v[1], X) - sympy.diff(v[0], Y)
    curlcurl = [sympy.diff(omega, Y), -sympy.diff(omega, X)]
    f = [nu * curlcurl[c] + sympy.diff(p, (X, Y)[c]) for c in range(2)]
    div_f = sympy.diff(f[0], X) + sympy.diff(f[1], Y)
    ev = lambda e: np.asarray(sympy.lambdify((X, Y), e, "numpy")(x[0], x[1]), dtype=np.float64) * np.ones(x.shape[1])
    assert sympy.simplify(sympy.diff(v[0], X) + sympy.diff(v[1], Y)) == 0
    return (np.stack([ev(v[0]), ev(v[1])]), ev(p), np.stack([ev(f[0]), ev(f[1])]), ev(div_f))


def _residual(A, n, bflag, nrm, beta, u, p, f, w, div_f):
    xe = np.concatenate([u.T.reshape(-1), p, [0.0]])
    b = oracle.stokes_rhs(2, n, bflag, nrm, f, w, div_f, beta)
    return A @ xe - b, np.abs(A) @ np.abs(xe) + np.abs(b)


@pytest.mark.parametrize("staggered", [False, True])
@pytest.mark.parametrize("nu", [1.0, 0.37])
def test_polynomial_fields_are_reproduced(nu, staggered):
    x, n, bflag, nrm, A, beta = _system(18, nu, staggered=staggered)
    u, p, f, div_f = _polynomial_fields(x, nu)
    r, scale = _residual(A, n, bflag, nrm, beta, u, p, f, u, div_f)
    rows = slice(0, 3 * n)  # all but the zero-mean row
    assert np.max(np.abs(r[rows]) / scale[rows]) < 1e-10
    assert np.any(bflag) and np.any(beta[bflag == 1] != 0.0)


def test_planted_sign_slip_is_caught():
    """The same check with the boundary pressure rows' velocity coupling
    negated (the sign printed beside Eq. grad-pressure-stencil-1) fails."""
    import scipy.sparse as sp

    x, n, bflag, nrm, A, beta = _system(18, 1.0)
    u, p, f, div_f = _polynomial_fields(x, 1.0)
    C = A.tocoo()
    flip = (C.row >= 2 * n) & (C.row < 3 * n) & (C.col < 2 * n)
    data = C.data.copy()
    data[flip] *= -1.0
    Af = sp.csr_matrix((data, (C.row, C.col)), shape=A.shape)
    r, scale = _residual(Af, n, bflag, nrm, beta, u, p, f, u, div_f)
    assert np.max(np.abs(r[2 * n:3 * n]) / scale[2 * n:3 * n]) > 1e-3


def test_manufactured_field_converges():
    hs, res = [], {"mom": [], "p_int": [], "p_bdry": []}
    for na in (20, 28, 40):
        x, n, bflag, nrm, A, beta = _system(na, 1.0)
        d = inputs.stokes_manufactured_2d(x, 1.0)
        r, _ = _residual(A, n, bflag, nrm, beta, d["u"], d["p"], d["f"], d["w"], d["div_f"])
        bf = bflag.astype(bool)
        mom = np.abs(r[:2 * n]).reshape(n, 2)
        assert np.all(mom[bf] == 0.0)  # Dirichlet rows: exact
        pr = np.abs(r[2 * n:3 * n])
        hs.append(1.0 / na)
        res["mom"].append(mom[~bf].max())
        res["p_int"].append(pr[~bf].max())
        res["p_bdry"].append(pr[bf].max())
    slope = {k: np.polyfit(np.log(hs), np.log(v), 1)[0] for k, v in res.items()}
    assert slope["mom"] > M - 1 - 0.7, slope
    assert slope["p_int"] > M - 1 - 0.7, slope
    assert slope["p_bdry"] > M - 2 - 0.7, slope


def test_structure():
    x, n, bflag, nrm, A, beta = _system(12, 1.0)
    nd = 2 * n
    rp, col = A.indptr, A.indices
    assert A.shape == (nd + n + 1, nd + n + 1)
    for I in range(n):
        for c in range(2):
            r = 2 * I + c
            cols = col[rp[r]:rp[r + 1]]
            if bflag[I]:
                assert list(cols) == [r] and A[r, r] == 1.0
            else:
                assert len(cols) == KV * 2 + KP and np.all(cols[KV * 2:] >= nd) and np.all(cols[:KV * 2] < nd)
        r = nd + I
        cols = col[rp[r]:rp[r + 1]]
        assert cols[-1] == nd + n and A[r, nd + n] == 1.0
        assert len(cols) == (KV * 2 + KP + 1 if bflag[I] else KP + 1)
        assert np.all(np.diff(cols) > 0)
    last = col[rp[nd + n]:rp[nd + n + 1]]
    assert np.array_equal(last, nd + np.arange(n))


def _solve_errors(x, n, A, bflag, nrm, beta, u, p, f, w, div_f):
    b = oracle.stokes_rhs(2, n, bflag, nrm, f, w, div_f, beta)
    sol = oracle.stokes_solve(A, b)
    us = sol[:2 * n].reshape(n, 2).T
    ps = sol[2 * n:3 * n]
    eu = np.sqrt(np.mean((us - u) ** 2))
    # the pressure is fixed up to a constant (the multiplier row sets its
    # discrete mean): compare mean-free parts
    ep = np.sqrt(np.mean(((ps - ps.mean()) - (p - p.mean())) ** 2))
    return eu, ep, sol[-1]


@pytest.mark.parametrize("staggered", [False, True])
@pytest.mark.parametrize("nu", [1.0, 0.37])
def test_polynomial_solution_is_recovered(nu, staggered):
    """The analogue of the paper's polynomial tables (Sec. 4.1): a velocity
    and pressure inside the bases are recovered by the solve up to rounding."""
    x, n, bflag, nrm, A, beta = _system(18, nu, staggered=staggered)
    u, p, f, div_f = _polynomial_fields(x, nu)
    eu, ep, lam = _solve_errors(x, n, A, bflag, nrm, beta, u, p, f, u, div_f)
    assert eu < 1e-9 * np.abs(u).max() and ep < 1e-8 * np.abs(p).max(), (eu, ep)


@pytest.mark.parametrize("staggered", [False, True])
def test_trigonometric_solution_converges(staggered):
    """Manufactured trigonometric field (Sec. 4.2 in 2D): the RMS error of the
    solved velocity and pressure decays at about the order of the basis."""
    hs, eus, eps_ = [], [], []
    for na in (16, 24, 32):
        x, n, bflag, nrm, A, beta = _system(na, 1.0, staggered=staggered)
        d = inputs.stokes_manufactured_2d(x, 1.0)
        eu, ep, _ = _solve_errors(x, n, A, bflag, nrm, beta, d["u"], d["p"], d["f"], d["w"], d["div_f"])
        hs.append(1.0 / na)
        eus.append(eu)
        eps_.append(ep)
    ru = np.polyfit(np.log(hs), np.log(eus), 1)[0]
    rp = np.polyfit(np.log(hs), np.log(eps_), 1)[0]
    assert ru > M - 1 and rp > M - 1, (ru, rp, eus, eps_)


def test_staggered_interior_rows():
    """With the staggered interior Laplacian only the interior pressure rows
    change; their weights sum to zero (the target's own weight is minus the
    sum of the others); dropping that self weight (a planted slip) breaks the
    reproduction of a pressure with a constant part."""
    import scipy.sparse as sp

    x, n, bflag, nrm, A0, beta = _system(18, 1.0)
    _, _, _, _, A1, _ = _system(18, 1.0, staggered=True)
    nd = 2 * n
    bf = bflag.astype(bool)
    D = (A1 - A0).tocsr()
    D.eliminate_zeros()
    changed = np.unique(D.tocoo().row)
    assert np.all(changed >= nd) and np.all(changed < nd + n) and np.all(~bf[changed - nd])
    assert len(changed) == np.count_nonzero(~bf)
    Ai = A1[nd:nd + n, nd:nd + n].tocsr()
    rs = np.asarray(Ai.sum(axis=1)).ravel()
    sc = np.asarray(abs(Ai).sum(axis=1)).ravel()
    assert np.all(np.abs(rs[~bf]) <= 1e-12 * sc[~bf])
    u, p, f, div_f = _polynomial_fields(x, 1.0)
    C = A1.tocoo()
    drop = (C.row >= nd) & (C.row < nd + n) & (C.col == C.row)
    drop &= ~bf[np.clip(C.row - nd, 0, n - 1)]
    Af = sp.csr_matrix((np.where(drop, 0.0, C.data), (C.row, C.col)), shape=A1.shape)
    r, scale = _residual(Af, n, bflag, nrm, beta, u, p, f, u, div_f)
    assert np.max(np.abs(r[nd:nd + n]) / scale[nd:nd + n]) > 1e-3


def test_manufactured_field_converges_staggered():
    hs, res = [], {"mom": [], "p_int": [], "p_bdry": []}
    for na in (20, 28, 40):
        x, n, bflag, nrm, A, beta = _system(na, 1.0, staggered=True)
        d = inputs.stokes_manufactured_2d(x, 1.0)
        r, _ = _residual(A, n, bflag, nrm, beta, d["u"], d["p"], d["f"], d["w"], d["div_f"])
        bf = bflag.astype(bool)
        pr = np.abs(r[2 * n:3 * n])
        hs.append(1.0 / na)
        res["mom"].append(np.abs(r[:2 * n]).reshape(n, 2)[~bf].max())
        res["p_int"].append(pr[~bf].max())
        res["p_bdry"].append(pr[bf].max())
    slope = {k: np.polyfit(np.log(hs), np.log(v), 1)[0] for k, v in res.items()}
    assert slope["p_int"] > MS - 0.7, (slope, res)
    assert slope["mom"] > M - 1 - 0.7 and slope["p_bdry"] > M - 2 - 0.7, (slope, res)


# ------------------------------------------------------------------- 3D
M3, KV3, KP3 = 3, 80, 40  # the porous-medium stencils: div-free 240 x 50, scalar 40 x 20


def _system3(na, nu, staggered=False, cloud=None):
    if cloud is None:
        x = inputs.jittered_grid(3, na, seed=1)
        bflag, nrm = inputs.box_boundary(3, na)
    else:
        x, bflag, nrm = cloud
    n = x.shape[1]
    tg = np.arange(n, dtype=np.int32)
    iv, ev = oracle.knn(x, tg, KV3, 1.5)
    ip, ep = oracle.knn(x, tg, KP3, 1.5)
    offv = np.arange(0, n * KV3 + 1, KV3)
    offp = np.arange(0, n * KP3 + 1, KP3)
    wcc, _, _ = oracle.stencils(x, tg, offv, iv.reshape(-1), ev, "divfree", M3, "curlcurl")
    wg, _, _ = oracle.stencils(x, tg, offp, ip.reshape(-1), ep, "scalar", M3, "grad", bflag=bflag, normals=nrm.T)
    wl, bl, _ = oracle.stencils(x, tg, offp, ip.reshape(-1), ep, "scalar", M3, "laplacian", bflag=bflag,
                                normals=nrm.T)
    pint = None
    if staggered:
        ws, _ = oracle.staggered_stencils(x, tg, offp, ip.reshape(-1), ep, M3 - 1, "laplacian")
        pint = (offp, ip.reshape(-1), ws)
    A = oracle.stokes_system(3, n, bflag, nrm, (offv, iv.reshape(-1), wcc),
                             (offp, ip.reshape(-1), wg, wl, bl[:, 0]), nu, pres_int=pint)
    return x, n, bflag, nrm, A, bl[:, 0]


def _polynomial_fields_3d(x, nu):
    """v = curl a (a of degree 4, so v is divergence-free of degree 3),
    p of degree 3; f = nu curl curl v + grad p, div f = Laplacian p."""
    X, Y, Z = sympy.symbols("x y z")
    V = (X, Y, Z)
    a = [X ** 2 * Y * Z - 2 * Y ** 3 * Z + X * Z ** 3,
         X ** 3 * Z - X * Y ** 2 * Z + 3 * Y * Z ** 3 - X ** 4,
         X * Y ** 3 - 2 * X ** 2 * Z ** 2 + Y ** 2 * Z ** 2 + Z ** 4]

    def curl(u):
        return [sympy.diff(u[2], Y) - sympy.diff(u[1], Z), sympy.diff(u[0], Z) - sympy.diff(u[2], X),
                sympy.diff(u[1], X) - sympy.diff(u[0], Y)]

    v = curl(a)
    cc = curl(curl(v))
    p = X ** 3 - 2 * X * Y * Z + 3 * Y ** 2 * Z - Z ** 3 + X * Y - 1
    f = [nu * cc[c] + sympy.diff(p, V[c]) for c in range(3)]
    div_f = sum(sympy.diff(f[c], V[c]) for c in range(3))
    assert sympy.simplify(sum(sympy.diff(v[c], V[c]) for c in range(3))) == 0
    ev = lambda e: np.asarray(sympy.lambdify(V, e, "numpy")(x[0], x[1], x[2]), dtype=np.float64) * np.ones(x.shape[1])
    return np.stack([ev(e) for e in v]), ev(p), np.stack([ev(e) for e in f]), ev(div_f)


@pytest.mark.parametrize("staggered", [False, True])
def test_polynomial_fields_are_reproduced_3d(staggered):
    """The 3D system (div-free degree 3 on 80 neighbours, scalar degree 3 on
    40, unit-cube boundary with edge and corner normals): every row but the
    zero-mean one holds for a divergence-free cubic velocity and a cubic
    pressure."""
    nu = 0.6
    x, n, bflag, nrm, A, beta = _system3(7, nu, staggered)
    u, p, f, div_f = _polynomial_fields_3d(x, nu)
    xe = np.concatenate([u.T.reshape(-1), p, [0.0]])
    b = oracle.stokes_rhs(3, n, bflag, nrm, f, u, div_f, beta)
    r = A @ xe - b
    scale = np.abs(A) @ np.abs(xe) + np.abs(b)
    rows = slice(0, 4 * n)
    assert np.max(np.abs(r[rows]) / scale[rows]) < 1e-10
    bf = bflag.astype(bool)
    assert 0 < bf.sum() < n and np.all(beta[bf] != 0.0) and np.all(beta[~bf] == 0.0)


def test_planted_normal_mixup_is_caught_3d():
    """The same check with the boundary rows assembled from normals whose y
    and z components are swapped fails on the boundary pressure rows."""
    nu = 0.6
    x, n, bflag, nrm, A, beta = _system3(7, nu)
    u, p, f, div_f = _polynomial_fields_3d(x, nu)
    tg = np.arange(n, dtype=np.int32)
    iv, ev = oracle.knn(x, tg, KV3, 1.5)
    offv = np.arange(0, n * KV3 + 1, KV3)
    wcc, _, _ = oracle.stencils(x, tg, offv, iv.reshape(-1), ev, "divfree", M3, "curlcurl")
    # rebuild with mixed-up normals in the coupling only (the stencils keep the right ones)
    C = A.tocoo()
    keep = ~((C.row >= 3 * n) & (C.row < 4 * n) & (C.col < 3 * n))
    bad = nrm[[0, 2, 1]]
    rows, cols, vals = [C.row[keep]], [C.col[keep]], [C.data[keep]]
    for I in np.flatnonzero(bflag):
        a3 = np.asarray(wcc[I])
        nda = bad[0][I] * a3[0] + bad[1][I] * a3[1] + bad[2][I] * a3[2]
        jv = iv[I].astype(np.int64)
        rows.append(np.full(3 * KV3, 3 * n + I))
        cols.append((jv[:, None] * 3 + np.arange(3)[None, :]).reshape(-1))
        vals.append(-(nu * (beta[I] * nda)).reshape(-1))
    import scipy.sparse as sp

    Af = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=A.shape)
    xe = np.concatenate([u.T.reshape(-1), p, [0.0]])
    b = oracle.stokes_rhs(3, n, bflag, nrm, f, u, div_f, beta)
    r = Af @ xe - b
    scale = np.abs(Af) @ np.abs(xe) + np.abs(b)
    pr = slice(3 * n, 4 * n)
    assert np.max(np.abs(r[pr]) / scale[pr]) > 1e-3


def test_cubic_fields_reproduced_porous():
    """The porous cube (lattice minus 64 spheres; boundary points on the
    sphere surfaces and the cube faces with their geometric normals): the
    cubic Stokes data of inputs.stokes_cubic_3d satisfy every row but the
    zero-mean one, and the data's own derivatives are consistent with the
    Taylor-basis stencils (a check of the generator against the oracle)."""
    pc = inputs.porous_cube(n_axis=12)
    nu = 0.8
    x, n, bflag, nrm, A, beta = _system3(None, nu, cloud=(pc["x"], pc["bflag"], pc["normals"]))
    d = inputs.stokes_cubic_3d(x, nu)
    xe = np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])
    b = oracle.stokes_rhs(3, n, bflag, nrm, d["f"], d["w"], d["div_f"], beta)
    r = A @ xe - b
    scale = np.abs(A) @ np.abs(xe) + np.abs(b)
    rows = slice(0, 4 * n)
    assert np.max(np.abs(r[rows]) / scale[rows]) < 1e-10
    assert np.sum(bflag) > 0.3 * n


@pytest.mark.parametrize("staggered", [False, True])
def test_cubic_solution_is_recovered_3d(staggered):
    """The 3D analogue of the polynomial tables (Sec. 4.1): the direct solve
    of the 3D system with the cubic data recovers the cubic velocity and
    pressure up to rounding."""
    nu = 0.6
    x, n, bflag, nrm, A, beta = _system3(7, nu, staggered)
    d = inputs.stokes_cubic_3d(x, nu)
    b = oracle.stokes_rhs(3, n, bflag, nrm, d["f"], d["w"], d["div_f"], beta)
    sol = oracle.stokes_solve(A, b)
    us = sol[:3 * n].reshape(n, 3).T
    ps = sol[3 * n:4 * n]
    eu = np.abs(us - d["u"]).max()
    ep = np.abs((ps - ps.mean()) - (d["p"] - d["p"].mean())).max()
    assert eu < 1e-9 * np.abs(d["u"]).max() and ep < 1e-8 * np.abs(d["p"]).max(), (eu, ep)
