"""GPU Stokes collocation system (Sec. 3.2, Eq. stokes-block-system) through
the C ABI, against the oracle's system built from the oracle's own neighbour
lists and stencils.

* structure (row_ptr, col) bit for bit;
* values per (row, block) within 1e-10 (FP64 stencils) / 1e-9 (FP32 +
  refinement) of the block's largest entry;
* the right-hand side and A x (gmls_csr_spmv) within the same tolerance of
  the oracle's, relative to sum |a| |x| + |b|;
* at GPU scale, the manufactured-field residual decays at the rates the
  oracle pins (h^(m-1) interior, h^(m-2) boundary pressure rows) and the
  Dirichlet rows are exact;
* each with the interior pressure rows taken either from the scalar
  Laplacian or from the staggered one of degree m - 1 (Sec. 3.2).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu

M, KV, KP = 4, 48, 36
MS = 3  # staggered interior Laplacian degree
TOL = {gmls.FP64: 1e-10, gmls.FP32_REFINE: 1e-9}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()
    c = gmls.Context(0, arena_bytes=16 << 30)
    c.set_option(gmls.OPT_POISON, 1)  # outputs start as NaN: unwritten entries cannot pass
    yield c
    c.close()


def _gpu(ctx, na, precision, nu, staggered=False):
    x = inputs.jittered_grid(2, na, seed=0)
    bflag, nrm = inputs.box_boundary(2, na)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, KV, 1.5)
    npr = ctx.neighbors_prefix(nv, KP, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, M, [gmls.CURLCURL], precision=precision)
    sp = ctx.stencils(npr, gmls.SCALAR, M, [gmls.GRAD, gmls.LAPLACIAN], precision=precision, neumann=True)
    ids = (cid, nv, npr, sv, sp)
    ss = 0
    if staggered:
        ss = ctx.stencils(npr, gmls.STAGGERED, MS, [gmls.LAPLACIAN], precision=precision)
        ids += (ss,)
    rp, col, val = ctx.stokes_assemble(sv, sp, nu, ss)
    return x, bflag, nrm, ids, (rp, col, val)


def _release(ctx, ids):
    for h in reversed(ids):
        ctx.release(h)


def _oracle(x, bflag, nrm, nu, staggered=False):
    n = x.shape[1]
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
    return A, bl[:, 0]


@pytest.mark.parametrize("staggered", [False, True])
@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
def test_system_matches_oracle(ctx, precision, staggered):
    nu = 0.7
    x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, 30, precision, nu, staggered)
    n = x.shape[1]
    nd = 2 * n
    A, beta = _oracle(x, bflag, nrm, nu, staggered)
    rp, col, val = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    assert np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
    tol = TOL[precision]
    block = np.where(A.indices < nd, 0, np.where(A.indices < nd + n, 1, 2))
    row = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    key = row * 3 + block
    scale = np.zeros(A.shape[0] * 3)
    np.maximum.at(scale, key, np.abs(A.data))
    err = np.abs(val - A.data) / np.where(scale[key] > 0, scale[key], 1.0)
    assert err.max() <= tol, err.max()
    # right-hand side and A x
    d = inputs.stokes_manufactured_2d(x, nu)
    xe = np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])
    b_orc = oracle.stokes_rhs(2, n, bflag, nrm, d["f"], d["w"], d["div_f"], beta)
    b_gpu = ctx.stokes_rhs(ids[3], ids[4], nu, d["f"], d["w"], d["div_f"]).cpu().numpy()
    nf = np.abs(nrm[0] * d["f"][0] + nrm[1] * d["f"][1])
    bscale = np.abs(b_orc)
    bscale[nd:nd + n] += np.abs(beta) * nf
    assert np.all(np.abs(b_gpu - b_orc) <= tol * np.maximum(bscale, 1e-300))
    y_gpu = ctx.spmv(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda(),
                     xe).cpu().numpy()
    y_orc = A @ xe
    yscale = np.abs(A) @ np.abs(xe)
    assert np.all(np.abs(y_gpu - y_orc) <= tol * yscale + 1e-300)
    _release(ctx, ids)


def test_manufactured_residual_converges_at_scale(ctx):
    """The GPU system alone at 64^2 .. 512^2 (the benchmark grid)."""
    hs, res = [], {"mom": [], "p_int": [], "p_bdry": []}
    for na in (64, 128, 256, 512):
        x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, na, gmls.FP32_REFINE, 1.0)
        n = x.shape[1]
        d = inputs.stokes_manufactured_2d(x, 1.0)
        xe = np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])
        b = ctx.stokes_rhs(ids[3], ids[4], 1.0, d["f"], d["w"], d["div_f"])
        r = (ctx.spmv(rp, col, val, xe) - b).cpu().numpy()
        bf = bflag.astype(bool)
        mom = np.abs(r[:2 * n]).reshape(n, 2)
        assert np.all(mom[bf] == 0.0)
        pr = np.abs(r[2 * n:3 * n])
        hs.append(1.0 / na)
        res["mom"].append(mom[~bf].max())
        res["p_int"].append(pr[~bf].max())
        res["p_bdry"].append(pr[bf].max())
        _release(ctx, ids)
    slope = {k: np.polyfit(np.log(hs), np.log(v), 1)[0] for k, v in res.items()}
    assert slope["mom"] > M - 1 - 0.7, (slope, res)
    assert slope["p_int"] > M - 1 - 0.7, (slope, res)
    assert slope["p_bdry"] > M - 2 - 0.7, (slope, res)


def test_bad_handles_are_rejected(ctx):
    x = inputs.jittered_grid(2, 12, seed=0)
    bflag, nrm = inputs.box_boundary(2, 12)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, KV, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, M, [gmls.CURLCURL])
    sp_plain = ctx.stencils(nv, gmls.SCALAR, M, [gmls.GRAD, gmls.LAPLACIAN])  # no Neumann constraint
    with pytest.raises(gmls.GmlsError) as e:
        ctx.stokes_size(sv, sp_plain, 1.0)
    assert e.value.code == gmls.EINVAL
    with pytest.raises(gmls.GmlsError):
        ctx.stokes_size(sp_plain, sv, 1.0)  # roles swapped
    sp = ctx.stencils(nv, gmls.SCALAR, M, [gmls.GRAD, gmls.LAPLACIAN], neumann=True)
    with pytest.raises(gmls.GmlsError) as e:
        ctx.stokes_size(sv, sp, 1.0, sp_plain)  # interior rows from a non-staggered handle
    assert e.value.code == gmls.EINVAL
    with pytest.raises(gmls.GmlsError) as e:
        ctx.stokes_size(sv, sp, 1.0, 10 ** 9)  # no such handle
    assert e.value.code == gmls.ENOTFOUND
    sg = ctx.stencils(nv, gmls.STAGGERED, MS, [gmls.GRAD])  # no Laplacian
    with pytest.raises(gmls.GmlsError) as e:
        ctx.stokes_size(sv, sp, 1.0, sg)
    assert e.value.code == gmls.EINVAL
    _release(ctx, [cid, nv, sv, sp_plain, sp, sg])


@pytest.mark.parametrize("n_extra_long", [20, 70])
def test_spmv_long_rows(ctx, n_extra_long):
    """gmls_csr_spmv on rows of very different lengths (1 .. 300,000 entries;
    rows above 8192 entries are split over blocks when there are at most 64
    of them, else summed by one block each): the correctly rounded row sums
    within rounding, and the same bits on a second call."""
    rng = np.random.default_rng(3)
    lens = np.concatenate([rng.integers(0, 200, 5000), [9000, 300000, 8193, 20000], rng.integers(1, 50, 3000)])
    for i in range(n_extra_long):
        lens = np.append(lens, 10000 + 37 * i)
    rp = np.zeros(len(lens) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    ncol = 50000
    col = rng.integers(0, ncol, int(rp[-1])).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    x = rng.standard_normal(ncol)
    t = [torch.from_numpy(a).cuda() for a in (rp, col, val)]
    y1 = ctx.spmv(*t, x).cpu().numpy()
    y2 = ctx.spmv(*t, x).cpu().numpy()
    assert np.array_equal(y1, y2)
    prod = val * x[col]
    ref = np.array([math.fsum(prod[a:b]) for a, b in zip(rp[:-1], rp[1:])])  # correctly rounded sums
    scale = np.array([np.abs(prod[a:b]).sum() for a, b in zip(rp[:-1], rp[1:])])
    assert np.all(np.abs(y1 - ref) <= 1e-12 * scale + 1e-300)


def _solve_errors(x, n, sol, u, p):
    us = sol[:2 * n].reshape(n, 2).T
    ps = sol[2 * n:3 * n]
    eu = np.sqrt(np.mean((us - u) ** 2))
    ep = np.sqrt(np.mean(((ps - ps.mean()) - (p - p.mean())) ** 2))
    return eu, ep


@pytest.mark.parametrize("staggered", [False, True])
def test_gmres_solution_matches_direct_solve(ctx, staggered):
    """The GPU solve (gmls_gmres on the GPU system) against the oracle's
    direct solve of the oracle's system, 32 x 32, FP64 stencils."""
    nu = 1.0
    x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, 32, gmls.FP64, nu, staggered)
    n = x.shape[1]
    A, beta = _oracle(x, bflag, nrm, nu, staggered)
    d = inputs.stokes_manufactured_2d(x, nu)
    b_orc = oracle.stokes_rhs(2, n, bflag, nrm, d["f"], d["w"], d["div_f"], beta)
    sol_orc = oracle.stokes_solve(A, b_orc)
    b = ctx.stokes_rhs(ids[3], ids[4], nu, d["f"], d["w"], d["div_f"])
    sol, its, rel = ctx.gmres(rp, col, val, b, restart=60, max_iter=4000, rtol=1e-12)
    sol = sol.cpu().numpy()
    assert rel <= 1e-12 and its > 0
    # the two systems agree to 1e-10 (stencils); the solution to the
    # system's conditioning times that
    assert np.max(np.abs(sol - sol_orc)) <= 1e-6 * np.abs(sol_orc).max()
    eu, ep = _solve_errors(x, n, sol, d["u"], d["p"])
    eu_o, ep_o = _solve_errors(x, n, sol_orc, d["u"], d["p"])
    assert abs(eu - eu_o) <= 1e-3 * eu_o and abs(ep - ep_o) <= 1e-3 * ep_o
    # reproducible bits
    sol2, its2, _ = ctx.gmres(rp, col, val, b, restart=60, max_iter=4000, rtol=1e-12)
    assert its2 == its and np.array_equal(sol2.cpu().numpy(), sol)
    _release(ctx, ids)


@pytest.mark.parametrize("staggered", [False, True])
def test_gmres_solution_converges_at_scale(ctx, staggered):
    """Solved trigonometric field at 32^2 .. 128^2 (FP32 + refinement
    stencils): RMS errors decay at about the order of the basis."""
    hs, eus, eps_ = [], [], []
    for na in (32, 64, 128):
        x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, na, gmls.FP32_REFINE, 1.0, staggered)
        n = x.shape[1]
        d = inputs.stokes_manufactured_2d(x, 1.0)
        b = ctx.stokes_rhs(ids[3], ids[4], 1.0, d["f"], d["w"], d["div_f"])
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=20000, rtol=1e-11)
        assert rel <= 1e-11, (na, its, rel)
        eu, ep = _solve_errors(x, n, sol.cpu().numpy(), d["u"], d["p"])
        hs.append(1.0 / na)
        eus.append(eu)
        eps_.append(ep)
        _release(ctx, ids)
    ru = np.polyfit(np.log(hs), np.log(eus), 1)[0]
    rp_ = np.polyfit(np.log(hs), np.log(eps_), 1)[0]
    assert ru > M - 1 and rp_ > M - 1, (ru, rp_, eus, eps_)


M3, KV3, KP3 = 3, 80, 40


@pytest.mark.parametrize("staggered", [False, True])
@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
def test_system_matches_oracle_3d(ctx, precision, staggered):
    """The 3D system (div-free degree 3 on 80 neighbours: 240 x 50; scalar
    degree 3 on the 40-prefix with the Neumann constraint on the cube's
    faces, edges and corners; optionally the staggered degree-2 Laplacian on
    the interior pressure rows) against the oracle's, and its A x."""
    nu = 0.6
    na = 9
    x = inputs.jittered_grid(3, na, seed=1)
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(3, na)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, KV3, 1.5)
    npr = ctx.neighbors_prefix(nv, KP3, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, M3, [gmls.CURLCURL], precision=precision)
    sp = ctx.stencils(npr, gmls.SCALAR, M3, [gmls.GRAD, gmls.LAPLACIAN], precision=precision, neumann=True)
    ids = [cid, nv, npr, sv, sp]
    ss = 0
    if staggered:
        ss = ctx.stencils(npr, gmls.STAGGERED, M3 - 1, [gmls.LAPLACIAN], precision=precision)
        ids.append(ss)
    rp, col, val = (t.cpu().numpy() for t in ctx.stokes_assemble(sv, sp, nu, ss))
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
    assert np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
    nd = 3 * n
    block = np.where(A.indices < nd, 0, np.where(A.indices < nd + n, 1, 2))
    row = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    key = row * 3 + block
    scale = np.zeros(A.shape[0] * 3)
    np.maximum.at(scale, key, np.abs(A.data))
    err = np.abs(val - A.data) / np.where(scale[key] > 0, scale[key], 1.0)
    tol = TOL[precision]
    assert err.max() <= tol, err.max()
    rng = np.random.default_rng(5)
    xr = rng.standard_normal(A.shape[0])
    y_gpu = ctx.spmv(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda(),
                     xr).cpu().numpy()
    assert np.all(np.abs(y_gpu - A @ xr) <= tol * (np.abs(A) @ np.abs(xr)) + 1e-300)
    _release(ctx, ids)


@pytest.mark.parametrize("staggered", [False, True])
def test_porous_cube_cubic_data_residual(ctx, staggered):
    """The 3D system on the porous cube (32^3 lattice minus 64 spheres;
    boundary rows on sphere surfaces and cube faces, geometric normals), FP32
    + refinement stencils: the cubic Stokes data (inside the degree-3 bases)
    satisfy every row but the zero-mean one to the stencils' rounding, a
    property that holds at any size (the benchmark checks it at 128^3)."""
    pc = inputs.porous_cube(n_axis=32)
    x = pc["x"]
    n = x.shape[1]
    cid = ctx.cloud(x, normals=pc["normals"], bflags=pc["bflag"])
    nv = ctx.neighbors(cid, KV3, 1.5)
    npr = ctx.neighbors_prefix(nv, KP3, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, M3, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    sp = ctx.stencils(npr, gmls.SCALAR, M3, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE, neumann=True)
    ids = [cid, nv, npr, sv, sp]
    ss = 0
    if staggered:
        ss = ctx.stencils(npr, gmls.STAGGERED, M3 - 1, [gmls.LAPLACIAN], precision=gmls.FP32_REFINE)
        ids.append(ss)
    rp, col, val = ctx.stokes_assemble(sv, sp, 1.0, ss)
    d = inputs.stokes_cubic_3d(x, 1.0)
    xe = np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])
    b = ctx.stokes_rhs(sv, sp, 1.0, d["f"], d["w"], d["div_f"])
    r = (ctx.spmv(rp, col, val, xe) - b).abs().cpu().numpy()
    scale = (ctx.spmv(rp, col, val.abs(), np.abs(xe)) + b.abs()).cpu().numpy()
    rel = r[:4 * n] / scale[:4 * n]
    bf = pc["bflag"].astype(bool)
    assert np.all(rel[:3 * n].reshape(n, 3)[bf] == 0.0)  # Dirichlet rows
    assert rel.max() <= 1e-8, (rel[:3 * n].max(), rel[3 * n:].max())
    _release(ctx, ids)


@pytest.mark.parametrize("staggered", [False, True])
def test_gmres_recovers_cubic_solution_3d(ctx, staggered):
    """The GPU solve of the 3D system (9^3 cube, FP32 + refinement stencils)
    with the cubic Stokes data: the velocity and the mean-free pressure are
    recovered up to the stencils' rounding (the 3D analogue of the paper's
    polynomial tables, Sec. 4.1)."""
    nu = 0.6
    na = 9
    x = inputs.jittered_grid(3, na, seed=1)
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(3, na)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, KV3, 1.5)
    npr = ctx.neighbors_prefix(nv, KP3, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, M3, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    sp = ctx.stencils(npr, gmls.SCALAR, M3, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE, neumann=True)
    ids = [cid, nv, npr, sv, sp]
    ss = 0
    if staggered:
        ss = ctx.stencils(npr, gmls.STAGGERED, M3 - 1, [gmls.LAPLACIAN], precision=gmls.FP32_REFINE)
        ids.append(ss)
    rp, col, val = ctx.stokes_assemble(sv, sp, nu, ss)
    d = inputs.stokes_cubic_3d(x, nu)
    b = ctx.stokes_rhs(sv, sp, nu, d["f"], d["w"], d["div_f"])
    sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=4000, rtol=1e-12)
    assert rel <= 1e-12 and its > 0, (its, rel)
    s = sol.cpu().numpy()
    us, ps = s[:3 * n].reshape(n, 3).T, s[3 * n:4 * n]
    eu = np.abs(us - d["u"]).max()
    ep = np.abs((ps - ps.mean()) - (d["p"] - d["p"].mean())).max()
    assert eu < 1e-6 * np.abs(d["u"]).max() and ep < 1e-5 * np.abs(d["p"]).max(), (eu, ep)
    _release(ctx, ids)


@pytest.mark.parametrize("degree,kv,kp", [(2, 42, 20), (4, 136, 84)])
def test_gmres_recovers_polynomial_solution_3d(ctx, degree, kv, kp):
    """Sec. 4.1's polynomial tests through the GPU operators on [-1, 1]^3
    (6^3 lattice): a quadratic / quartic divergence-free velocity and
    pressure, reproduced exactly by the degree-2 / degree-4 bases, recovered
    by the row-equilibrated GMRES solve up to the stencils' rounding."""
    na = 6
    x = inputs.jittered_grid(3, na, seed=2) * 2.0 - 1.0
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(3, na)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, kv, 1.5)
    npr = ctx.neighbors_prefix(nv, kp, 1.5)
    sv = ctx.stencils(nv, gmls.DIVFREE, degree, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    sp = ctx.stencils(npr, gmls.SCALAR, degree, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE, neumann=True)
    rp, col, val = ctx.stokes_assemble(sv, sp, 1.0, 0)
    d = inputs.stokes_polynomial_3d(x, degree, 1.0)
    b = ctx.stokes_rhs(sv, sp, 1.0, d["f"], d["w"], d["div_f"])
    sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=4000, rtol=1e-12, row_scaling=True)
    assert rel <= 1e-12 and its > 0, (its, rel)
    s = sol.cpu().numpy()
    us, ps = s[:3 * n].reshape(n, 3).T, s[3 * n:4 * n]
    eu = np.abs(us - d["u"]).max()
    ep = np.abs((ps - ps.mean()) - (d["p"] - d["p"].mean())).max()
    assert eu < 1e-6 * np.abs(d["u"]).max() and ep < 1e-5 * np.abs(d["p"]).max(), (eu, ep)
    _release(ctx, [cid, nv, npr, sv, sp])


def test_trig_solution_converges_3d(ctx):
    """The paper's trigonometric 3D Stokes field (Sec. 4.1) with degree-2
    stencils: the solved velocity's L2 error falls at least at order 2 from
    N = 12 to N = 24 points per axis on [-1, 1]^3 (measured: about 2.5)."""
    errs = []
    for na in (12, 24):
        x = inputs.jittered_grid(3, na, seed=na) * 2.0 - 1.0
        n = x.shape[1]
        bflag, nrm = inputs.box_boundary(3, na)
        cid = ctx.cloud(x, normals=nrm, bflags=bflag)
        nv = ctx.neighbors(cid, 42, 1.5)
        npr = ctx.neighbors_prefix(nv, 20, 1.5)
        sv = ctx.stencils(nv, gmls.DIVFREE, 2, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
        sp = ctx.stencils(npr, gmls.SCALAR, 2, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE, neumann=True)
        rp, col, val = ctx.stokes_assemble(sv, sp, 1.0, 0)
        d = inputs.stokes_trig_3d(x, 1.0)
        b = ctx.stokes_rhs(sv, sp, 1.0, d["f"], d["w"], d["div_f"])
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=4000, rtol=1e-12, row_scaling=True)
        assert rel <= 1e-12, (its, rel)
        us = sol.cpu().numpy()[:3 * n].reshape(n, 3).T
        errs.append(np.sqrt(np.mean((us - d["u"]) ** 2)))
        _release(ctx, [cid, nv, npr, sv, sp])
    order = np.log(errs[0] / errs[1]) / np.log(23.0 / 11.0)
    assert order >= 2.0, (errs, order)


def test_gmres_row_scaling_matches_direct_solve(ctx):
    """GMRES on the row-equilibrated system (row_scaling = 1), 32 x 32, FP64
    stencils, against the oracle's direct solve of the oracle's system; the
    same bits on a second solve."""
    nu = 1.0
    x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, 32, gmls.FP64, nu)
    n = x.shape[1]
    A, beta = _oracle(x, bflag, nrm, nu)
    d = inputs.stokes_manufactured_2d(x, nu)
    b_orc = oracle.stokes_rhs(2, n, bflag, nrm, d["f"], d["w"], d["div_f"], beta)
    sol_orc = oracle.stokes_solve(A, b_orc)
    b = ctx.stokes_rhs(ids[3], ids[4], nu, d["f"], d["w"], d["div_f"])
    sol, its, rel = ctx.gmres(rp, col, val, b, restart=60, max_iter=4000, rtol=1e-12, row_scaling=True)
    assert rel <= 1e-12 and its > 0
    s = sol.cpu().numpy()
    assert np.max(np.abs(s - sol_orc)) <= 1e-6 * np.abs(sol_orc).max()
    sol2, its2, _ = ctx.gmres(rp, col, val, b, restart=60, max_iter=4000, rtol=1e-12, row_scaling=True)
    assert its2 == its and np.array_equal(sol2.cpu().numpy(), s)
    _release(ctx, ids)


def test_gmres_row_scaling_solves_256(ctx):
    """At 256 x 256 (196,609 unknowns) GMRES(100) with the Jacobi scaling
    alone stalls (relative residual about 0.96); on the row-equilibrated
    system it converges, and the solved field is more accurate than at
    128 x 128 by about the order of the basis."""
    errs = []
    for na in (128, 256):
        x, bflag, nrm, ids, (rp, col, val) = _gpu(ctx, na, gmls.FP32_REFINE, 1.0)
        n = x.shape[1]
        d = inputs.stokes_manufactured_2d(x, 1.0)
        b = ctx.stokes_rhs(ids[3], ids[4], 1.0, d["f"], d["w"], d["div_f"])
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=20000, rtol=1e-10, row_scaling=True)
        assert rel <= 1e-10, (na, its, rel)
        errs.append(_solve_errors(x, n, sol.cpu().numpy(), d["u"], d["p"]))
        _release(ctx, ids)
    (eu1, ep1), (eu2, ep2) = errs
    assert eu2 < eu1 / 4 and ep2 < ep1 / 4, errs
