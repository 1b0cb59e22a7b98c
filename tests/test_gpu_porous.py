"""GPU parity on the 3D porous-medium workload: a jittered lattice in the unit
cube minus random non-overlapping spheres, degree-3 scalar basis (20 terms,
40 neighbours) with a Neumann pressure constraint at boundary targets, and
the degree-3 divergence-free vector basis (50 terms, 80 neighbours, 240 x 50
systems).  Boundary targets (sphere surfaces and cube faces) carry their
geometric outward normals.  Neighbour lists must match the oracle bit for
bit; weights and Neumann coefficients within 1e-10 (FP64) / 1e-9 (FP32 +
refinement) relative, per (target, functional row)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu

TOL = {gmls.FP64: 1e-10, gmls.FP32_REFINE: 1e-9}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()
    c = gmls.Context(0, arena_bytes=24 << 30)
    c.set_option(gmls.OPT_POISON, 1)  # outputs start as NaN: unwritten entries cannot pass
    yield c
    c.close()


def _rel_err_rows(wg, wo):
    T, R = wo.shape[:2]
    a = np.abs(wg - wo).reshape(T, R, -1).max(axis=2)
    b = np.abs(wo).reshape(T, R, -1).max(axis=2)
    return float(np.max(a / np.where(b > 0, b, 1.0)))


def _check_targets(ctx, pc, cid, sample, precision, tol):
    """kNN lists and both stencil families on the targets ``sample``."""
    x, bf, nr = pc["x"], pc["bflag"], pc["normals"]
    ns = len(sample)
    tg = torch.from_numpy(sample.astype(np.int32))
    for basis, m, k, fns in ((gmls.SCALAR, 3, 40, ("grad", "laplacian")), (gmls.DIVFREE, 3, 80, ("vec_laplacian",))):
        nid = ctx.neighbors(cid, k, 1.5, targets=tg)
        idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
        eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
        oi, oe = oracle.knn(x, sample, k, 1.5, method="grid")
        assert np.array_equal(idx.reshape(ns, k), oi) and np.array_equal(eps, oe)
        codes = [getattr(gmls, f.upper()) for f in fns]
        neumann = basis == gmls.SCALAR
        sid = ctx.stencils(nid, basis, m, codes, precision=precision, neumann=neumann)
        status = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
        assert np.all((status & (gmls.T_RANK_DEFICIENT | gmls.T_TOO_FEW_NEIGHBOURS)) == 0)
        off = np.arange(0, ns * k + 1, k)
        kind = "scalar" if neumann else "divfree"
        if neumann:
            beta = ctx.export(sid, gmls.X_BETA, torch.float64).cpu().numpy().reshape(ns, -1)
        r0 = 0
        for fn, code in zip(fns, codes):
            extra = dict(bflag=bf[sample], normals=nr.T[sample]) if neumann else {}
            wo, bo, _ = oracle.stencils(x, sample, off, oi.reshape(-1), oe, kind, m, fn, **extra)
            wg = ctx.weights(sid, code).cpu().numpy().reshape(wo.shape)
            assert _rel_err_rows(wg, wo) <= tol, (fn, _rel_err_rows(wg, wo))
            if neumann:
                rows = wo.shape[1]
                bg = beta[:, r0:r0 + rows]
                scale = np.abs(bo) + np.abs(wo).reshape(ns, rows, -1).max(axis=2) * eps[:, None]
                assert np.all(np.abs(bg - bo) <= tol * scale)
                assert np.all(bg[bf[sample] == 0] == 0.0)
                assert np.any(bg[bf[sample] == 1] != 0.0)
                r0 += rows
        ctx.release(sid)
        ctx.release(nid)


@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
def test_porous_cube_small(ctx, precision):
    """Every target of a 20^3-lattice porous cube (about 6,700 points, half of
    them on a boundary)."""
    pc = inputs.porous_cube(n_axis=20)
    n = pc["x"].shape[1]
    assert 0.3 < pc["bflag"].mean() < 0.7
    cid = ctx.cloud(pc["x"], normals=pc["normals"], bflags=pc["bflag"])
    _check_targets(ctx, pc, cid, np.arange(n, dtype=np.int32), precision, TOL[precision])
    ctx.release(cid)


def test_porous_cube_full_size_sampled(ctx):
    """The full-size cloud (128^3 lattice, 2,097,152 points before the
    spheres are cut out): neighbour search over all points, stencils on a
    sample of interior and boundary targets that the oracle computes one by
    one."""
    pc = inputs.porous_cube(n_axis=128)
    n = pc["x"].shape[1]
    assert n > 1_500_000
    cid = ctx.cloud(pc["x"], normals=pc["normals"], bflags=pc["bflag"])
    # all-target neighbour lists at full size, sampled against the oracle
    nid = ctx.neighbors(cid, 80, 1.5)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy().reshape(n, 80)
    probe = np.unique((inputs.uniform(1, 98, 400) * n).astype(np.int32))
    oi, _ = oracle.knn(pc["x"], probe, 80, 1.5, method="grid")
    assert np.array_equal(idx[probe], oi)
    ctx.release(nid)
    bidx = np.flatnonzero(pc["bflag"])
    iidx = np.flatnonzero(pc["bflag"] == 0)
    pick_b = bidx[(inputs.uniform(1, 96, 150) * len(bidx)).astype(np.int64)]
    pick_i = iidx[(inputs.uniform(1, 97, 150) * len(iidx)).astype(np.int64)]
    sample = np.unique(np.concatenate([pick_b, pick_i])).astype(np.int32)
    _check_targets(ctx, pc, cid, sample, gmls.FP32_REFINE, TOL[gmls.FP32_REFINE])
    ctx.release(cid)
