"""Edge cases of the GPU path through the C ABI: empty and single-target
lists, k equal to the number of points, the largest k, duplicated points
(ties broken by id, bit-exact against the oracle), a degenerate cloud whose
systems are rank deficient (flagged, weights zero), and argument errors
returned before any work is queued."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()
    c = gmls.Context(0, arena_bytes=4 << 30)
    c.set_option(gmls.OPT_POISON, 1)  # outputs start as NaN: unwritten entries cannot pass
    yield c
    c.close()


def test_empty_target_list(ctx):
    x = inputs.jittered_grid(2, 16, seed=0)
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, 12, 1.5, targets=np.zeros(0, dtype=np.int32))
    sid = ctx.stencils(nid, gmls.SCALAR, 2, [gmls.LAPLACIAN], precision=gmls.FP32_REFINE)
    nt, rows, nc, nvals = ctx.stencil_info(sid, gmls.LAPLACIAN)
    assert nt == 0 and nvals == 0
    rp, col, val = ctx.assemble_csr(sid, gmls.LAPLACIAN)
    assert rp.cpu().numpy().tolist() == [0]
    ctx.sync()
    for h in (sid, nid, cid):
        ctx.release(h)


def test_single_target_and_k_equal_n(ctx):
    x = inputs.jittered_grid(2, 7, seed=2)  # 49 points
    n = x.shape[1]
    cid = ctx.cloud(x)
    tg = np.array([24], dtype=np.int32)
    nid = ctx.neighbors(cid, n, 1.5, targets=tg)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    oi, oe = oracle.knn(x, tg, n, 1.5)
    assert np.array_equal(idx, oi.reshape(-1)) and np.array_equal(eps, oe)
    sid = ctx.stencils(nid, gmls.SCALAR, 4, [gmls.GRAD], precision=gmls.FP64)
    wo, _, _ = oracle.stencils(x, tg, np.array([0, n]), oi.reshape(-1), oe, "scalar", 4, "grad")
    wg = ctx.weights(sid, gmls.GRAD).cpu().numpy().reshape(wo.shape)
    assert np.max(np.abs(wg - wo)) <= 1e-10 * np.abs(wo).max()
    for h in (sid, nid, cid):
        ctx.release(h)


def test_largest_k(ctx):
    x = inputs.jittered_grid(3, 14, seed=4)  # 2,744 points
    cid = ctx.cloud(x)
    tg = np.arange(0, x.shape[1], 97, dtype=np.int32)
    nid = ctx.neighbors(cid, 1024, 1.5, targets=tg)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    oi, oe = oracle.knn(x, tg, 1024, 1.5)
    assert np.array_equal(idx, oi.reshape(-1)) and np.array_equal(eps, oe)
    with pytest.raises(gmls.GmlsError) as e:
        ctx.neighbors(cid, 1025, 1.5, targets=tg)
    assert e.value.code == gmls.EINVAL
    for h in (nid, cid):
        ctx.release(h)


def test_duplicated_points_tie_by_id(ctx):
    base = inputs.jittered_grid(2, 10, seed=6)
    x = np.concatenate([base, base[:, ::3], base[:, ::5]], axis=1)  # exact duplicates
    n = x.shape[1]
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, 16, 1.5)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    oi, oe = oracle.knn(x, np.arange(n, dtype=np.int32), 16, 1.5)
    assert np.array_equal(idx, oi.reshape(-1)) and np.array_equal(eps, oe)
    for h in (nid, cid):
        ctx.release(h)


@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
def test_collinear_cloud_is_rank_deficient(ctx, precision):
    t = np.linspace(0.0, 1.0, 60)
    x = np.stack([t, 0.5 * t + 0.1])  # every point on one line: no quadratic fit in 2D
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, 12, 1.5)
    sid = ctx.stencils(nid, gmls.SCALAR, 2, [gmls.LAPLACIAN], precision=precision)
    st = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    w = ctx.weights(sid, gmls.LAPLACIAN).cpu().numpy()
    assert np.all((st & gmls.T_RANK_DEFICIENT) != 0)
    assert np.all(w == 0.0)
    for h in (sid, nid, cid):
        ctx.release(h)


def test_argument_errors(ctx):
    x = inputs.jittered_grid(2, 8, seed=0)
    with pytest.raises(gmls.GmlsError) as e:
        ctx.cloud(np.zeros((4, 10)))  # dim 4
    assert e.value.code == gmls.EINVAL
    cid = ctx.cloud(x)
    with pytest.raises(gmls.GmlsError):
        ctx.neighbors(cid, 65, 1.5)  # k > n
    nid = ctx.neighbors(cid, 12, 1.5)
    with pytest.raises(gmls.GmlsError):
        ctx.stencils(nid, gmls.SCALAR, 5, [gmls.GRAD])  # degree 5
    with pytest.raises(gmls.GmlsError):
        ctx.stencils(nid, gmls.SCALAR, 2, [gmls.VEC_LAPLACIAN])  # vector functional on a scalar basis
    with pytest.raises(gmls.GmlsError):
        ctx.stencils(nid, gmls.STAGGERED, 2, [gmls.GRAD], neumann=True)  # no Neumann on the staggered basis
    with pytest.raises(gmls.GmlsError) as e:
        ctx.release(cid)  # still referenced by the neighbour handle
    assert e.value.code == gmls.EBUSY
    ctx.release(nid)
    ctx.release(cid)
    with pytest.raises(gmls.GmlsError) as e:
        ctx.release(cid)
    assert e.value.code == gmls.ENOTFOUND


def test_factored_divfree_kernel_on_a_small_arena(ctx):
    """The factored divergence-free kernel takes per-warp scratch from the
    arena (53 MB for a full grid of the 3D degree-3 basis); on an arena that
    cannot hold it the launch runs a smaller grid, with the same weights
    bit for bit."""
    x = inputs.jittered_grid(3, 12, seed=4)
    small = gmls.Context(0, arena_bytes=48 << 20)
    small.set_option(gmls.OPT_FORCE_VARIANT, -3)
    ctx.set_option(gmls.OPT_FORCE_VARIANT, -3)
    try:
        out = []
        for c in (ctx, small):
            cid = c.cloud(x)
            nid = c.neighbors(cid, 80, 1.5)
            sid = c.stencils(nid, gmls.DIVFREE, 3, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE)
            out.append(c.weights(sid, gmls.VEC_LAPLACIAN).cpu().numpy())
            c.sync()
            for h in (sid, nid, cid):
                c.release(h)
        assert np.all(np.isfinite(out[0])) and np.array_equal(out[0], out[1])
    finally:
        ctx.set_option(gmls.OPT_FORCE_VARIANT, 0)
        small.close()
