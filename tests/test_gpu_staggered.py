"""GPU staggered GMLS stencils (Sec. 2.4, GMLS_BASIS_STAGGERED) through the C
ABI, against the oracle (quadrature line integrals of the vector basis,
pseudo-inverse least squares) on the same neighbour lists: per (target, row)
within 1e-10 (FP64) / 1e-9 (FP32 + refinement) of the row's largest weight,
and, at a size the oracle does not reach, reproduction of the Laplacian of a
polynomial of degree m + 1."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs
from tests import _poly

pytestmark = pytest.mark.gpu

TOL = {gmls.FP64: 1e-10, gmls.FP32_REFINE: 1e-9}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()
    c = gmls.Context(0, arena_bytes=8 << 30)
    c.set_option(gmls.OPT_POISON, 1)  # outputs start as NaN: unwritten entries cannot pass
    yield c
    c.close()


# kernel: "auto" (autotuner), "generic" (shared-memory kernel), or a forced
# register kernel with 32 / 16 lanes per target (skipped where not instantiated)
VARIANT = {"reg32": -1, "reg16": -2}


@pytest.mark.parametrize("precision,kernel", [(gmls.FP64, "generic"), (gmls.FP32_REFINE, "generic"),
                                              (gmls.FP32_REFINE, "auto"), (gmls.FP32_REFINE, "reg32"),
                                              (gmls.FP32_REFINE, "reg16")])
@pytest.mark.parametrize("dim,na,m,k", [(2, 24, 2, 24), (2, 24, 3, 36), (2, 24, 4, 48), (3, 9, 2, 40)])
def test_staggered_matches_oracle(ctx, dim, na, m, k, precision, kernel):
    x = inputs.jittered_grid(dim, na, seed=m)
    n = x.shape[1]
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, k, 1.5)
    ctx.set_option(gmls.OPT_FORCE_GENERIC, int(kernel == "generic"))
    ctx.set_option(gmls.OPT_FORCE_VARIANT, VARIANT.get(kernel, 0))
    try:
        sid = ctx.stencils(nid, gmls.STAGGERED, m, [gmls.LAPLACIAN, gmls.GRAD], precision=precision)
    except gmls.GmlsError as e:
        ctx.release(nid)
        ctx.release(cid)
        if e.code == gmls.EINVAL and kernel in VARIANT:
            pytest.skip(f"no {kernel} variant for this shape")
        raise
    finally:
        ctx.set_option(gmls.OPT_FORCE_GENERIC, 0)
        ctx.set_option(gmls.OPT_FORCE_VARIANT, 0)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    st = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    assert np.all((st & (gmls.T_RANK_DEFICIENT | gmls.T_UNSUPPORTED | gmls.T_TOO_FEW_NEIGHBOURS)) == 0)
    sample = np.arange(0, n, max(1, n // 150), dtype=np.int32)
    off = np.arange(0, len(sample) * k + 1, k)
    sub_idx = idx.reshape(n, k)[sample].reshape(-1)
    for fn, name in ((gmls.LAPLACIAN, "laplacian"), (gmls.GRAD, "grad")):
        wo, _ = oracle.staggered_stencils(x, sample, off, sub_idx, eps[sample], m, name)
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(n, wo.shape[1], k, 1)[sample]
        a = np.abs(wg - wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        b = np.abs(wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        assert np.max(a / b) <= TOL[precision], (name, np.max(a / b))
    for h in (sid, nid, cid):
        ctx.release(h)


def test_staggered_reproduces_degree_m_plus_1_at_scale(ctx):
    dim, na, m, k = 2, 256, 3, 36
    x = inputs.jittered_grid(dim, na, seed=5)
    n = x.shape[1]
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, k, 1.5)
    sid = ctx.stencils(nid, gmls.STAGGERED, m, [gmls.LAPLACIAN], precision=gmls.FP32_REFINE)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy().reshape(n, k)
    w = ctx.weights(sid, gmls.LAPLACIAN).cpu().numpy().reshape(n, k)
    p = _poly.random_poly(np.random.default_rng(11), dim, m + 1)
    vals = _poly.evaluate(p, x)
    lap = _poly.evaluate(_poly.laplacian(p, dim), x)
    approx = np.einsum("tk,tk->t", w, vals[idx])
    scale = np.einsum("tk,tk->t", np.abs(w), np.abs(vals[idx])) + np.abs(lap)
    assert np.all(np.abs(approx - lap) <= 1e-9 * scale)
    assert np.allclose(w.sum(axis=1), 0.0, atol=1e-9 * np.abs(w).max())
    for h in (sid, nid, cid):
        ctx.release(h)
