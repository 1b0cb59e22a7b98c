"""GPU parity: libgmls (through its C ABI) against the FP64 CPU oracle.

Neighbour lists and CSR structure must match bit for bit; stencil weights
must satisfy, per (target, functional row),
    |w_gpu - w_oracle|_inf <= tol * |w_oracle|_inf
with tol = 1e-10 for the FP64 path and 1e-9 for the FP32 + refinement path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-9


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


def _gpu_knn(ctx, x, k, f, targets=None, halfspace=None):
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, k, f, targets=targets, halfspace=halfspace)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    st = ctx.export(nid, gmls.X_NBR_STATUS, torch.uint8).cpu().numpy()
    return cid, nid, idx, eps, st


def _release(ctx, *ids):
    for i in reversed(ids):
        ctx.release(i)


def _rel_err_rows(wg, wo):
    """max over (target,row) of |wg - wo|_inf / |wo|_inf; arrays [T, R, k, C]."""
    T, R = wo.shape[:2]
    a = np.abs(wg - wo).reshape(T, R, -1).max(axis=2)
    b = np.abs(wo).reshape(T, R, -1).max(axis=2)
    return float(np.max(a / np.where(b > 0, b, 1.0)))


def _scaled_err(wg, wo, kappa, tol):
    """max over (target, row) of the relative row error divided by the bar
    max(tol, 1e-15 kappa): targets whose FP64 factor has a large
    kappa = max|r_ii| / min|r_ii| are compared at a bar that grows with kappa
    instead of being left out.  For the FP32 path (tol 1e-9) this is
    tol * max(1, kappa * 1e-6); the FP64 path (tol 1e-10) takes the same
    growth term, about 9 kappa u_64: two backward-stable FP64 solutions of a
    problem of condition kappa differ by a small multiple of kappa u_64, which
    a bar of 1e-16 kappa (below kappa u_64) would not admit.  <= 1 passes."""
    T, R = wo.shape[:2]
    a = np.abs(wg - wo).reshape(T, R, -1).max(axis=2)
    b = np.abs(wo).reshape(T, R, -1).max(axis=2)
    rel = a / np.where(b > 0, b, 1.0)
    bar = np.maximum(tol, 1e-15 * kappa)
    return float(np.max(rel / bar[:, None]))


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("dim,n_axis,k,jitter", [(2, 32, 12, 0.25), (2, 40, 48, 0.25), (3, 12, 40, 0.25),
                                                 (3, 10, 80, 0.25), (2, 16, 13, 0.0), (3, 8, 27, 0.0),
                                                 (2, 5, 7, 0.25)])
def test_knn_bit_exact(ctx, dim, n_axis, k, jitter):
    x = inputs.jittered_grid(dim, n_axis, jitter=jitter, seed=1)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, k, 1.5)
    oi, oe = oracle.knn(x, np.arange(n, dtype=np.int32), k, 1.5, method="grid")
    assert np.all(st == 0)
    assert np.array_equal(idx.reshape(n, k), oi)
    assert np.array_equal(eps, oe)  # bit for bit
    _release(ctx, cid, nid)


def test_prefix_equals_direct_search(ctx):
    x = inputs.jittered_grid(2, 64, seed=6)
    cid = ctx.cloud(x)
    n48 = ctx.neighbors(cid, 48, 1.5)
    direct = ctx.neighbors(cid, 36, 1.5)
    pref = ctx.neighbors_prefix(n48, 36, 1.5)
    for what, dt in ((gmls.X_NBR_INDEX, torch.int32), (gmls.X_NBR_EPS, torch.float64),
                     (gmls.X_NBR_STATUS, torch.uint8), (gmls.X_NBR_OFFSETS, torch.int64)):
        assert torch.equal(ctx.export(pref, what, dt), ctx.export(direct, what, dt))
    _release(ctx, cid, n48, direct, pref)


def test_knn_halfspace_and_subset_targets(ctx):
    x = inputs.jittered_grid(2, 48, seed=4)
    n = x.shape[1]
    inner = np.flatnonzero((np.abs(x[0] - 0.5) < 0.35) & (np.abs(x[1] - 0.5) < 0.35)).astype(np.int32)
    tg = inner[::3]
    hs = inputs.unit_vectors(2, 7, len(tg), 2).T.copy()
    hs[::4] = 0.0
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, 20, 1.8, targets=tg, halfspace=hs)
    oi, oe = oracle.knn(x, tg, 20, 1.8, halfspace=hs, method="grid")
    assert np.array_equal(idx.reshape(len(tg), 20), oi) and np.array_equal(eps, oe)
    _release(ctx, cid, nid)


def test_radius_bit_exact(ctx):
    x = inputs.jittered_grid(3, 20, seed=2)
    n = x.shape[1]
    tg = np.arange(0, n, 5, dtype=np.int32)
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, 20, 1.8, mode=gmls.RADIUS, cap=160, targets=tg)
    off = ctx.export(nid, gmls.X_NBR_OFFSETS, torch.int64).cpu().numpy()
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    _, oe = oracle.knn(x, tg, 20, 1.8, method="grid")
    assert np.array_equal(eps, oe)
    ooff, oidx = oracle.radius(x, tg, oe, 160, method="grid")
    assert np.array_equal(off, ooff) and np.array_equal(idx, oidx)
    _release(ctx, cid, nid)


def test_too_few_neighbours_is_flagged(ctx):
    x = inputs.jittered_grid(2, 6, seed=1)  # 36 points
    cid = ctx.cloud(x)
    hs = np.zeros((36, 2))
    hs[0] = [1.0, 1.0]  # corner target, half-plane pointing inwards: few points qualify
    hs[0] /= np.sqrt(2.0)
    nid = ctx.neighbors(cid, 12, 1.5, halfspace=hs)
    st = ctx.export(nid, gmls.X_NBR_STATUS, torch.uint8).cpu().numpy()
    assert st[0] & gmls.T_TOO_FEW_NEIGHBOURS
    assert np.all(st[1:] == 0)
    sid = ctx.stencils(nid, gmls.SCALAR, 2, [gmls.LAPLACIAN])
    sst = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    w = ctx.weights(sid, gmls.LAPLACIAN).cpu().numpy().reshape(36, 12)
    assert sst[0] & gmls.T_TOO_FEW_NEIGHBOURS and np.all(w[0] == 0.0)
    _release(ctx, cid, nid, sid)


# -------------------------------------------------------------------- stencils
CASES = [
    # dim, n_axis, basis, m, k, functionals
    (2, 32, gmls.SCALAR, 2, 12, [gmls.LAPLACIAN, gmls.GRAD]),
    (2, 40, gmls.SCALAR, 4, 36, [gmls.GRAD, gmls.DIV, gmls.LAPLACIAN]),
    (2, 40, gmls.DIVFREE, 4, 48, [gmls.VEC_LAPLACIAN, gmls.CURLCURL, gmls.DIV]),
    (2, 24, gmls.DIVFREE, 2, 22, [gmls.VEC_LAPLACIAN]),
    (2, 30, gmls.DIVFREE, 3, 34, [gmls.VEC_LAPLACIAN, gmls.CURLCURL]),
    (3, 12, gmls.SCALAR, 3, 40, [gmls.GRAD, gmls.LAPLACIAN]),
    (3, 12, gmls.DIVFREE, 3, 80, [gmls.VEC_LAPLACIAN]),
    (3, 9, gmls.SCALAR, 4, 84, [gmls.GRAD, gmls.LAPLACIAN]),
    (3, 9, gmls.DIVFREE, 2, 42, [gmls.CURLCURL]),
    (3, 9, gmls.DIVFREE, 4, 136, [gmls.VEC_LAPLACIAN]),  # 408 x 85: tiles in global memory
]
NAMES = {gmls.GRAD: "grad", gmls.LAPLACIAN: "laplacian", gmls.DIV: "div", gmls.VEC_LAPLACIAN: "vec_laplacian",
         gmls.CURLCURL: "curlcurl"}


# forced variants: register kernel (-1, -2, -4: 32, 16, 8 lanes a target);
# factored div-free kernel (-3); shared-memory kernel G + 8 * placement
# (split: float-float tile in global memory; global: both tiles there)
VARIANT = {"reg32": -1, "reg16": -2, "dfx": -3, "reg8": -4, "split4": 4 + 8, "global1": 1 + 16, "global2": 2 + 16}


@pytest.mark.parametrize("precision,kernel", [(gmls.FP64, "generic"), (gmls.FP32_REFINE, "generic"),
                                              (gmls.FP32_REFINE, "auto"), (gmls.FP32_REFINE, "reg32"),
                                              (gmls.FP32_REFINE, "reg16"), (gmls.FP32_REFINE, "reg8"),
                                              (gmls.FP32_REFINE, "dfx"),
                                              (gmls.FP32_REFINE, "split4"),
                                              (gmls.FP32_REFINE, "global1"), (gmls.FP64, "global2")])
@pytest.mark.parametrize("dim,n_axis,basis,m,k,fns", CASES)
def test_stencils_match_oracle(ctx, dim, n_axis, basis, m, k, fns, precision, kernel):
    x = inputs.jittered_grid(dim, n_axis, seed=m)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, k, 1.5)
    ctx.set_option(gmls.OPT_FORCE_GENERIC, int(kernel == "generic"))
    ctx.set_option(gmls.OPT_FORCE_VARIANT, VARIANT.get(kernel, 0))
    try:
        sid = ctx.stencils(nid, basis, m, fns, precision=precision)
    except gmls.GmlsError as e:
        _release(ctx, cid, nid)
        if e.code == gmls.EINVAL and kernel in VARIANT:
            pytest.skip(f"no {kernel} variant for this shape")
        raise
    finally:
        ctx.set_option(gmls.OPT_FORCE_GENERIC, 0)
        ctx.set_option(gmls.OPT_FORCE_VARIANT, 0)
    status = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    tg = np.arange(n, dtype=np.int32)
    off = np.arange(0, n * k + 1, k)
    kind = "scalar" if basis == gmls.SCALAR else "divfree"
    tol = TOL64 if precision == gmls.FP64 else TOL32
    for fn in fns:
        wo, _, diag = oracle.stencils(x, tg, off, idx, eps, kind, m, NAMES[fn])
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(wo.shape)
        if fn == gmls.DIV and basis == gmls.DIVFREE:
            # divergence of a divergence-free reconstruction: exactly zero on
            # the GPU, zero up to rounding in the oracle
            assert np.all(wg == 0.0)
            assert np.abs(wo).max() <= 1e-9 / eps.min()
            continue
        kappa = diag[:, 0] / diag[:, 1]
        err = _scaled_err(wg, wo, kappa, tol)  # every target, ill-conditioned ones at the scaled bar
        assert err <= 1.0, (NAMES[fn], err * tol)
    assert np.all((status & (gmls.T_RANK_DEFICIENT | gmls.T_TOO_FEW_NEIGHBOURS)) == 0)
    _release(ctx, cid, nid, sid)


@pytest.mark.parametrize("precision,kernel", [(gmls.FP64, "generic"), (gmls.FP32_REFINE, "auto"),
                                              (gmls.FP32_REFINE, "generic")])
@pytest.mark.parametrize("m,k,jitter", [(4, 15, 1e-4), (3, 10, 1e-5), (2, 6, 1e-6)])
def test_ill_conditioned_targets(ctx, m, k, jitter, precision, kernel):
    """Nearly exact lattices (jitter 1e-6 .. 1e-4 of the spacing) with as
    many neighbours as basis functions: many factors have
    kappa = max|r_ii| / min|r_ii| far above 1e6 (up to ~1e11).  Every target
    is compared, at max(tol, 1e-15 kappa); the FP32 path hands the
    ill-conditioned ones to its FP64 redo and flags them."""
    x = inputs.jittered_grid(2, 30, jitter=jitter, seed=m)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, k, 1.5)
    ctx.set_option(gmls.OPT_FORCE_GENERIC, int(kernel == "generic"))
    try:
        sid = ctx.stencils(nid, gmls.SCALAR, m, [gmls.GRAD, gmls.LAPLACIAN], precision=precision)
    finally:
        ctx.set_option(gmls.OPT_FORCE_GENERIC, 0)
    status = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    tg = np.arange(n, dtype=np.int32)
    off = np.arange(0, n * k + 1, k)
    tol = TOL64 if precision == gmls.FP64 else TOL32
    for fn in (gmls.GRAD, gmls.LAPLACIAN):
        wo, _, diag = oracle.stencils(x, tg, off, idx, eps, "scalar", m, NAMES[fn])
        kappa = diag[:, 0] / diag[:, 1]
        assert (kappa > 1e6).sum() >= 20  # the case does exercise the scaled bar
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(wo.shape)
        assert _scaled_err(wg, wo, kappa, tol) <= 1.0
        if precision == gmls.FP32_REFINE:
            # the FP32 factor of a target with kappa > 1e7 cannot pass the
            # FP32 conditioning test: such targets must have been redone
            redone = (status & gmls.T_FP64_FALLBACK) != 0
            assert np.all(redone[kappa > 1e7])
    assert np.all((status & gmls.T_TOO_FEW_NEIGHBOURS) == 0)
    _release(ctx, cid, nid, sid)


@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
@pytest.mark.parametrize("shift", [0.0, 1.0, 1e2, 1e4])
@pytest.mark.parametrize("dim,n_axis,basis,m,k", [(2, 40, gmls.SCALAR, 4, 36), (2, 40, gmls.DIVFREE, 4, 48),
                                                  (3, 10, gmls.DIVFREE, 3, 80)])
def test_translated_and_scaled_clouds(ctx, dim, n_axis, basis, m, k, shift, precision):
    """The same jittered grid at spacing h = 2^-12, translated by
    c in {0, 1, 1e2, 1e4} along every axis: neighbour lists and eps bit for
    bit, and every target's weights within the bar.  Offsets x_j - x_T are
    FP64 differences on both sides (the stencils depend on the cloud only
    through them, Sec. 2.1), so the GPU result does not degrade with |x| / h."""
    x = inputs.jittered_grid(dim, n_axis, h=2.0 ** -12, lo=shift, seed=m + 7)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, k, 1.5)
    tg = np.arange(n, dtype=np.int32)
    oi, oe = oracle.knn(x, tg, k, 1.5, method="grid")
    assert np.all(st == 0)
    assert np.array_equal(idx.reshape(n, k), oi) and np.array_equal(eps, oe)
    fn = gmls.GRAD if basis == gmls.SCALAR else gmls.VEC_LAPLACIAN
    sid = ctx.stencils(nid, basis, m, [fn], precision=precision)
    off = np.arange(0, n * k + 1, k)
    kind = "scalar" if basis == gmls.SCALAR else "divfree"
    wo, _, diag = oracle.stencils(x, tg, off, idx, eps, kind, m, NAMES[fn])
    wg = ctx.weights(sid, fn).cpu().numpy().reshape(wo.shape)
    tol = TOL64 if precision == gmls.FP64 else TOL32
    assert _scaled_err(wg, wo, diag[:, 0] / diag[:, 1], tol) <= 1.0
    _release(ctx, cid, nid, sid)


def test_refinement_iterations_and_fallback_flags(ctx):
    x = inputs.jittered_grid(2, 40, seed=4)
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, 48, 1.5)
    sid = ctx.stencils(nid, gmls.DIVFREE, 4, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE)
    it = ctx.export(sid, gmls.X_ITERS, torch.uint8).cpu().numpy()
    status = ctx.export(sid, gmls.X_STATUS, torch.uint8).cpu().numpy()
    redone = (status & gmls.T_FP64_FALLBACK) != 0
    assert np.all(it[~redone] >= 1) and np.all(it <= 3)
    _release(ctx, cid, nid, sid)


def test_factored_kernel_hands_refinement_misses_to_fp32_kernel(ctx):
    """The factored div-free kernel refines once.  A well-conditioned target
    whose one step misses the tolerance goes on to the shared-memory FP32
    kernel, which refines further: with max_refine = 1 such targets are FP64
    redos (flagged), with the default they are not, and their weights meet
    the bar against the oracle."""
    x = inputs.jittered_grid(2, 160, seed=11)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, 48, 1.5)
    ctx.set_option(gmls.OPT_FORCE_VARIANT, -3)
    try:
        s1 = ctx.stencils(nid, gmls.DIVFREE, 4, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE, max_refine=1)
        st1 = ctx.export(s1, gmls.X_STATUS, torch.uint8).cpu().numpy()
        ctx.release(s1)
        s3 = ctx.stencils(nid, gmls.DIVFREE, 4, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE)
    finally:
        ctx.set_option(gmls.OPT_FORCE_VARIANT, 0)
    st3 = ctx.export(s3, gmls.X_STATUS, torch.uint8).cpu().numpy()
    miss = ((st1 & gmls.T_REFINE_NOT_CONVERGED) != 0) & ((st1 & gmls.T_ILL_CONDITIONED) == 0)
    assert np.all((st1[miss] & gmls.T_FP64_FALLBACK) != 0)
    assert miss.sum() > 0  # the case exercises the hand-off
    assert not np.any(st3[miss] & gmls.T_FP64_FALLBACK)
    tg = np.nonzero(miss)[0].astype(np.int32)
    k = 48
    wo, _, diag = oracle.stencils(x, tg, np.arange(0, tg.size * k + 1, k), idx.reshape(n, k)[tg].ravel(), eps[tg],
                                  "divfree", 4, NAMES[gmls.VEC_LAPLACIAN])
    wg = ctx.weights(s3, gmls.VEC_LAPLACIAN).cpu().numpy().reshape((n,) + wo.shape[1:])[tg]
    assert _scaled_err(wg, wo, diag[:, 0] / diag[:, 1], TOL32) <= 1.0
    _release(ctx, cid, nid, s3)


# ------------------------------------------------------------------- Neumann
@pytest.mark.parametrize("precision", [gmls.FP64, gmls.FP32_REFINE])
@pytest.mark.parametrize("dim,n_axis,m,k", [(2, 24, 2, 12), (2, 24, 4, 36), (3, 10, 3, 40)])
def test_neumann_matches_oracle(ctx, dim, n_axis, m, k, precision):
    x = inputs.jittered_grid(dim, n_axis, seed=3)
    n = x.shape[1]
    nrm = inputs.unit_vectors(5, 6, n, dim)
    bflag = (inputs.uniform(5, 8, n) < 0.3).astype(np.uint8)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nid = ctx.neighbors(cid, k, 1.5)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
    sid = ctx.stencils(nid, gmls.SCALAR, m, [gmls.LAPLACIAN, gmls.GRAD], precision=precision, neumann=True)
    beta = ctx.export(sid, gmls.X_BETA, torch.float64).cpu().numpy().reshape(n, -1)
    tg = np.arange(n, dtype=np.int32)
    off = np.arange(0, n * k + 1, k)
    tol = TOL64 if precision == gmls.FP64 else TOL32
    # solve rows are ordered grad (dim rows) then laplacian
    for fn, rows in ((gmls.GRAD, slice(0, dim)), (gmls.LAPLACIAN, slice(dim, dim + 1))):
        wo, bo, _ = oracle.stencils(x, tg, off, idx, eps, "scalar", m, NAMES[fn], bflag=bflag, normals=nrm.T)
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(wo.shape)
        assert _rel_err_rows(wg, wo) <= tol
        bg = beta[:, rows]
        # beta multiplies h = n . grad u ~ u / eps, so it scales like |w| eps
        scale = np.abs(bo) + np.abs(wo).reshape(n, wo.shape[1], -1).max(axis=2) * eps[:, None]
        assert np.all(np.abs(bg - bo) <= tol * scale)
        assert np.all(bg[bflag == 0] == 0.0)
    _release(ctx, cid, nid, sid)


@pytest.mark.parametrize("variant", [-1, -2])
@pytest.mark.parametrize("dim,n_axis,m,k", [(2, 24, 4, 36), (3, 10, 3, 40)])
def test_neumann_register_kernel_matches_oracle(ctx, dim, n_axis, m, k, variant):
    """The register kernel's Neumann instantiation (boundary targets in a
    second launch over the list the first one fills), a warp (-1) or half a
    warp (-2) per target."""
    ctx.set_option(gmls.OPT_FORCE_VARIANT, variant)
    try:
        test_neumann_matches_oracle(ctx, dim, n_axis, m, k, gmls.FP32_REFINE)
    finally:
        ctx.set_option(gmls.OPT_FORCE_VARIANT, 0)


# ------------------------------------------------------------------------ CSR
@pytest.mark.parametrize("basis,m,k,fn", [(gmls.SCALAR, 4, 36, gmls.GRAD), (gmls.DIVFREE, 4, 48, gmls.VEC_LAPLACIAN),
                                          (gmls.SCALAR, 4, 36, gmls.DIV)])
def test_csr_structure_bit_exact(ctx, basis, m, k, fn):
    x = inputs.jittered_grid(2, 30, seed=2)
    n = x.shape[1]
    cid, nid, idx, eps, st = _gpu_knn(ctx, x, k, 1.5)
    sid = ctx.stencils(nid, basis, m, [fn])
    rp, col, val = (t.cpu().numpy() for t in ctx.assemble_csr(sid, fn))
    wg = ctx.weights(sid, fn).cpu().numpy()
    nt, rows, nc, _ = ctx.stencil_info(sid, fn)
    off = np.arange(0, n * k + 1, k)
    wq = [wg[q * rows * k * nc:(q + 1) * rows * k * nc].reshape(rows, k, nc) for q in range(n)]
    orp, ocol, oval, _ = oracle.csr(off, idx, wq, n)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    assert np.array_equal(val, oval)  # the same weights, permuted: bit for bit
    _release(ctx, cid, nid, sid)


@pytest.mark.parametrize("parent_first", [False, True])
def test_csr_of_prefix_lists_equals_direct_lists(ctx, parent_first):
    """The id order of a prefix list is derived from its parent's: CSR of the
    36-prefix of 48-nearest lists equals CSR of the 36-nearest lists, bit for
    bit, whether or not the parent's CSR was assembled first."""
    x = inputs.jittered_grid(2, 40, seed=6)
    cid = ctx.cloud(x)
    n48 = ctx.neighbors(cid, 48, 1.5)
    n36p = ctx.neighbors_prefix(n48, 36, 1.5)
    n36 = ctx.neighbors(cid, 36, 1.5)
    s48 = ctx.stencils(n48, gmls.SCALAR, 4, [gmls.GRAD])
    if parent_first:
        ctx.assemble_csr(s48, gmls.GRAD)
    sp = ctx.stencils(n36p, gmls.SCALAR, 4, [gmls.GRAD, gmls.DIV])
    sd = ctx.stencils(n36, gmls.SCALAR, 4, [gmls.GRAD, gmls.DIV])
    for fn in (gmls.GRAD, gmls.DIV):
        a = [t.cpu().numpy() for t in ctx.assemble_csr(sp, fn)]
        b = [t.cpu().numpy() for t in ctx.assemble_csr(sd, fn)]
        assert all(np.array_equal(u, v) for u, v in zip(a, b))
    _release(ctx, cid, n48, n36p, n36, s48, sp, sd)


@pytest.mark.parametrize("dim,n_axis,basis,m,k,fn,mode", [(2, 30, gmls.SCALAR, 4, 36, gmls.GRAD, gmls.KNN),
                                                          (3, 10, gmls.DIVFREE, 3, 80, gmls.VEC_LAPLACIAN, gmls.KNN),
                                                          (2, 28, gmls.SCALAR, 2, 12, gmls.GRAD, gmls.RADIUS)])
def test_csr_column_order_same_for_both_key_widths(ctx, dim, n_axis, basis, m, k, fn, mode):
    """The id order of the lists (the CSR column order) is sorted on 32-bit
    keys for clouds below 2^25 - 1 points and on 64-bit keys above: forcing
    the 64-bit keys on a small cloud gives the same operator bit for bit
    (lists of up to 64 and of 65..128 entries, fixed-k and radius lists)."""
    x = inputs.jittered_grid(dim, n_axis, seed=9)
    cid = ctx.cloud(x)
    kw = {"mode": mode, "cap": 40} if mode == gmls.RADIUS else {}
    out = []
    for key64 in (0, 1):
        ctx.set_option(gmls.OPT_ORDER_KEY64, key64)
        try:
            nid = ctx.neighbors(cid, k, 1.6 if mode == gmls.RADIUS else 1.5, **kw)
            sid = ctx.stencils(nid, basis, m, [fn])
            out.append([t.cpu().numpy() for t in ctx.assemble_csr(sid, fn)])
        finally:
            ctx.set_option(gmls.OPT_ORDER_KEY64, 0)
        _release(ctx, nid, sid)
    assert all(np.array_equal(u, v) for u, v in zip(out[0], out[1]))
    assert np.all(np.diff(out[0][1].reshape(-1)[: out[0][0][1]]) > 0)  # first row: ascending columns
    _release(ctx, cid)


def test_csr_assembled_in_target_ranges(ctx):
    """gmls_assemble_csr_at: an operator assembled range by range (one
    neighbour handle per contiguous target range, uneven range sizes, radius
    lists) equals the operator assembled at once, bit for bit."""
    x = inputs.jittered_grid(2, 28, seed=4)
    n = x.shape[1]
    cid = ctx.cloud(x)
    whole = ctx.neighbors(cid, 12, 1.6, mode=gmls.RADIUS, cap=40)
    sw = ctx.stencils(whole, gmls.SCALAR, 2, [gmls.GRAD])
    rp, col, val = (t.cpu().numpy() for t in ctx.assemble_csr(sw, gmls.GRAD))
    out = (torch.full((len(rp),), -7, dtype=torch.int64, device=ctx.device),
           torch.full((len(col),), -7, dtype=torch.int32, device=ctx.device),
           torch.full((len(val),), -7.0, dtype=torch.float64, device=ctx.device))
    bounds = [0, 1, 300, 300, 301, 560, n]  # includes an empty range
    nnz = 0
    for a, b in zip(bounds[:-1], bounds[1:]):
        tg = torch.arange(a, b, dtype=torch.int32, device=ctx.device)
        nid = ctx.neighbors(cid, 12, 1.6, mode=gmls.RADIUS, cap=40, targets=tg)
        sid = ctx.stencils(nid, gmls.SCALAR, 2, [gmls.GRAD])
        _, _, z = ctx.csr_size(sid, gmls.GRAD)
        ctx.assemble_csr(sid, gmls.GRAD, out=(out[0][2 * a:2 * b + 1], out[1][nnz:nnz + z], out[2][nnz:nnz + z]),
                         nnz_offset=nnz)
        nnz += z
        _release(ctx, nid, sid)
    assert nnz == len(col)
    assert np.array_equal(out[0].cpu().numpy(), rp)
    assert np.array_equal(out[1].cpu().numpy(), col) and np.array_equal(out[2].cpu().numpy(), val)
    with pytest.raises(gmls.GmlsError) as e:
        ctx.assemble_csr(sw, gmls.GRAD, out=out, nnz_offset=-1)
    assert e.value.code == gmls.EINVAL
    _release(ctx, cid, whole, sw)


# ----------------------------------------------------- full-size configuration
def test_full_size_512x512_sampled(ctx):
    """The benchmark's workload (262,144 targets on a 512 x 512 jittered grid,
    scalar m=4 with 36 neighbours and divergence-free m=4 with 48), checked
    on sampled targets that the oracle computes one by one."""
    x = inputs.jittered_grid(2, 512, seed=0)
    n = x.shape[1]
    cid = ctx.cloud(x)
    sample = np.unique((inputs.uniform(0, 99, 300) * n).astype(np.int32))
    for basis, k, fn in ((gmls.SCALAR, 36, gmls.GRAD), (gmls.DIVFREE, 48, gmls.VEC_LAPLACIAN)):
        nid = ctx.neighbors(cid, k, 1.5)
        sid = ctx.stencils(nid, basis, 4, [fn], precision=gmls.FP32_REFINE)
        idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).cpu().numpy().reshape(n, k)
        eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64).cpu().numpy()
        oi, oe = oracle.knn(x, sample, k, 1.5, method="grid")
        assert np.array_equal(idx[sample], oi) and np.array_equal(eps[sample], oe)
        kind = "scalar" if basis == gmls.SCALAR else "divfree"
        off = np.arange(0, len(sample) * k + 1, k)
        wo, _, _ = oracle.stencils(x, sample, off, oi.reshape(-1), oe, kind, 4, NAMES[fn])
        _, rows, nc, _ = ctx.stencil_info(sid, fn)
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(n, rows, k, nc)[sample]
        assert _rel_err_rows(wg, wo) <= TOL32
        ctx.release(sid)
        ctx.release(nid)
    ctx.release(cid)
