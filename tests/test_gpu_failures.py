"""GPU tests of the host-side failure paths through the C ABI.

* allocation faults: with GMLS_OPT_FAIL_ALLOC = n the n-th sub-allocation of
  a call fails; every position makes the call return GMLS_ENOMEM, leaves the
  arena exactly as it was (no leaked block) and leaves the context usable: a
  later call gives the same result as on a fresh context;
* request cancellation: a request still waiting for admission is cancelled
  and never runs (wait and result report GMLS_ECANCELED), the others finish
  with the same results as alone; a running or finished request cannot be
  cancelled (GMLS_EBUSY), an unknown ticket is GMLS_ENOTFOUND.
No GPU fault, trap or hang is involved: the failures are made on the host.
"""
import numpy as np
import pytest
import torch

from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()


def _pipeline(ctx, x, basis, m, k, fns, precision):
    """cloud -> lists -> stencils -> CSR; on an error the handles made so far
    are released (newest first) before it propagates."""
    made = []
    try:
        made.append(ctx.cloud(x))
        made.append(ctx.neighbors(made[0], k, 1.5))
        made.append(ctx.stencils(made[1], basis, m, fns, precision=precision))
        w = [ctx.weights(made[2], f).cpu().numpy().copy() for f in fns]
        rp, col, val = (t.cpu().numpy() for t in ctx.assemble_csr(made[2], fns[0]))
        ctx.sync()
        return w, (rp, col, val)
    finally:
        for h in reversed(made):
            ctx.release(h)


@pytest.mark.parametrize("basis,m,k,fns,precision", [
    (gmls.SCALAR, 4, 36, [gmls.GRAD, gmls.LAPLACIAN], gmls.FP32_REFINE),
    (gmls.DIVFREE, 3, 80, [gmls.VEC_LAPLACIAN], gmls.FP32_REFINE),
    (gmls.SCALAR, 2, 12, [gmls.LAPLACIAN], gmls.FP64)])
def test_every_allocation_fault_unwinds(built, basis, m, k, fns, precision):
    dim = 3 if basis == gmls.DIVFREE else 2
    x = inputs.jittered_grid(dim, 9 if dim == 3 else 24, seed=2)
    ref = _pipeline(gmls.Context(0, arena_bytes=1 << 30), x, basis, m, k, fns, precision)
    ctx = gmls.Context(0, arena_bytes=1 << 30)
    _pipeline(ctx, x, basis, m, k, fns, precision)  # autotune once, outside the faults
    faults = 0
    for n in range(1, 80):
        used0 = ctx.arena_usage()[0]
        ctx.set_option(gmls.OPT_FAIL_ALLOC, n)
        try:
            got = _pipeline(ctx, x, basis, m, k, fns, precision)
        except gmls.GmlsError as e:
            assert e.code == gmls.ENOMEM, e
            faults += 1
            ctx.set_option(gmls.OPT_FAIL_ALLOC, 0)
            ctx.sync()
            assert ctx.arena_usage()[0] == used0, n  # the failed call and its predecessors left nothing
            continue
        ctx.set_option(gmls.OPT_FAIL_ALLOC, 0)
        # past the last allocation of the pipeline: nothing failed
        assert all(np.array_equal(a, b) for a, b in zip(got[0], ref[0]))
        assert all(np.array_equal(a, b) for a, b in zip(got[1], ref[1]))
        break
    assert faults >= 5  # cloud, lists, stencils and CSR each allocate
    # the context is still usable after the faults
    got = _pipeline(ctx, x, basis, m, k, fns, precision)
    assert all(np.array_equal(a, b) for a, b in zip(got[0], ref[0]))
    ctx.close()


def test_fault_inside_one_call_leaves_no_block(built):
    """Within a single gmls_stencils call every allocation position fails
    cleanly: the call returns GMLS_ENOMEM with the arena usage unchanged."""
    x = inputs.jittered_grid(3, 8, seed=5)
    ctx = gmls.Context(0, arena_bytes=1 << 30)
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, 80, 1.5)
    ctx.release(ctx.stencils(nid, gmls.DIVFREE, 3, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE))
    ctx.sync()
    used0 = ctx.arena_usage()[0]
    hit = 0
    for n in range(1, 40):
        ctx.set_option(gmls.OPT_FAIL_ALLOC, n)
        try:
            sid = ctx.stencils(nid, gmls.DIVFREE, 3, [gmls.VEC_LAPLACIAN], precision=gmls.FP32_REFINE)
        except gmls.GmlsError as e:
            assert e.code == gmls.ENOMEM
            ctx.sync()
            assert ctx.arena_usage()[0] == used0, n
            hit += 1
            continue
        finally:
            ctx.set_option(gmls.OPT_FAIL_ALLOC, 0)
        ctx.release(sid)
        ctx.sync()
        assert ctx.arena_usage()[0] == used0
        break
    assert hit >= 3
    for h in (nid, cid):
        ctx.release(h)
    ctx.close()


def test_cancel_a_waiting_request(built):
    xs = [inputs.jittered_grid(3, 40, seed=1), inputs.jittered_grid(2, 64, seed=2),
          inputs.jittered_grid(2, 48, seed=3)]
    specs = [(gmls.DIVFREE, 3, 80, [gmls.VEC_LAPLACIAN]), (gmls.SCALAR, 4, 36, [gmls.GRAD]),
             (gmls.SCALAR, 2, 12, [gmls.LAPLACIAN])]
    srv = gmls.Server(0, arena_bytes=4 << 30, streams=1, max_inflight=1)  # one slot: the others wait
    t = [srv.submit(x, *sp) for x, sp in zip(xs, specs)]
    assert srv.cancel(t[1]) == gmls.OK  # still waiting behind the first request
    with pytest.raises(gmls.GmlsError) as e:
        srv.wait(t[1], 1000)
    assert e.value.code == gmls.ECANCELED
    with pytest.raises(gmls.GmlsError) as e:
        srv.result(t[1], gmls.X_WEIGHTS, torch.float64, gmls.GRAD)
    assert e.value.code == gmls.ECANCELED
    for i in (0, 2):
        assert srv.wait(t[i], 120000)
    assert srv.cancel(t[0]) == gmls.EBUSY  # finished: nothing to cancel
    with pytest.raises(gmls.GmlsError) as e:
        srv.cancel(123456)
    assert e.value.code == gmls.ENOTFOUND
    st = srv.stats()
    assert st["completed"] == 2 and st["pending"] == 0
    # the survivors equal the same requests run alone
    for i in (0, 2):
        alone = gmls.Server(0, arena_bytes=4 << 30, streams=1, max_inflight=1)
        ta = alone.submit(xs[i], *specs[i])
        assert alone.wait(ta, 120000)
        for f in specs[i][3]:
            a = alone.result(ta, gmls.X_WEIGHTS, torch.float64, f)
            b = srv.result(t[i], gmls.X_WEIGHTS, torch.float64, f)
            assert torch.equal(a, b)
        alone.release(ta)
        alone.close()
    for i in range(3):
        srv.release(t[i])
    srv.close()
