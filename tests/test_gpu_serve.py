"""GPU tests of the continuous-batching server (gmls_server_*): every result in
a concurrent mix equals the same request run alone (bit for bit) and matches
the oracle on sampled targets; requests wait for arena memory and are admitted
as earlier ones are released; a request larger than the arena fails cleanly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu

K = {(2, "scalar", 2): 12, (2, "scalar", 3): 20, (2, "scalar", 4): 36, (2, "divfree", 2): 22,
     (2, "divfree", 3): 34, (2, "divfree", 4): 48, (3, "scalar", 2): 20, (3, "scalar", 3): 40,
     (3, "scalar", 4): 84, (3, "divfree", 2): 42, (3, "divfree", 3): 80, (3, "divfree", 4): 136}
FUN = {"scalar": [gmls.GRAD, gmls.LAPLACIAN], "divfree": [gmls.VEC_LAPLACIAN]}


def _requests(count, seed, nmax=6000):
    out = []
    for i in range(count):
        u = inputs.uniform(seed, 7, 4, offset=4 * i)
        dim = 2 if u[0] < 0.5 else 3
        kind = "scalar" if u[1] < 0.5 else "divfree"
        m = 2 + int(3 * u[2])
        n_axis = int((500 + (nmax - 500) * u[3]) ** (1.0 / dim))
        x = inputs.jittered_grid(dim, n_axis, seed=seed + i)
        out.append((dim, kind, m, x))
    return out


def _submit(srv, req):
    dim, kind, m, x = req
    return srv.submit(x, gmls.SCALAR if kind == "scalar" else gmls.DIVFREE, m, K[(dim, kind, m)], FUN[kind])


def _weights(srv, t, kind):
    return [srv.result(t, gmls.X_WEIGHTS, torch.float64, f).numpy() for f in FUN[kind]]


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()


def test_mix_equals_alone_and_oracle(built):
    reqs = _requests(12, 3)
    srv = gmls.Server(0, arena_bytes=8 << 30, streams=4, max_inflight=8)
    tickets = [_submit(srv, r) for r in reqs]  # all submitted at once: they overlap
    for t in tickets:
        assert srv.wait(t, 120000)
    mixed = [_weights(srv, t, r[1]) for t, r in zip(tickets, reqs)]
    idx = [srv.result(t, gmls.X_NBR_INDEX, torch.int32).numpy() for t in tickets]
    eps = [srv.result(t, gmls.X_NBR_EPS, torch.float64).numpy() for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    for t in tickets:
        srv.release(t)
    # alone: one request at a time through the same server
    for r, wm in zip(reqs, mixed):
        t = _submit(srv, r)
        assert srv.wait(t, 120000)
        wa = _weights(srv, t, r[1])
        srv.release(t)
        for a, b in zip(wa, wm):
            assert np.array_equal(a, b)
    srv.close()
    # oracle on sampled targets
    names = {gmls.GRAD: "grad", gmls.LAPLACIAN: "laplacian", gmls.VEC_LAPLACIAN: "vec_laplacian"}
    for (dim, kind, m, x), wm, ix, ep in zip(reqs, mixed, idx, eps):
        n = x.shape[1]
        k = K[(dim, kind, m)]
        samp = np.arange(0, n, max(1, n // 20), dtype=np.int32)
        off = np.arange(0, len(samp) * k + 1, k)
        ixr = ix.reshape(n, k)
        for f, w in zip(FUN[kind], wm):
            wo, _, diag = oracle.stencils(x, samp, off, ixr[samp].reshape(-1), ep[samp], kind, m, names[f])
            rows, nc = wo.shape[1], wo.shape[3]
            wg = w.reshape(n, rows, k, nc)[samp]
            err = np.abs(wg - wo).reshape(len(samp), -1).max(1) / np.abs(wo).reshape(len(samp), -1).max(1)
            kappa = diag[:, 0] / diag[:, 1]
            assert np.all(err <= 1e-9 * np.maximum(1.0, kappa * 1e-6)), (dim, kind, m, err.max())


def test_admission_waits_for_memory(built):
    reqs = _requests(6, 9, nmax=3000)
    srv = gmls.Server(0, arena_bytes=160 << 20, streams=2, max_inflight=8)
    tickets = [_submit(srv, r) for r in reqs]
    done = set()
    for _ in range(2000):
        for t in tickets:
            if t not in done and srv.wait(t, 1):
                done.add(t)
                srv.release(t)  # frees arena for the requests still waiting
        if len(done) == len(tickets):
            break
    assert len(done) == len(tickets)
    assert srv.stats()["completed"] == len(tickets)
    srv.close()


def test_request_larger_than_arena_fails_cleanly(built):
    srv = gmls.Server(0, arena_bytes=64 << 20, streams=1, max_inflight=2)
    x = inputs.jittered_grid(3, 60, seed=1)  # 216,000 points, 3D div-free m=4
    t = srv.submit(x, gmls.DIVFREE, 4, 136, [gmls.VEC_LAPLACIAN])
    with pytest.raises(gmls.GmlsError):
        srv.wait(t, 60000)
    srv.release(t)
    srv.close()


def test_divfree_request_slice_covers_kernel_scratch(built):
    """A 3D degree-3 divergence-free request runs through the factored kernel,
    whose per-warp scratch (tens of MB) comes out of the request's slice."""
    srv = gmls.Server(0, arena_bytes=1 << 30, streams=1, max_inflight=1)
    x = inputs.jittered_grid(3, 24, seed=5)  # 13,824 points
    t = srv.submit(x, gmls.DIVFREE, 3, 80, [gmls.VEC_LAPLACIAN])
    assert srv.wait(t, 60000)
    w = srv.result(t, gmls.X_WEIGHTS, torch.float64, gmls.VEC_LAPLACIAN).numpy()
    assert w.size == x.shape[1] * 80 * 9 and np.all(np.isfinite(w))
    srv.release(t)
    srv.close()
