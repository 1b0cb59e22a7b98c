"""gmls_knn_noalloc: neighbour lists for callers that cannot allocate device
memory where they need them (e.g. a solver inside a simulation code that
reserves all device memory at start-up).  Called through the C ABI with
torch-owned device buffers, it must return exactly what gmls_cloud +
gmls_neighbors return, on consecutive calls that share its static scratch
array (a smaller cloud after a larger one would expose any stale counter).

This file is collected last on purpose (test_zz_*): a stop at its failure
leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2104_14447_gb300 import gmls, inputs

pytestmark = pytest.mark.gpu


def _reference(ctx, x, k, f):
    cid = ctx.cloud(x)
    nid = ctx.neighbors(cid, k, f)
    idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32)
    eps = ctx.export(nid, gmls.X_NBR_EPS, torch.float64)
    st = ctx.export(nid, gmls.X_NBR_STATUS, torch.uint8)
    ctx.sync()
    ctx.release(nid)
    ctx.release(cid)
    return idx, eps, st


def test_noalloc_knn_matches_context_path_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2104_14447_gb300 import build

    build.build()
    lib = gmls.load()
    ctx = gmls.Context(0, arena_bytes=1 << 30)
    stream = torch.cuda.current_stream()
    cases = [(2, 512, 36, 1.5), (3, 24, 40, 1.5), (2, 40, 12, 1.8)]  # largest first, then smaller clouds
    for dim, n_axis, k, f in cases:
        x = torch.from_numpy(inputs.jittered_grid(dim, n_axis, seed=7)).cuda()
        n = x.shape[1]
        ref_idx, ref_eps, ref_st = _reference(ctx, x, k, f)
        for call in range(2):
            idx = torch.full((n * k,), -7, dtype=torch.int32, device="cuda")
            eps = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            rc = lib.gmls_knn_noalloc(dim, n, ctypes.c_void_p(x.data_ptr()), k, f, ctypes.c_void_p(idx.data_ptr()),
                                      ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
            assert rc == gmls.OK, lib.gmls_last_error(None)
            torch.cuda.synchronize()
            assert torch.equal(idx, ref_idx), (dim, n_axis, call)
            assert torch.equal(eps, ref_eps), (dim, n_axis, call)  # bit for bit
            assert torch.equal(st, ref_st)
    ctx.close()


def test_noalloc_rejects_clouds_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    lib = gmls.load()
    n = gmls.NOALLOC_MAX_POINTS + 1
    x = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    out = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    eps = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    rc = lib.gmls_knn_noalloc(2, n, ctypes.c_void_p(x.data_ptr()), 4, 1.5, ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(st.data_ptr()), None)
    assert rc == gmls.EINVAL
    assert b"at most 262144" in lib.gmls_last_error(None)


def test_noalloc_rejects_host_memory():
    """Coordinates or outputs that are not memory of the current device are
    an argument error, not a kernel fault."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    lib = gmls.load()
    x_host = torch.from_numpy(inputs.jittered_grid(2, 8, seed=1))
    n, k = x_host.shape[1], 4
    idx = torch.zeros(n * k, dtype=torch.int32, device="cuda")
    eps = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    rc = lib.gmls_knn_noalloc(2, n, ctypes.c_void_p(x_host.data_ptr()), k, 1.5, ctypes.c_void_p(idx.data_ptr()),
                              ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(st.data_ptr()), None)
    assert rc == gmls.EINVAL
    assert b"current device" in lib.gmls_last_error(None)
