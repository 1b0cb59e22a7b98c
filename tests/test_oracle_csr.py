"""Pin of the oracle's CSR assembly (Sec. 3.2: entries placed through the
local-to-global map J = LTG(I, j)) against scipy.sparse."""
import numpy as np
import scipy.sparse as sp

import oracle
from paper_2104_14447_gb300 import inputs


def test_csr_matches_scipy():
    x = inputs.jittered_grid(2, 12, seed=1)
    n = x.shape[1]
    tg = np.arange(n, dtype=np.int32)
    idx, eps = oracle.knn(x, tg, 22, 1.5)
    off = np.arange(0, n * 22 + 1, 22)
    w, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, "divfree", 2, "vec_laplacian")
    row_ptr, col, val, ncols = oracle.csr(off, idx.reshape(-1), w, n)
    rows, cols, vals = [], [], []
    for q in range(n):
        for r in range(2):
            for j in range(22):
                for c in range(2):
                    rows.append(q * 2 + r)
                    cols.append(idx[q, j] * 2 + c)
                    vals.append(w[q, r, j, c])
    ref = sp.coo_matrix((vals, (rows, cols)), shape=(2 * n, ncols)).tocsr()
    ref.sort_indices()
    assert np.array_equal(row_ptr, ref.indptr)
    assert np.array_equal(col, ref.indices)
    assert np.array_equal(val, ref.data)


def test_csr_fixed_k_fast_path_equals_general_path():
    x = inputs.jittered_grid(2, 10, seed=3)
    n = x.shape[1]
    tg = np.arange(n, dtype=np.int32)
    idx, eps = oracle.knn(x, tg, 12, 1.5)
    off = np.arange(0, n * 12 + 1, 12)
    w, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, "scalar", 2, "grad")
    a = oracle.csr(off, idx.reshape(-1), w, n)
    b = oracle.csr(off, idx.reshape(-1), list(w), n)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
