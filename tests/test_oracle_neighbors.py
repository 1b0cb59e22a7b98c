"""Pins of the oracle's neighbour search (Sec. 2.1: the particles within the
support of x_T) against brute force written independently in numpy/Python."""
import numpy as np
import pytest

import oracle
from paper_2104_14447_gb300 import inputs


def _np_knn(x, t, k, hs=None):
    """Reference kNN: exact squared distance ((dx*dx + dy*dy) + dz*dz) in numpy
    (element-wise, no fused multiply-add), order by (d2, index)."""
    dim, n = x.shape
    d = x - x[:, t:t + 1]
    d2 = d[0] * d[0]
    for c in range(1, dim):
        d2 = d2 + d[c] * d[c]
    ids = np.arange(n)
    if hs is not None and np.any(hs != 0):
        s = hs[0] * d[0]
        for c in range(1, dim):
            s = s + hs[c] * d[c]
        keep = s <= 0.0
        d2, ids = d2[keep], ids[keep]
    order = np.lexsort((ids, d2))
    return ids[order[:k]], d2[order[:k]]


@pytest.mark.parametrize("dim,n_axis,k", [(2, 24, 12), (2, 20, 48), (3, 9, 40), (3, 8, 80)])
def test_knn_brute_and_grid_match_numpy(dim, n_axis, k):
    x = inputs.jittered_grid(dim, n_axis, seed=3)
    n = x.shape[1]
    tg = np.arange(0, n, 7, dtype=np.int32)
    ib, eb = oracle.knn(x, tg, k, 1.5, method="brute")
    ig, eg = oracle.knn(x, tg, k, 1.5, method="grid")
    assert np.array_equal(ib, ig)
    assert np.array_equal(eb, eg)
    for q, t in enumerate(tg[:40]):
        ids, d2 = _np_knn(x, t, k)
        assert np.array_equal(ib[q], ids)
        assert eb[q] == 1.5 * np.sqrt(d2[-1])
        assert ib[q, 0] == t  # the target itself is neighbour 0 (d2 = 0)


def test_knn_ties_on_exact_lattice_break_by_index():
    # no jitter and a dyadic spacing (h = 1/8): coordinate differences are
    # exact, so many squared distances are exactly equal
    x = inputs.jittered_grid(2, 8, jitter=0.0)
    tg = np.arange(64, dtype=np.int32)
    ib, _ = oracle.knn(x, tg, 13, 1.5, method="brute")
    ig, _ = oracle.knn(x, tg, 13, 1.5, method="grid")
    assert np.array_equal(ib, ig)
    # pure-Python brute force on the interior point 36 (row 4, column 4)
    t = 36
    keyed = []
    for j in range(64):
        dx = x[0, j] - x[0, t]
        dy = x[1, j] - x[1, t]
        keyed.append((dx * dx + dy * dy, j))
    keyed.sort()
    assert list(ib[t]) == [j for _, j in keyed[:13]]
    # the four axis neighbours tie and come in index order
    assert list(ib[t, 1:5]) == [28, 35, 37, 44]


def test_knn_halfspace():
    x = inputs.jittered_grid(2, 24, seed=5)
    n = x.shape[1]
    # interior targets: every half-plane through them holds enough points
    inner = np.flatnonzero((np.abs(x[0] - 0.5) < 0.3) & (np.abs(x[1] - 0.5) < 0.3))
    tg = inner[::5].astype(np.int32)
    nrm = inputs.unit_vectors(7, 9, len(tg), 2).T.copy()
    nrm[::3] = 0.0  # every third target unfiltered
    ib, eb = oracle.knn(x, tg, 12, 1.5, halfspace=nrm, method="brute")
    ig, eg = oracle.knn(x, tg, 12, 1.5, halfspace=nrm, method="grid")
    assert np.array_equal(ib, ig) and np.array_equal(eb, eg)
    for q, t in enumerate(tg[:30]):
        ids, _ = _np_knn(x, t, 12, nrm[q])
        assert np.array_equal(ib[q], ids)


def test_radius_matches_numpy_and_cap():
    x = inputs.jittered_grid(3, 10, seed=2)
    n = x.shape[1]
    tg = np.arange(0, n, 13, dtype=np.int32)
    _, eps = oracle.knn(x, tg, 10, 1.8)
    cap = 40
    ob, ib = oracle.radius(x, tg, eps, cap, method="brute")
    og, ig = oracle.radius(x, tg, eps, cap, method="grid")
    assert np.array_equal(ob, og) and np.array_equal(ib, ig)
    for q, t in enumerate(tg):
        ids, d2 = _np_knn(x, t, n)
        inside = d2 < eps[q] * eps[q]
        want = ids[inside][:cap]
        assert np.array_equal(ib[ob[q]:ob[q + 1]], want)


def test_knn_too_few_is_an_error():
    x = inputs.jittered_grid(2, 6, seed=1)
    with pytest.raises(ValueError):
        oracle.knn(x, np.arange(4, dtype=np.int32), 37, 1.5)
