"""Convergence of the oracle's stencils at the rate m + 1 - |beta| (Sec. 2.5,
the bound quoted after Eq. polynomial-approximation-derivative) on smooth
manufactured fields: the 2D Stokes field u = (sin pi x cos pi y,
-cos pi x sin pi y), p = cos 2 pi x, and the paper's 3D trigonometric field
(Eq. manufactured-solution-sin).  RMS error over interior targets; the fitted
slope must be within 0.3 of the predicted rate."""
import numpy as np
import pytest

import oracle
from paper_2104_14447_gb300 import inputs

K2 = {("scalar", 2): 12, ("scalar", 4): 36, ("divfree", 2): 22, ("divfree", 4): 48}


@pytest.mark.parametrize("kind,m,name,beta", [
    ("scalar", 2, "grad", 1), ("scalar", 4, "grad", 1), ("scalar", 2, "laplacian", 2),
    ("scalar", 4, "laplacian", 2), ("divfree", 2, "vec_laplacian", 2), ("divfree", 4, "vec_laplacian", 2)])
def test_rates_2d(kind, m, name, beta):
    hs, errs = [], []
    for na in (32, 64, 128, 256):
        x = inputs.jittered_grid(2, na)
        f = inputs.manufactured_2d(x)
        inner = np.flatnonzero((np.abs(x[0] - 0.5) < 0.2) & (np.abs(x[1] - 0.5) < 0.2))
        tg = inner[:: max(1, len(inner) // 300)].astype(np.int32)
        k = K2[(kind, m)]
        idx, eps = oracle.knn(x, tg, k, 1.5, method="grid")
        off = np.arange(0, len(tg) * k + 1, k)
        w, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, kind, m, name)
        if kind == "scalar":
            got = np.einsum("trj,tj->tr", w[..., 0], f["p"][idx])
            want = f["grad_p"][:, tg].T if name == "grad" else f["lap_p"][tg][:, None]
        else:
            vals = np.stack([f["u"][0][idx], f["u"][1][idx]], axis=-1)
            got = np.einsum("trjc,tjc->tr", w, vals)
            want = f["lap_u"][:, tg].T
        hs.append(1.0 / na)
        errs.append(np.sqrt(np.mean((got - want) ** 2)))
    slope = np.polyfit(np.log2(hs), np.log2(errs), 1)[0]
    assert abs(slope - (m + 1 - beta)) <= 0.3, (slope, errs)


@pytest.mark.parametrize("kind,m,name,beta,k", [("scalar", 2, "grad", 1, 20), ("divfree", 2, "vec_laplacian", 2, 42)])
def test_rates_3d_paper_trig_field(kind, m, name, beta, k):
    hs, errs = [], []
    for na in (10, 20, 40):
        x = inputs.jittered_grid(3, na, seed=1) * 2.0 - 1.0  # bi-unit cube of Sec. 4
        X, Y, Z = x
        inner = np.flatnonzero(np.max(np.abs(x), axis=0) < 0.4)
        tg = inner[:: max(1, len(inner) // 200)].astype(np.int32)
        idx, eps = oracle.knn(x, tg, k, 1.5, method="grid")
        off = np.arange(0, len(tg) * k + 1, k)
        w, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, kind, m, name)
        if kind == "scalar":
            p = np.sin(X) * np.sin(Y) * np.sin(Z)
            got = np.einsum("trj,tj->tr", w[..., 0], p[idx])
            want = np.stack([np.cos(X) * np.sin(Y) * np.sin(Z), np.sin(X) * np.cos(Y) * np.sin(Z),
                             np.sin(X) * np.sin(Y) * np.cos(Z)])[:, tg].T
        else:
            v = np.stack([np.sin(Y) * np.sin(Z), np.sin(X) * np.sin(Z), np.sin(X) * np.sin(Y)])
            got = np.einsum("trjc,tjc->tr", w, np.stack([v[c][idx] for c in range(3)], axis=-1))
            want = (-2.0 * v)[:, tg].T
        hs.append(2.0 / na)
        errs.append(np.sqrt(np.mean((got - want) ** 2)))
    slope = np.polyfit(np.log2(hs), np.log2(errs), 1)[0]
    assert abs(slope - (m + 1 - beta)) <= 0.3, (slope, errs)
