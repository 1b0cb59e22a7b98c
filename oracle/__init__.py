"""FP64 CPU oracle for GMLS stencil generation (arXiv 2104.14447, Sec. 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path.  The arithmetic lives in ``gmls_oracle.c`` (plain C, FP64,
``-ffp-contract=off``, OpenMP over targets); this module builds it, wraps it
with ctypes and adds the bookkeeping that is pure layout (CSR assembly, the
per-component divergence layout).

Pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against
textbook finite differences, a square (interpolatory) case solved by a library
routine, exact polynomial reproduction, the least-squares projection property,
an extended-precision normal-equation solve, an extended-precision KKT solve
for the Neumann variant, the paper's 2D divergence-free example and the
convergence rate m + 1 - |beta|.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import basis as _basis

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmls_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgmls_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _soa(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.ndim == 2, "coordinates are (dim, n) structure-of-arrays"
    return x


def set_threads(n: int) -> None:
    """Limit OpenMP threads (used for the single-core baseline)."""
    os.environ["OMP_NUM_THREADS"] = str(n)


# ---------------------------------------------------------------- neighbours
def knn(x, targets, k, eps_factor, halfspace=None, method="brute", cell_h=None, r0=None):
    """k nearest neighbours of each target, sorted by (d^2, index).

    Returns (idx int32 [n_tgt, k], eps float64 [n_tgt]) with
    eps = eps_factor * sqrt(d^2 of the k-th neighbour)."""
    x = _soa(x)
    dim, n = x.shape
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    hs = None if halfspace is None else np.ascontiguousarray(halfspace, dtype=np.float64).reshape(len(tg), dim)
    idx = np.empty((len(tg), k), dtype=np.int32)
    eps = np.empty(len(tg), dtype=np.float64)
    L = lib()
    if method == "brute":
        rc = L.orc_knn_brute(ctypes.c_int(dim), ctypes.c_int64(n), _p(x), ctypes.c_int64(len(tg)), _p(tg),
                             ctypes.c_int(k), ctypes.c_double(eps_factor), _p(hs), _p(idx), _p(eps))
    else:
        span = float(np.max(np.ptp(x, axis=1))) if n > 1 else 1.0
        h = cell_h if cell_h is not None else span / max(1.0, (n ** (1.0 / dim)))
        rr = r0 if r0 is not None else h * (k ** (1.0 / dim))
        rc = L.orc_knn_grid(ctypes.c_int(dim), ctypes.c_int64(n), _p(x), ctypes.c_int64(len(tg)), _p(tg),
                            ctypes.c_int(k), ctypes.c_double(eps_factor), _p(hs), ctypes.c_double(h),
                            ctypes.c_double(rr), _p(idx), _p(eps))
    if rc != 0:
        raise ValueError(f"oracle knn failed rc={rc} (too few neighbours?)")
    return idx, eps


def radius(x, targets, eps, cap, halfspace=None, method="brute", cell_h=None):
    """All neighbours with d^2 < eps^2, sorted by (d^2, index), at most cap.

    Returns (offsets int64 [n_tgt+1], idx int32 [nnz])."""
    x = _soa(x)
    dim, n = x.shape
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    ep = np.ascontiguousarray(eps, dtype=np.float64)
    hs = None if halfspace is None else np.ascontiguousarray(halfspace, dtype=np.float64).reshape(len(tg), dim)
    buf = np.empty((len(tg), cap), dtype=np.int32)
    cnt = np.empty(len(tg), dtype=np.int32)
    L = lib()
    if method == "brute":
        rc = L.orc_radius_brute(ctypes.c_int(dim), ctypes.c_int64(n), _p(x), ctypes.c_int64(len(tg)), _p(tg),
                                _p(ep), ctypes.c_int(cap), _p(hs), _p(buf), _p(cnt))
    else:
        h = cell_h if cell_h is not None else float(np.max(ep))
        rc = L.orc_radius_grid(ctypes.c_int(dim), ctypes.c_int64(n), _p(x), ctypes.c_int64(len(tg)), _p(tg),
                               _p(ep), ctypes.c_int(cap), _p(hs), ctypes.c_double(h), _p(buf), _p(cnt))
    if rc != 0:
        raise ValueError(f"oracle radius failed rc={rc}")
    off = np.zeros(len(tg) + 1, dtype=np.int64)
    off[1:] = np.cumsum(cnt)
    idx = np.concatenate([buf[q, : cnt[q]] for q in range(len(tg))]) if len(tg) else np.zeros(0, np.int32)
    return off, idx.astype(np.int32)


# ------------------------------------------------------------------ stencils
def make_basis(kind: str, dim: int, m: int):
    if kind == "scalar":
        return _basis.basis_table(_basis.taylor_basis(dim, m), 1)
    if kind == "divfree":
        return _basis.basis_table(_basis.divfree_basis(dim, m), dim)
    raise ValueError(kind)


def stencils(x, targets, nbr_off, nbr_idx, eps, kind, m, functional, wpow=4.0, bflag=None, normals=None,
             basis_table=None):
    """GMLS stencil weights for one functional on every target.

    Returns (w, beta, diag):
      w     list/array: target q -> array [rows, k_q, nc]  (stacked to
            [n_tgt, rows, k, nc] when all k_q are equal)
      beta  [n_tgt, rows]  Neumann coefficient of h (zero for interior targets)
      diag  [n_tgt, 2]     max |r_ii|, min |r_ii| of the triangular factor
    ``functional`` is a name of ``basis.functional_terms`` or a row list.
    For kind == 'scalar' and functional == 'div' the divergence of a vector
    field reconstructed component by component is returned (layout only:
    component c uses the d/dx_c weights)."""
    x = _soa(x)
    dim, n = x.shape
    if kind == "scalar" and functional == "div":
        g, beta, diag = stencils(x, targets, nbr_off, nbr_idx, eps, kind, m, "grad", wpow, bflag, normals,
                                 basis_table)
        return _div_from_grad(g, dim), beta[:, :1] * 0.0, diag
    nb, nc, b_off, b_coef, b_expo = basis_table if basis_table is not None else make_basis(kind, dim, m)
    rows = _basis.functional_terms(functional, dim) if isinstance(functional, str) else functional
    nrows, f_off, f_coef, f_comp, f_beta = _basis.functional_table(rows)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    off = np.ascontiguousarray(nbr_off, dtype=np.int64)
    idx = np.ascontiguousarray(nbr_idx, dtype=np.int32)
    ep = np.ascontiguousarray(eps, dtype=np.float64)
    nt = len(tg)
    ks = np.diff(off)
    w_off = np.zeros(nt + 1, dtype=np.int64)
    w_off[1:] = np.cumsum(ks * nc * nrows)
    out_w = np.zeros(int(w_off[-1]), dtype=np.float64)
    out_beta = np.zeros((nt, nrows), dtype=np.float64)
    out_diag = np.zeros((nt, 2), dtype=np.float64)
    bf = None if bflag is None else np.ascontiguousarray(bflag, dtype=np.uint8)
    nr = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64).reshape(nt, dim)
    if bf is not None and kind != "scalar":
        raise ValueError("the Neumann constraint applies to the scalar (pressure) basis")
    rc = lib().orc_stencils(
        ctypes.c_int(dim), ctypes.c_int64(n), _p(x), ctypes.c_int64(nt), _p(tg), _p(off), _p(idx), _p(ep),
        ctypes.c_double(wpow), ctypes.c_int(nb), ctypes.c_int(nc), _p(b_off), _p(b_coef), _p(b_expo),
        ctypes.c_int(nrows), _p(f_off), _p(f_coef), _p(f_comp), _p(f_beta), _p(bf), _p(nr), _p(w_off),
        _p(out_w), _p(out_beta), _p(out_diag))
    if rc != 0:
        raise ValueError(f"oracle stencils failed rc={rc}")
    ws = [out_w[w_off[q]:w_off[q + 1]].reshape(nrows, ks[q], nc) for q in range(nt)]
    if nt and np.all(ks == ks[0]):
        ws = np.stack(ws)
    return ws, out_beta, out_diag


def _div_from_grad(g, dim):
    if isinstance(g, np.ndarray):
        # g [T, dim, k, 1] -> [T, 1, k, dim]
        return np.ascontiguousarray(np.transpose(g[..., 0], (0, 2, 1))[:, None, :, :])
    return [np.ascontiguousarray(gq[..., 0].T[None, :, :]) for gq in g]


# ----------------------------------------------------------------------- CSR
def csr(nbr_off, nbr_idx, weights, n_cols_points):
    """CSR of one operator (Sec. 3.2, local-to-global map J = LTG(I, j)).

    weights: per target an array [rows, k, nc].  Operator row (q, r) is
    q*rows + r; its entries are (idx_j * nc + c, w[r, j, c]) sorted by column.
    Returns (row_ptr int64, col int32, val float64, n_cols)."""
    off = np.asarray(nbr_off, dtype=np.int64)
    idx = np.asarray(nbr_idx, dtype=np.int64)
    nt = len(off) - 1
    w0 = weights[0]
    rows, _, nc = w0.shape
    if isinstance(weights, np.ndarray) and nt:
        # every target has the same k: the same steps, vectorised over targets
        k = weights.shape[2]
        colq = (idx.reshape(nt, k)[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(nt, k * nc)
        order = np.argsort(colq, axis=1, kind="stable")
        cols = np.take_along_axis(colq, order, axis=1)
        vals = np.take_along_axis(weights.reshape(nt, rows, k * nc), order[:, None, :], axis=2)
        row_ptr = np.arange(nt * rows + 1, dtype=np.int64) * (k * nc)
        return (row_ptr, np.repeat(cols[:, None, :], rows, axis=1).reshape(-1).astype(np.int32),
                vals.reshape(-1).astype(np.float64), int(n_cols_points) * nc)
    row_ptr = [0]
    cols, vals = [], []
    for q in range(nt):
        nb = idx[off[q]:off[q + 1]]
        wq = weights[q]
        colq = (nb[:, None] * nc + np.arange(nc)[None, :]).reshape(-1)
        order = np.argsort(colq, kind="stable")
        for r in range(rows):
            cols.append(colq[order])
            vals.append(wq[r].reshape(-1)[order])
            row_ptr.append(row_ptr[-1] + len(colq))
    return (np.asarray(row_ptr, dtype=np.int64), np.concatenate(cols).astype(np.int32),
            np.concatenate(vals).astype(np.float64), int(n_cols_points) * nc)


def qr(A):
    """The oracle's Householder QR (column-major in/out) -- exposed for tests."""
    A = np.asfortranarray(np.array(A, dtype=np.float64))
    M, n = A.shape
    tau = np.zeros(n, dtype=np.float64)
    lib().orc_qr(ctypes.c_int(M), ctypes.c_int(n), _p(A), _p(tau))
    return A, tau


def apply_q(A, tau, z):
    A = np.asfortranarray(A)
    z = np.array(z, dtype=np.float64)
    M, n = A.shape
    lib().orc_apply_q(ctypes.c_int(M), ctypes.c_int(n), _p(A), _p(tau), _p(z))
    return z


# ------------------------------------------------------------ Stokes system
def stokes_system(dim, n, bflag, normals, vel, pres, nu, pres_int=None):
    """Collocation system of the Stokes problem (Sec. 3.2, Eq.
    stokes-block-system), assembled from per-point stencils.

    Unknowns: velocity v (point J, component c at J*dim + c), pressure phi
    (n*dim + J) and the zero-mean multiplier lambda (n*dim + n).
    Rows (Eqs. stokes-velocity-target .. stokes-pressure-neumann-target):
      I interior, component c: nu * (curl curl stencil) v + (gradient stencil) phi
      I boundary, component c: v_{I,c}                        (Dirichlet, delta rows)
      I interior, pressure:    (Laplacian stencil) phi + lambda
      I boundary, pressure:    -nu beta_I n_I . (curl curl stencil) v
                               + (Neumann-constrained Laplacian stencil) phi + lambda
      last row:                sum_J phi_J                    (zero mean)
    The boundary pressure row follows from the Neumann condition
    n . grad phi = n . f - nu n . curl curl v eliminated by the constrained
    stencil (Laplacian ~ sum w_j phi_j + beta h): the velocity coefficient is
    -nu beta n . (curl curl stencil); the right-hand side is
    div f - beta n . f.  n . a is evaluated as ((n_0 a_0) + (n_1 a_1)) + (n_2 a_2)
    and the coefficient as nu * (beta * (n . a)).

    vel  = (off, idx, w_cc) with w_cc[I] of shape [dim, k_I, dim] (curl curl
           rows, input components), targets = all points in order;
    pres = (off, idx, w_grad, w_lap, beta_lap) with w_grad[I] [dim, k_I, 1],
           w_lap[I] [1, k_I, 1] (constrained at boundary points) and
           beta_lap[I] the Laplacian row's beta (zero at interior points);
    pres_int = None, or (off, idx, w_lap) of staggered Laplacian stencils
           (Sec. 2.4, w_lap[I] [1, k_I, 1], the target in its own list):
           the interior pressure rows then take these weights on their own
           neighbour list, as Sec. 3.2 prescribes for points inside the
           domain (Eq. laplacian-pressure-stencil); boundary rows keep the
           Neumann-constrained scalar stencil.
    Returns scipy.sparse.csr_matrix with ascending columns in every row."""
    import scipy.sparse as sp

    off_v, idx_v, w_cc = vel
    off_p, idx_p, w_grad, w_lap, beta = pres
    nd = n * dim
    rows, cols, vals = [], [], []
    for I in range(n):
        jv = np.asarray(idx_v[off_v[I]:off_v[I + 1]], dtype=np.int64)
        jp = np.asarray(idx_p[off_p[I]:off_p[I + 1]], dtype=np.int64)
        a3 = np.asarray(w_cc[I])        # [dim, kv, dim]
        a1 = np.asarray(w_grad[I])[..., 0]  # [dim, kp]
        a2 = np.asarray(w_lap[I])[0, :, 0]  # [kp]
        vcol = (jv[:, None] * dim + np.arange(dim)[None, :]).reshape(-1)
        pcol = nd + jp
        if bflag[I]:
            for c in range(dim):
                rows.append(np.array([I * dim + c]))
                cols.append(np.array([I * dim + c]))
                vals.append(np.array([1.0]))
            nda = normals[0][I] * a3[0]
            for c in range(1, dim):
                nda = nda + normals[c][I] * a3[c]
            vv = nu * (beta[I] * nda)
            r = nd + I
            rows.append(np.full(len(vcol) + len(pcol) + 1, r))
            cols.append(np.concatenate([vcol, pcol, [nd + n]]))
            vals.append(np.concatenate([-vv.reshape(-1), a2, [1.0]]))
        else:
            for c in range(dim):
                r = I * dim + c
                rows.append(np.full(len(vcol) + len(pcol), r))
                cols.append(np.concatenate([vcol, pcol]))
                vals.append(np.concatenate([nu * a3[c].reshape(-1), a1[c]]))
            if pres_int is not None:
                off_s, idx_s, w_s = pres_int
                pcol = nd + np.asarray(idx_s[off_s[I]:off_s[I + 1]], dtype=np.int64)
                a2 = np.asarray(w_s[I])[0, :, 0]
            r = nd + I
            rows.append(np.full(len(pcol) + 1, r))
            cols.append(np.concatenate([pcol, [nd + n]]))
            vals.append(np.concatenate([a2, [1.0]]))
    rows.append(np.full(n, nd + n))
    cols.append(nd + np.arange(n))
    vals.append(np.ones(n))
    N = nd + n + 1
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
    A.sort_indices()
    return A


def stokes_rhs(dim, n, bflag, normals, f, w, div_f, beta_lap):
    """Right-hand side of the system of ``stokes_system``: f (interior
    momentum rows), w (Dirichlet rows), div f (interior pressure rows),
    div f - beta n . f (boundary pressure rows), 0 (zero-mean row)."""
    nd = n * dim
    b = np.zeros(nd + n + 1)
    bf = np.asarray(bflag).astype(bool)
    for c in range(dim):
        b[c:nd:dim] = np.where(bf, w[c], f[c])
    nf = normals[0] * f[0]
    for c in range(1, dim):
        nf = nf + normals[c] * f[c]
    b[nd:nd + n] = np.where(bf, div_f - beta_lap * nf, div_f)
    return b


# ---------------------------------------------------- staggered GMLS (Sec. 2.4)
def staggered_xi(dx, eps, dim, m, n_gauss=None):
    """Line integrals xi_i(x_j) = int_{x_T}^{x_j} phi_i(x) . dx (Eq. vector-xi)
    of the vector basis phi_(c, alpha) = e_c (x - x_T)^alpha / (alpha! eps^|alpha|),
    |alpha| <= m (a basis of pi_m^v), along the straight segment from the
    target, by Gauss-Legendre quadrature (exact for these polynomials).
    dx: [k, dim] offsets x_j - x_T.  Returns Xi [k, dim * C(m+dim, dim)],
    columns ordered (c, alpha) with c slowest."""
    alphas = _basis.graded_exponents(dim, m)
    ng = n_gauss or (m // 2 + 2)
    t, wq = np.polynomial.legendre.leggauss(ng)
    t, wq = 0.5 * (t + 1.0), 0.5 * wq  # on [0, 1]
    dx = np.asarray(dx, dtype=np.float64).reshape(-1, dim)
    cols = []
    for c in range(dim):
        for a in alphas:
            fact = 1.0
            for v in a[:dim]:
                for q in range(2, v + 1):
                    fact *= q
            val = np.zeros(dx.shape[0])
            for tq, wgt in zip(t, wq):
                pt = tq * dx / eps  # scaled offset of the point on the segment
                mono = np.ones(dx.shape[0])
                for k in range(dim):
                    mono = mono * pt[:, k] ** a[k]
                val = val + wgt * (mono / fact) * dx[:, c]
            cols.append(val)
    return np.stack(cols, axis=1)


def staggered_functional(dim, m, eps, name):
    """Rows of the target functional on the vector basis: 'laplacian' =
    div q_h(x_T) (Eq. staggered-laplacian-approximation): div phi_(c, alpha)(x_T)
    = 1/eps for alpha = e_c, else 0; 'grad' = q_h(x_T): component c' of
    phi_(c, alpha)(x_T) = 1 for c = c', alpha = 0."""
    alphas = _basis.graded_exponents(dim, m)
    nq = dim * len(alphas)
    if name == "laplacian":
        lam = np.zeros((1, nq))
        for c in range(dim):
            lam[0, c * len(alphas) + alphas.index(_e3(c))] = 1.0 / eps
        return lam
    if name == "grad":
        lam = np.zeros((dim, nq))
        for c in range(dim):
            lam[c, c * len(alphas) + 0] = 1.0
        return lam
    raise ValueError(name)


def _e3(k):
    b = [0, 0, 0]
    b[k] = 1
    return tuple(b)


def staggered_stencils(x, targets, nbr_off, nbr_idx, eps, m, functional, wpow=4.0):
    """Staggered GMLS stencils (Sec. 2.4) on point values p.

    Per target: rho_j = p_j - p(x_T) (Eq. vector-rho), the weighted least
    squares of Eq. staggered-matrix-vector-multiplication over the line
    integrals Xi, c = (Xi^T W Xi)^+ Xi^T W rho (Eq. staggered-vector-c; the
    pseudo-inverse, because the line integrals of a basis of pi_m^v are
    linearly dependent: e.g. e_x xi_y and e_y xi_x integrate to the same
    xi_x xi_y / 2), and the functional row lambda gives weights on rho,
    w_rho = W Xi (Xi^T W Xi)^+ lambda^T.  On p: w_j for every neighbour j but
    the target itself, and -sum_j w_j for the target's own entry.
    Returns [n_tgt, rows, k, 1] (all k equal) and the ranks of Xi."""
    x = _soa(x)
    dim, n = x.shape
    off = np.asarray(nbr_off, dtype=np.int64)
    idx = np.asarray(nbr_idx, dtype=np.int64)
    out, ranks = [], []
    for q, t in enumerate(np.asarray(targets, dtype=np.int64)):
        nb = idx[off[q]:off[q + 1]]
        dx = (x[:, nb] - x[:, t:t + 1]).T
        r = np.sqrt(np.sum(dx * dx, axis=1))
        e = float(eps[q])
        W = np.where(r < e, (1.0 - r / e), 0.0) ** wpow
        Xi = staggered_xi(dx, e, dim, m)
        lam = staggered_functional(dim, m, e, functional)
        B = np.sqrt(W)[:, None] * Xi
        Bp = np.linalg.pinv(B, rcond=1e-11)
        ranks.append(np.linalg.matrix_rank(B, tol=1e-11 * np.linalg.norm(B, 2)))
        w_rho = (np.sqrt(W)[:, None] * (Bp.T @ lam.T)).T  # [rows, k]
        self_pos = np.flatnonzero(nb == t)
        if len(self_pos) != 1:
            raise ValueError("the target must appear once in its own neighbour list")
        w = w_rho.copy()
        w[:, self_pos[0]] = 0.0
        w[:, self_pos[0]] = -np.sum(w, axis=1)
        out.append(w[:, :, None])
    return np.stack(out), np.asarray(ranks)


def stokes_solve(A, b):
    """Solution of the collocation system (Sec. 3.2) by a sparse direct
    factorisation (SuperLU through scipy): the reference for the GPU's
    iterative solve."""
    import scipy.sparse.linalg as spla

    return spla.spsolve(A.tocsc(), b)
