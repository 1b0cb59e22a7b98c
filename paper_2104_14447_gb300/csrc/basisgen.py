"""Generate ``basis_tables.cuh``: straight-line device code for the GMLS bases.

Run ``python basisgen.py`` (the build does this when the header is missing or
older than this script).  Exact rational arithmetic throughout.

Bases are written in the normalised scaled monomials of the paper's Taylor
basis (Eq. basis-functions-3d), p_g(xi) = xi^g / g!, xi = (x - x_T)/eps:

* scalar: p_g for all |g| <= m  (span pi_m(R^d), Sec. 2.1);
* staggered (Sec. 2.4): p_g for 1 <= |g| <= m+1.  The line integrals
  int_{x_T}^{x_j} phi . dx of the vector monomials phi = e_c p_a (|a| <= m,
  the paper's basis of pi_m^v) are eps xi_c xi^a / (a! (|a| + 1)): monomials
  of degree 1..m+1, so their span has this basis (the paper's d C(m+d, d)
  columns are linearly dependent).  On it the staggered Laplacian
  div q_h(x_T) is the Laplacian at 0 and q_h(x_T) the gradient at 0, and the
  least squares fits the differences p_j - p(x_T);
* divergence-free: a basis of pi^div_m(R^d) (Sec. 2.2) obtained as the
  reduced-row-echelon null space of the divergence map on (pi_m)^d.  With
  this normalisation d/dxi_k p_g = p_{g - e_k}, so the coefficient of p_q in
  div(sum a_{c,g} p_g e_c) is sum_c a_{c, q + e_c}: a 0/1 matrix whose null
  space has small integer entries.

Target functionals at x_T (Sec. 2.5) follow from p_g(0) = [g = 0] and the
shift rule: grad_k picks p_{e_k}, the Laplacian sums p_{2 e_k}; both scale
with eps^{-|beta|} at run time.  On the divergence-free basis the vector
Laplacian row c is sum_k a_{c, 2 e_k}, curl curl is its negative (Sec. 3.1
vector identity with div = 0), and the divergence row is identically zero.
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction
from math import comb

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "basis_tables.cuh")
DIMS = (2, 3)
KID = {"scalar": 0, "divfree": 1, "staggered": 2}  # basis codes of the C ABI
DEGREES = (1, 2, 3, 4)


def monomials(d: int, m: int):
    """Exponents with |g| <= m, degree ascending; within a degree g_x
    descends.  The linear monomials are entries 1..d (used by the Neumann
    elimination)."""
    out = []
    for s in range(m + 1):
        if d == 2:
            for gx in range(s, -1, -1):
                out.append((gx, s - gx, 0))
        else:
            for gx in range(s, -1, -1):
                for gy in range(s - gx, -1, -1):
                    out.append((gx, gy, s - gx - gy))
    assert len(out) == comb(m + d, d)
    return out


def rref_nullspace(rows, ncols):
    """Null-space basis of a rational matrix given as a list of dict rows."""
    mat = [[Fraction(r.get(c, 0)) for c in range(ncols)] for r in rows]
    pivots = []
    r = 0
    for c in range(ncols):
        p = next((i for i in range(r, len(mat)) if mat[i][c] != 0), None)
        if p is None:
            continue
        mat[r], mat[p] = mat[p], mat[r]
        inv = 1 / mat[r][c]
        mat[r] = [v * inv for v in mat[r]]
        for i in range(len(mat)):
            if i != r and mat[i][c] != 0:
                f = mat[i][c]
                mat[i] = [a - f * b for a, b in zip(mat[i], mat[r])]
        pivots.append(c)
        r += 1
        if r == len(mat):
            break
    free = [c for c in range(ncols) if c not in pivots]
    basis = []
    for fcol in free:
        v = [Fraction(0)] * ncols
        v[fcol] = Fraction(1)
        for i, pc in enumerate(pivots):
            v[pc] = -mat[i][fcol]
        basis.append(v)
    return basis


def divfree(d: int, m: int):
    mons = monomials(d, m)
    index = {g: i for i, g in enumerate(mons)}
    nm = len(mons)
    # unknowns a_{c,g} at column c*nm + index[g]; one constraint per q, |q| <= m-1
    rows = []
    for q in monomials(d, m - 1) if m >= 1 else []:
        row = {}
        for c in range(d):
            g = list(q)
            g[c] += 1
            row[c * nm + index[tuple(g)]] = 1
        rows.append(row)
    # an all-zero constraint set (m = 0) leaves every constant field
    ns = rref_nullspace(rows, d * nm) if rows else [
        [Fraction(int(i == j)) for i in range(d * nm)] for j in range(d * nm)]
    want = (m + 1) * (m + 4) // 2 if d == 2 else 3 * comb(m + 3, 3) - comb(m + 2, 3)
    assert len(ns) == want, (d, m, len(ns), want)
    funcs = []
    for v in ns:
        terms = [(c, i, v[c * nm + i]) for c in range(d) for i in range(nm) if v[c * nm + i] != 0]
        funcs.append(terms)
    # sanity: exact zero divergence
    for terms in funcs:
        div = {}
        for c, i, a in terms:
            g = mons[i]
            if g[c] == 0:
                continue
            h = list(g)
            h[c] -= 1
            div[tuple(h)] = div.get(tuple(h), 0) + a
        assert all(val == 0 for val in div.values())
    return mons, funcs


def cnum(fr: Fraction) -> str:
    if fr.denominator == 1:
        return f"{fr.numerator}.0"
    return f"({fr.numerator}.0/{fr.denominator}.0)"


def f32_split(fr: Fraction):
    """float-float split (h, l) of a rational: h = fl32(v), l = fl32(v - h)."""
    import numpy as np
    v = fr.numerator / fr.denominator
    h = np.float32(v)
    lo = np.float32(v - float(h))
    return float(h), float(lo)


def cconst(fr: Fraction) -> str:
    """A constant of type T: exact value for double, float-float split for ff."""
    h, lo = f32_split(fr)
    return f"gmls_cst(T(), {cnum(fr)}, {h.hex()}f, {lo.hex()}f)"


def emit_monomials(d, m, lines, ind):
    """px{a} = xi_x^a / a! etc. (no factor for a = 0)."""
    names = "xyz"
    for k in range(d):
        for a in range(1, m + 1):
            if a == 1:
                lines.append(f"{ind}const T p{names[k]}1 = xi[{k}];")
            elif a & (a - 1) == 0:  # 1/a is a power of two: exact scaling
                lines.append(f"{ind}const T p{names[k]}{a} = gmls_scale2(p{names[k]}{a - 1} * xi[{k}], {1.0 / a!r}f);")
            else:
                lines.append(f"{ind}const T p{names[k]}{a} = (p{names[k]}{a - 1} * xi[{k}]) * {cconst(Fraction(1, a))};")


def emit_scaled_products(d, mons, used, lines, ind):
    """q{i} = s * prod_k p{k}{g_k} for the used monomials, built axis by axis
    from memoised partial products s * px_a, s * px_a * py_b, ... so that every
    monomial costs at most one product beyond its prefix."""
    names = "xyz"
    made = {}

    def partial(g, k):  # name of s * prod_{j <= k} p{j}{g_j}
        key = tuple(g[:k + 1])
        if key in made:
            return made[key]
        if k < 0:
            return "s"
        prev = partial(g, k - 1) if k > 0 else "s"
        if g[k] == 0:
            made[key] = prev
            return prev
        nm = "t" + "_".join(str(e) for e in key)
        lines.append(f"{ind}const T {nm} = {prev} * p{names[k]}{g[k]};")
        made[key] = nm
        return nm

    for i, g in enumerate(mons):
        if i in used:
            lines.append(f"{ind}const T q{i} = {partial(g, d - 1)};")


def gen():
    L = []
    L.append("// Generated by basisgen.py -- do not edit.  Bases for GMLS stencils on the")
    L.append("// GPU (scaled Taylor monomials; divergence-free null-space basis).")
    L.append("#pragma once")
    L.append("namespace gmls_gen {")
    L.append("")
    L.append("// constants and exact power-of-two scalings for T = double; the float-float")
    L.append("// type provides its own overloads (found by argument-dependent lookup)")
    L.append("__device__ __forceinline__ double gmls_cst(double, double c, float, float) { return c; }")
    L.append("__device__ __forceinline__ double gmls_scale2(double x, float p) { return x * (double)p; }")
    L.append("")
    summary = []
    for kind in ("scalar", "divfree", "staggered"):
        for d in DIMS:
            for m in DEGREES:
                if kind == "scalar":
                    mons = monomials(d, m)
                    nb, nc = len(mons), 1
                    funcs = [[(0, i, Fraction(1))] for i in range(nb)]
                elif kind == "staggered":
                    mons = monomials(d, m + 1)
                    funcs = [[(0, i, Fraction(1))] for i in range(1, len(mons))]  # no constant
                    nb, nc = len(funcs), 1
                else:
                    mons, funcs = divfree(d, m)
                    nb, nc = len(funcs), d
                name = f"{kind}_{d}d_m{m}"
                nterms = sum(len(f) for f in funcs)
                summary.append((kind, d, m, nb, nc, nterms))
                L.append(f"// {name}: {nb} functions, {nc} component(s), {nterms} terms")
                L.append(f"// out[i * ld + c] = s * psi_i,c(xi)")
                L.append("template <typename T, typename O = T*>")
                L.append(f"__device__ __forceinline__ void eval_{name}(const T* xi, O out, int ld, const T s) {{")
                ind = "  "
                emit_monomials(d, m + 1 if kind == "staggered" else m, L, ind)
                used = {mi for f in funcs for (_, mi, _) in f}
                emit_scaled_products(d, mons, used, L, ind)
                # out[i*ld + c] = sum terms
                for i, f in enumerate(funcs):
                    for c in range(nc):
                        ts = [(mi, a) for (cc, mi, a) in f if cc == c]
                        if not ts:
                            L.append(f"{ind}out[{i} * ld + {c}] = gmls_cst(T(), 0.0, 0.0f, 0.0f);")
                            continue
                        expr = " + ".join(
                            (f"q{mi}" if a == 1 else f"-q{mi}" if a == -1 else f"{cconst(a)} * q{mi}") for mi, a in ts)
                        L.append(f"{ind}out[{i} * ld + {c}] = {expr};")
                L.append("}")
                # functional rows (coefficients before the eps^{-|beta|} factor)
                if kind in ("scalar", "staggered"):
                    bm = mons if kind == "scalar" else mons[1:]  # the basis' monomials, in column order
                    grad = [[1 if g == tuple(int(j == k) for j in range(3)) else 0 for g in bm] for k in range(d)]
                    lap = [[1 if (sum(g) == 2 and max(g) == 2) else 0 for g in bm]]
                    L.append(f"__device__ constexpr float lam_grad_{name}[{d}][{nb}] = {{" + ", ".join(
                        "{" + ", ".join(f"{v}.0" for v in row) + "}" for row in grad) + "};")
                    L.append(f"__device__ constexpr float lam_lap_{name}[1][{nb}] = {{" + ", ".join(
                        "{" + ", ".join(f"{v}.0" for v in row) + "}" for row in lap) + "};")
                else:
                    idx2 = [mons.index(e) for e in (tuple(2 * int(j == k) for j in range(3)) for k in range(d)) if e in mons]
                    vlap = []
                    for c in range(d):
                        row = []
                        for f in funcs:
                            s = sum((a for (cc, mi, a) in f if cc == c and mi in idx2), Fraction(0))
                            row.append(s)
                        vlap.append(row)
                    assert all(v.denominator == 1 and abs(v.numerator) < 2 ** 24 for row in vlap for v in row)
                    L.append(f"__device__ constexpr float lam_vlap_{name}[{d}][{nb}] = {{" + ", ".join(
                        "{" + ", ".join(cnum(v) for v in row) + "}" for row in vlap) + "};")
                L.append("")
    L.append("}  // namespace gmls_gen")
    L.append("")
    # dispatch helpers
    L.append("namespace gmls_gen {")
    L.append("// basis size for (kind, d, m); 0 when unsupported")
    L.append("__host__ __device__ constexpr int basis_size(int kind, int d, int m) {")
    L.append("  return")
    for kind, d, m, nb, nc, _ in summary:
        L.append(f"    (kind == {KID[kind]} && d == {d} && m == {m}) ? {nb} :")
    L.append("    0;")
    L.append("}")
    L.append("// O: the output (T* or any type whose operator[] returns an assignable element)")
    L.append("template <typename T, typename O = T*>")
    L.append("__device__ __forceinline__ void eval_basis(int kind, int d, int m, const T* xi, O out, int ld, const T s) {")
    L.append("  switch (kind * 100 + d * 10 + m) {")
    for kind, d, m, nb, nc, _ in summary:
        name = f"{kind}_{d}d_m{m}"
        L.append(f"    case {KID[kind] * 100 + d * 10 + m}: eval_{name}<T, O>(xi, out, ld, s); break;")
    L.append("    default: break;")
    L.append("  }")
    L.append("}")
    L.append("// compile-time dispatch: BasisEval<kind, d, m>::run<T>(xi, out, ld)")
    L.append("template <int KIND, int D, int M> struct BasisEval;")
    for kind, d, m, nb, nc, _ in summary:
        name = f"{kind}_{d}d_m{m}"
        kid = KID[kind]
        L.append(f"template <> struct BasisEval<{kid}, {d}, {m}> {{")
        L.append("  template <typename T, typename O = T*>")
        L.append(f"  __device__ __forceinline__ static void run(const T* xi, O out, int ld, const T s) {{ eval_{name}<T, O>(xi, out, ld, s); }}")
        L.append("};")
    L.append("// functional row coefficient (before the eps^{-|beta|} factor)")
    L.append("// fn: 0 grad (d rows), 1 laplacian (1 row), 2 vector Laplacian (d rows),")
    L.append("//     3 curl curl (d rows), 4 divergence of a div-free field (1 row, zero)")
    L.append("__device__ __forceinline__ float lam_coef_raw(int kind, int d, int m, int fn, int row, int i) {")
    L.append("  switch (kind * 100 + d * 10 + m) {")
    for kind, d, m, nb, nc, _ in summary:
        name = f"{kind}_{d}d_m{m}"
        key = KID[kind] * 100 + d * 10 + m
        if kind in ("scalar", "staggered"):
            L.append(f"    case {key}: return fn == 0 ? lam_grad_{name}[row][i] : fn == 1 ? lam_lap_{name}[0][i] : 0.0f;")
        else:
            L.append(f"    case {key}: return fn == 2 ? lam_vlap_{name}[row][i] : fn == 3 ? -lam_vlap_{name}[row][i] : 0.0f;")
    L.append("    default: return 0.0f;")
    L.append("  }")
    L.append("}")
    L.append("// every coefficient is a small integer: exact in FP32 and in FP64")
    L.append("__device__ __forceinline__ float lam_coef_f(int kind, int d, int m, int fn, int row, int i) {")
    L.append("  return lam_coef_raw(kind, d, m, fn, row, i);")
    L.append("}")
    L.append("__device__ __forceinline__ double lam_coef(int kind, int d, int m, int fn, int row, int i) {")
    L.append("  return (double)lam_coef_raw(kind, d, m, fn, row, i);")
    L.append("}")
    L.append("}  // namespace gmls_gen")
    return "\n".join(L) + "\n", summary


def main():
    text, summary = gen()
    with open(OUT, "w") as fh:
        fh.write(text)
    for row in summary:
        print(*row)


if __name__ == "__main__":
    sys.exit(main())
