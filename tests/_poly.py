"""Small polynomial helpers for the tests (independent of oracle and CUDA path).

A polynomial is a dict {(ax, ay, az): coef}.  Derivatives use the power rule.
"""
from __future__ import annotations

import numpy as np


def evaluate(poly, pts):
    """pts: (dim, n) array (dim <= 3)."""
    dim, n = pts.shape
    out = np.zeros(n)
    for a, c in poly.items():
        term = np.full(n, float(c))
        for k in range(dim):
            if a[k]:
                term = term * pts[k] ** a[k]
        out += term
    return out


def deriv(poly, k, times=1):
    out = {}
    for a, c in poly.items():
        if a[k] < times:
            continue
        f = 1
        for i in range(times):
            f *= a[k] - i
        b = list(a)
        b[k] -= times
        out[tuple(b)] = out.get(tuple(b), 0) + c * f
    return out


def add(*polys, scale=None):
    out = {}
    for i, p in enumerate(polys):
        s = 1 if scale is None else scale[i]
        for a, c in p.items():
            out[a] = out.get(a, 0) + s * c
    return out


def laplacian(poly, dim):
    return add(*[deriv(poly, k, 2) for k in range(dim)])


def random_poly(rng, dim, m):
    out = {}
    for s in range(m + 1):
        for az in range(s + 1 if dim == 3 else 1):
            for ay in range(s - az + 1 if dim >= 2 else 1):
                ax = s - ay - az
                out[(ax, ay, az)] = float(rng.uniform(-1, 1))
    return out


def parse_terms(text):
    poly = {}
    for term in text.split(","):
        term = term.strip()
        if not term:
            continue
        c, ax, ay, *az = term.split()
        key = (int(ax), int(ay), int(az[0]) if az else 0)
        poly[key] = poly.get(key, 0) + float(c)
    return poly
