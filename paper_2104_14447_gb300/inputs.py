"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no GMLS arithmetic: only point clouds, flags, normals,
degrees and request streams, all drawn from one counter-based generator
(splitmix64, Steele, Lea & Flood 2014) so that every value is a pure function
of (seed, stream, counter) and identical on every machine.

Workloads (the paper's own workloads are quasi-uniform particle lattices,
Sec. 4; no dataset is involved):

* ``jittered_grid``   -- lattice x = lo + (i + 1/2) h + U(-h/4, h/4) per coordinate.
* ``porous_cube``     -- 3D lattice in the unit cube minus random non-overlapping
                         spheres; near-surface points are projected onto the
                         spheres and flagged as boundary targets with the
                         fluid's outward normal; cube-face layers are flagged too.
* ``mixed_batch``     -- 2D and 3D lattices trimmed to a target count, per-target
                         degrees from {2, 3, 4} and a seeded fraction of
                         one-sided (half-space) targets with random unit normals.
* ``request_stream``  -- Poisson arrivals of stencil requests with log-uniform sizes.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """64-bit outputs for the given counters: mix(key + (counter + 1) * golden),
    key = mix(seed * 2^20 + stream)."""
    with np.errstate(over="ignore"):
        key = _mix(np.asarray([np.uint64((seed << 20) + stream)], dtype=np.uint64))[0]
        z = key + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
    return _mix(z)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): top 53 bits of splitmix64 times 2^-53."""
    r = splitmix64(seed, stream, np.arange(offset, offset + n, dtype=np.uint64))
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# stream ids (fixed so that every workload draws from its own sequence)
S_JITTER, S_SPHERE, S_DEGREE, S_HALFSPACE, S_HSNORMAL, S_REQUEST = 1, 2, 3, 4, 5, 6


def jittered_grid(dim: int, n_axis: int, h: float | None = None, jitter: float = 0.25, seed: int = 0,
                  lo: float = 0.0, stream: int = S_JITTER) -> np.ndarray:
    """(dim, n_axis**dim) SoA coordinates, x fastest; jitter U(-jitter h, jitter h)."""
    h = 1.0 / n_axis if h is None else h
    n = n_axis ** dim
    idx = np.arange(n, dtype=np.int64)
    x = np.empty((dim, n), dtype=np.float64)
    for c in range(dim):
        ic = (idx // (n_axis ** c)) % n_axis
        u = uniform(seed, stream, n, offset=c * n)
        x[c] = lo + (ic + 0.5) * h + (2.0 * u - 1.0) * (jitter * h)
    return x


def porous_cube(n_axis: int = 128, n_spheres: int = 64, rmin: float = 0.05, rmax: float = 0.12, seed: int = 0,
                max_tries: int = 100000):
    """3D porous medium: unit-cube jittered lattice minus random non-overlapping spheres.

    Returns dict with x (3, N), bflag uint8 (N), normals (3, N) (zero for interior
    points), spheres (S, 4) = (cx, cy, cz, r), porosity (fraction of the cube
    volume outside the spheres), lattice_points."""
    h = 1.0 / n_axis
    # random sequential addition: centres and radii from the sphere stream
    spheres = []
    ctr = 0
    while len(spheres) < n_spheres and ctr < max_tries:
        u = uniform(seed, S_SPHERE, 4, offset=4 * ctr)
        ctr += 1
        r = rmin + (rmax - rmin) * u[3]
        c = r + (1.0 - 2.0 * r) * u[:3]
        if all(np.sum((c - s[:3]) ** 2) > (r + s[3]) ** 2 for s in spheres):
            spheres.append(np.array([c[0], c[1], c[2], r]))
    spheres = np.array(spheres).reshape(-1, 4)
    x = jittered_grid(3, n_axis, h, 0.25, seed)
    n = x.shape[1]
    keep = np.ones(n, dtype=bool)
    bflag = np.zeros(n, dtype=np.uint8)
    normals = np.zeros((3, n), dtype=np.float64)
    for s in spheres:
        d = x - s[:3, None]
        r = np.sqrt(np.sum(d * d, axis=0))
        inside = r < s[3]
        keep &= ~inside
        near = (~inside) & (r < s[3] + 0.5 * h)
        # project onto the sphere; fluid outward normal points into the sphere
        if np.any(near):
            u = d[:, near] / r[near]
            x[:, near] = s[:3, None] + s[3] * u
            normals[:, near] = -u
            bflag[near] = 1
    # cube faces: outermost lattice layers
    idx = np.arange(n)
    for c in range(3):
        ic = (idx // (n_axis ** c)) % n_axis
        for layer, sgn in ((0, -1.0), (n_axis - 1, 1.0)):
            on = (ic == layer) & (bflag == 0)
            normals[c, on] = sgn
            bflag[on] = 1
    x, bflag, normals = x[:, keep], bflag[keep], normals[:, keep]
    porosity = 1.0 - float(np.sum(4.0 / 3.0 * np.pi * spheres[:, 3] ** 3))
    return {"x": np.ascontiguousarray(x), "bflag": bflag, "normals": np.ascontiguousarray(normals),
            "spheres": spheres, "porosity": porosity, "lattice_points": n}


def box_boundary(dim: int, n_axis: int):
    """Boundary flags and outward unit normals of a jittered_grid cloud on the
    unit box: the outermost lattice layer on each face (x fastest in the point
    order); corner and edge points get the normalised sum of their faces'
    normals.  Returns (bflag uint8 [N], normals [dim, N])."""
    n = n_axis ** dim
    idx = np.arange(n)
    nrm = np.zeros((dim, n))
    for c in range(dim):
        ic = (idx // (n_axis ** c)) % n_axis
        nrm[c, ic == 0] = -1.0
        nrm[c, ic == n_axis - 1] = 1.0
    length = np.sqrt(np.sum(nrm * nrm, axis=0))
    bflag = (length > 0).astype(np.uint8)
    nrm[:, length > 0] /= length[length > 0]
    return bflag, np.ascontiguousarray(nrm)


def stokes_manufactured_2d(x: np.ndarray, nu: float = 1.0):
    """Data of the 2D Stokes problem (Sec. 3.1) whose solution is the
    manufactured field u = (sin pi x cos pi y, -cos pi x sin pi y),
    p = cos 2 pi x: f = nu curl curl u + grad p (curl curl u = 2 pi^2 u),
    w = u on the boundary, div f = lap p."""
    m = manufactured_2d(x)
    curlcurl = -m["lap_u"]
    f = nu * curlcurl + m["grad_p"]
    return {"u": m["u"], "p": m["p"], "f": f, "w": m["u"], "div_f": m["lap_p"], "curlcurl_u": curlcurl}


def stokes_cubic_3d(x: np.ndarray, nu: float = 1.0):
    """Data of a 3D Stokes problem (Sec. 3.1) whose solution is a
    divergence-free cubic velocity and a cubic pressure (inside the degree-3
    bases, so degree-3 stencils reproduce it):
    u = (y^3 + y z^2, x^2 z + z^3, x y^2 - x^3) (no component depends on its
    own coordinate: div u = 0), curl curl u = -lap u = (-8 y, -8 z, 4 x),
    p = x^3 - 2 x y z + 3 y^2 z - z^3 + x y - 1, lap p = 6 x;
    f = nu curl curl u + grad p, w = u, div f = lap p."""
    X, Y, Z = (np.asarray(c, dtype=np.float64) for c in x[:3])
    u = np.stack([Y ** 3 + Y * Z ** 2, X ** 2 * Z + Z ** 3, X * Y ** 2 - X ** 3])
    cc = np.stack([-8.0 * Y, -8.0 * Z, 4.0 * X])
    p = X ** 3 - 2.0 * X * Y * Z + 3.0 * Y ** 2 * Z - Z ** 3 + X * Y - 1.0
    gp = np.stack([3.0 * X ** 2 - 2.0 * Y * Z + Y, -2.0 * X * Z + 6.0 * Y * Z + X, -2.0 * X * Y + 3.0 * Y ** 2 - 3.0 * Z ** 2])
    f = nu * cc + gp
    return {"u": u, "p": p, "f": f, "w": u, "div_f": 6.0 * X, "curlcurl_u": cc}


def stokes_polynomial_3d(x: np.ndarray, degree: int, nu: float = 1.0):
    """Data of a 3D Stokes problem (Sec. 3.1) whose solution is a
    divergence-free velocity and a pressure of the given degree (2 or 4;
    the polynomial tests of Sec. 4.1, which degree-2 or degree-4 bases
    reproduce exactly).  No velocity component depends on its own coordinate
    (div u = 0).  Degree 2:
      u = (y^2 + y z, x^2 + z^2, x y + x^2), lap u = (2, 4, 2),
      p = x^2 - y z + 2 x z + y - 1, lap p = 2;
    degree 4:
      u = (y^4 + y^2 z^2 + y z^3, x^3 z + z^4 - x^2 z^2, x^2 y^2 + x y^3 - y^4),
      lap u = (14 y^2 + 2 z^2 + 6 y z, 6 x z + 10 z^2 - 2 x^2, 2 x^2 - 10 y^2 + 6 x y),
      p = x^4 - 2 x^2 y z + y^3 z + x z^2 - y^2 + 1, lap p = 12 x^2 + 2 y z + 2 x - 2;
    curl curl u = -lap u, f = nu curl curl u + grad p, w = u, div f = lap p."""
    X, Y, Z = (np.asarray(c, dtype=np.float64) for c in x[:3])
    one = np.ones_like(X)
    if degree == 2:
        u = np.stack([Y ** 2 + Y * Z, X ** 2 + Z ** 2, X * Y + X ** 2])
        lap_u = np.stack([2.0 * one, 4.0 * one, 2.0 * one])
        p = X ** 2 - Y * Z + 2.0 * X * Z + Y - 1.0
        gp = np.stack([2.0 * X + 2.0 * Z, -Z + 1.0, -Y + 2.0 * X])
        lap_p = 2.0 * one
    elif degree == 4:
        u = np.stack([Y ** 4 + Y ** 2 * Z ** 2 + Y * Z ** 3, X ** 3 * Z + Z ** 4 - X ** 2 * Z ** 2,
                      X ** 2 * Y ** 2 + X * Y ** 3 - Y ** 4])
        lap_u = np.stack([14.0 * Y ** 2 + 2.0 * Z ** 2 + 6.0 * Y * Z, 6.0 * X * Z + 10.0 * Z ** 2 - 2.0 * X ** 2,
                          2.0 * X ** 2 - 10.0 * Y ** 2 + 6.0 * X * Y])
        p = X ** 4 - 2.0 * X ** 2 * Y * Z + Y ** 3 * Z + X * Z ** 2 - Y ** 2 + 1.0
        gp = np.stack([4.0 * X ** 3 - 4.0 * X * Y * Z + Z ** 2, -2.0 * X ** 2 * Z + 3.0 * Y ** 2 * Z - 2.0 * Y,
                       -2.0 * X ** 2 * Y + Y ** 3 + 2.0 * X * Z])
        lap_p = 12.0 * X ** 2 + 2.0 * Y * Z + 2.0 * X - 2.0
    else:
        raise ValueError("degree 2 or 4")
    cc = -lap_u
    f = nu * cc + gp
    return {"u": u, "p": p, "f": f, "w": u, "div_f": lap_p, "curlcurl_u": cc}


def stokes_trig_3d(x: np.ndarray, nu: float = 1.0):
    """Data of the 3D Stokes problem of the paper's convergence study
    (Sec. 4.1): u = (sin y sin z, sin x sin z, sin x sin y) (div u = 0,
    lap u = -2 u, curl curl u = 2 u), p = sin x sin y sin z (lap p = -3 p);
    f = nu curl curl u + grad p, w = u, div f = lap p."""
    X, Y, Z = (np.asarray(c, dtype=np.float64) for c in x[:3])
    sx, sy, sz, cx, cy, cz = np.sin(X), np.sin(Y), np.sin(Z), np.cos(X), np.cos(Y), np.cos(Z)
    u = np.stack([sy * sz, sx * sz, sx * sy])
    p = sx * sy * sz
    gp = np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz])
    cc = 2.0 * u
    return {"u": u, "p": p, "f": nu * cc + gp, "w": u, "div_f": -3.0 * p, "curlcurl_u": cc}


def unit_vectors(seed: int, stream: int, n: int, dim: int) -> np.ndarray:
    """n random unit vectors (dim, n) from normalised uniform cube samples."""
    out = np.zeros((dim, n), dtype=np.float64)
    u = uniform(seed, stream, n * dim).reshape(dim, n) * 2.0 - 1.0
    nrm = np.sqrt(np.sum(u * u, axis=0))
    nrm[nrm == 0.0] = 1.0
    out[:] = u / nrm
    return out


def mixed_batch(n_per_dim: int = 500_000, seed: int = 0, one_sided: float = 0.2):
    """Two clouds (2D 708^2 and 3D 80^3 lattices trimmed to n_per_dim points, in
    lattice order) with per-target degree U{2,3,4} and a one-sided fraction."""
    out = []
    for dim, axis, stream_off in ((2, 708, 0), (3, 80, 16)):
        while axis ** dim < n_per_dim:
            axis += 1
        x = jittered_grid(dim, axis, 1.0 / axis, 0.25, seed)[:, :n_per_dim]
        deg = 2 + np.floor(3.0 * uniform(seed, S_DEGREE + stream_off, n_per_dim)).astype(np.int8)
        hs_mask = uniform(seed, S_HALFSPACE + stream_off, n_per_dim) < one_sided
        nrm = unit_vectors(seed, S_HSNORMAL + stream_off, n_per_dim, dim)
        nrm[:, ~hs_mask] = 0.0
        out.append({"dim": dim, "x": np.ascontiguousarray(x), "degree": deg, "halfspace": np.ascontiguousarray(nrm.T),
                    "one_sided": hs_mask})
    return out


def request_stream(n_requests: int = 2000, rate: float = 200.0, seed: int = 0, nmin: float = 1e3, nmax: float = 5e5):
    """Poisson arrivals (exponential gaps) of stencil requests.  Each request:
    dim in {2, 3} (p = 1/2), n log-uniform in [nmin, nmax], degree U{2,3,4},
    basis scalar/divfree (p = 1/2)."""
    u = uniform(seed, S_REQUEST, 5 * n_requests).reshape(n_requests, 5)
    gaps = -np.log1p(-u[:, 0]) / rate
    t = np.cumsum(gaps)
    reqs = []
    for i in range(n_requests):
        dim = 2 if u[i, 1] < 0.5 else 3
        n = int(np.exp(np.log(nmin) + (np.log(nmax) - np.log(nmin)) * u[i, 2]))
        deg = 2 + int(np.floor(3.0 * u[i, 3]))
        kind = "scalar" if u[i, 4] < 0.5 else "divfree"
        reqs.append({"id": i, "t": float(t[i]), "dim": dim, "n": n, "degree": deg, "basis": kind, "seed": seed + 1 + i})
    return reqs


def manufactured_2d(x: np.ndarray):
    """Manufactured Stokes field on [0,1]^2: u = (sin pi x cos pi y, -cos pi x sin pi y),
    p = cos 2 pi x, with its exact vector Laplacian, pressure gradient and Laplacian."""
    X, Y = x[0], x[1]
    pi = np.pi
    u = np.stack([np.sin(pi * X) * np.cos(pi * Y), -np.cos(pi * X) * np.sin(pi * Y)])
    p = np.cos(2 * pi * X)
    return {"u": u, "p": p, "lap_u": -2 * pi ** 2 * u,
            "grad_p": np.stack([-2 * pi * np.sin(2 * pi * X), np.zeros_like(X)]),
            "lap_p": -4 * pi ** 2 * np.cos(2 * pi * X), "div_u": np.zeros_like(X)}
