"""The seeded synthetic inputs (paper_2104_14447_gb300/inputs.py) against
their stated recipes: the counter-based generator against the published
splitmix64 sequence, and each workload generator against the properties its
docstring promises (CPU only, small sizes)."""
import numpy as np

from paper_2104_14447_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    # seed 0, stream 0 give key 0, so the counters run the reference
    # generator from state 0 (Steele, Lea & Flood; Vigna's splitmix64.c)
    got = inputs.splitmix64(0, 0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_streams():
    u = inputs.uniform(3, 7, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    assert not np.array_equal(u[:100], inputs.uniform(3, 8, 100))  # streams differ
    assert np.array_equal(inputs.uniform(3, 7, 50, offset=10), u[10:60])  # counter-based


def test_jittered_grid_cells_and_order():
    n_axis = 17
    for dim in (2, 3):
        x = inputs.jittered_grid(dim, n_axis, seed=5)
        h = 1.0 / n_axis
        idx = np.arange(n_axis ** dim)
        for c in range(dim):
            i = (idx // n_axis ** c) % n_axis  # x fastest
            off = x[c] - (i + 0.5) * h
            assert np.all(np.abs(off) <= 0.25 * h + 1e-15)


def test_mixed_batch_recipe():
    for c in inputs.mixed_batch(20_000, seed=1):
        d, n = c["dim"], c["x"].shape[1]
        assert n == 20_000 and c["x"].shape[0] == d
        assert np.all((c["x"] >= 0.0) & (c["x"] <= 1.0))
        counts = np.bincount(c["degree"], minlength=5)[2:]
        assert counts.sum() == n and np.all(np.abs(counts / n - 1.0 / 3.0) < 0.02)
        frac = c["one_sided"].mean()
        assert abs(frac - 0.2) < 0.02
        lens = np.linalg.norm(c["halfspace"], axis=1)
        assert np.allclose(lens[c["one_sided"]], 1.0) and np.all(lens[~c["one_sided"]] == 0.0)


def test_porous_cube_recipe():
    pc = inputs.porous_cube(n_axis=24)
    x, bf, nr, sph = pc["x"], pc["bflag"], pc["normals"], pc["spheres"]
    assert sph.shape == (64, 4) and np.all((sph[:, 3] >= 0.05) & (sph[:, 3] <= 0.12))
    for a in range(len(sph)):  # non-overlapping
        d = np.linalg.norm(sph[a, :3] - sph[a + 1:, :3], axis=1)
        assert np.all(d > sph[a, 3] + sph[a + 1:, 3])
    for s in sph:  # no point inside a sphere (surface points lie on it)
        r = np.linalg.norm(x - s[:3, None], axis=0)
        assert np.all(r >= s[3] * (1.0 - 1e-12))
    lens = np.linalg.norm(nr, axis=0)
    assert np.allclose(lens[bf == 1], 1.0) and np.all(lens[bf == 0] == 0.0)
    assert 0.8 < pc["porosity"] < 0.9


def test_box_boundary_normals():
    bf, nr = inputs.box_boundary(2, 10)
    assert bf.sum() == 36  # the outermost layer of a 10 x 10 lattice
    lens = np.linalg.norm(nr, axis=0)
    assert np.allclose(lens[bf == 1], 1.0) and np.all(lens[bf == 0] == 0.0)
    assert np.allclose(nr[:, 0], -np.ones(2) / np.sqrt(2.0))  # corner (0, 0): outward diagonal


def test_request_stream_recipe():
    reqs = inputs.request_stream(4000, rate=200.0, seed=2)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0.0)
    assert abs(np.mean(np.diff(t)) - 1.0 / 200.0) < 0.0005
    n = np.array([r["n"] for r in reqs])
    assert n.min() >= 1000 and n.max() <= 500_000
    assert abs(np.mean(np.log(n)) - 0.5 * (np.log(1e3) + np.log(5e5))) < 0.1  # log-uniform
    assert {r["degree"] for r in reqs} == {2, 3, 4} and {r["dim"] for r in reqs} == {2, 3}
    assert {r["basis"] for r in reqs} == {"scalar", "divfree"}


def test_stokes_cubic_3d_fields():
    """The hand-derived cubic Stokes data against symbolic differentiation."""
    sympy = __import__("pytest").importorskip("sympy")
    X, Y, Z = sympy.symbols("x y z")
    V = (X, Y, Z)
    u = [Y ** 3 + Y * Z ** 2, X ** 2 * Z + Z ** 3, X * Y ** 2 - X ** 3]
    p = X ** 3 - 2 * X * Y * Z + 3 * Y ** 2 * Z - Z ** 3 + X * Y - 1

    def curl(a):
        return [sympy.diff(a[2], Y) - sympy.diff(a[1], Z), sympy.diff(a[0], Z) - sympy.diff(a[2], X),
                sympy.diff(a[1], X) - sympy.diff(a[0], Y)]

    assert sympy.expand(sum(sympy.diff(u[c], V[c]) for c in range(3))) == 0
    nu = 0.45
    cc = curl(curl(u))
    f = [nu * cc[c] + sympy.diff(p, V[c]) for c in range(3)]
    div_f = sum(sympy.diff(f[c], V[c]) for c in range(3))
    x = inputs.jittered_grid(3, 5, seed=3)
    d = inputs.stokes_cubic_3d(x, nu)
    ev = lambda e: np.asarray(sympy.lambdify(V, e, "numpy")(*x), dtype=np.float64) * np.ones(x.shape[1])
    for c in range(3):
        assert np.allclose(d["u"][c], ev(u[c]), rtol=0, atol=1e-13)
        assert np.allclose(d["curlcurl_u"][c], ev(cc[c]), rtol=0, atol=1e-13)
        assert np.allclose(d["f"][c], ev(f[c]), rtol=0, atol=1e-13)
    assert np.allclose(d["p"], ev(p), rtol=0, atol=1e-13)
    assert np.allclose(d["div_f"], ev(div_f), rtol=0, atol=1e-13)


def test_stokes_polynomial_3d_fields():
    """The hand-derived quadratic and quartic Stokes data against symbolic
    differentiation (divergence-free velocity, curl curl, f, div f)."""
    sympy = __import__("pytest").importorskip("sympy")
    X, Y, Z = sympy.symbols("x y z")
    V = (X, Y, Z)
    fields = {
        2: ([Y ** 2 + Y * Z, X ** 2 + Z ** 2, X * Y + X ** 2], X ** 2 - Y * Z + 2 * X * Z + Y - 1),
        4: ([Y ** 4 + Y ** 2 * Z ** 2 + Y * Z ** 3, X ** 3 * Z + Z ** 4 - X ** 2 * Z ** 2,
             X ** 2 * Y ** 2 + X * Y ** 3 - Y ** 4], X ** 4 - 2 * X ** 2 * Y * Z + Y ** 3 * Z + X * Z ** 2 - Y ** 2 + 1),
    }

    def curl(a):
        return [sympy.diff(a[2], Y) - sympy.diff(a[1], Z), sympy.diff(a[0], Z) - sympy.diff(a[2], X),
                sympy.diff(a[1], X) - sympy.diff(a[0], Y)]

    x = inputs.jittered_grid(3, 5, seed=4) * 2.0 - 1.0
    ev = lambda e: np.asarray(sympy.lambdify(V, e, "numpy")(*x), dtype=np.float64) * np.ones(x.shape[1])
    nu = 0.7
    for degree, (u, p) in fields.items():
        assert all(sympy.Poly(c, *V).total_degree() == degree for c in u) and sympy.Poly(p, *V).total_degree() == degree
        assert sympy.expand(sum(sympy.diff(u[c], V[c]) for c in range(3))) == 0
        cc = curl(curl(u))
        f = [nu * cc[c] + sympy.diff(p, V[c]) for c in range(3)]
        div_f = sum(sympy.diff(f[c], V[c]) for c in range(3))
        d = inputs.stokes_polynomial_3d(x, degree, nu)
        for c in range(3):
            assert np.allclose(d["u"][c], ev(u[c]), rtol=0, atol=1e-13)
            assert np.allclose(d["curlcurl_u"][c], ev(cc[c]), rtol=0, atol=1e-12)
            assert np.allclose(d["f"][c], ev(f[c]), rtol=0, atol=1e-12)
        assert np.allclose(d["p"], ev(p), rtol=0, atol=1e-13)
        assert np.allclose(d["div_f"], ev(div_f), rtol=0, atol=1e-12)


def test_stokes_trig_3d_fields():
    """The trigonometric Stokes data against symbolic differentiation."""
    sympy = __import__("pytest").importorskip("sympy")
    X, Y, Z = sympy.symbols("x y z")
    V = (X, Y, Z)
    u = [sympy.sin(Y) * sympy.sin(Z), sympy.sin(X) * sympy.sin(Z), sympy.sin(X) * sympy.sin(Y)]
    p = sympy.sin(X) * sympy.sin(Y) * sympy.sin(Z)

    def curl(a):
        return [sympy.diff(a[2], Y) - sympy.diff(a[1], Z), sympy.diff(a[0], Z) - sympy.diff(a[2], X),
                sympy.diff(a[1], X) - sympy.diff(a[0], Y)]

    assert sympy.simplify(sum(sympy.diff(u[c], V[c]) for c in range(3))) == 0
    nu = 1.3
    cc = curl(curl(u))
    f = [nu * cc[c] + sympy.diff(p, V[c]) for c in range(3)]
    div_f = sum(sympy.diff(f[c], V[c]) for c in range(3))
    x = inputs.jittered_grid(3, 5, seed=6) * 2.0 - 1.0
    ev = lambda e: np.asarray(sympy.lambdify(V, e, "numpy")(*x), dtype=np.float64) * np.ones(x.shape[1])
    d = inputs.stokes_trig_3d(x, nu)
    for c in range(3):
        assert np.allclose(d["u"][c], ev(u[c]), rtol=0, atol=1e-14)
        assert np.allclose(d["curlcurl_u"][c], ev(cc[c]), rtol=0, atol=1e-13)
        assert np.allclose(d["f"][c], ev(f[c]), rtol=0, atol=1e-13)
    assert np.allclose(d["p"], ev(p), rtol=0, atol=1e-14)
    assert np.allclose(d["div_f"], ev(div_f), rtol=0, atol=1e-13)
