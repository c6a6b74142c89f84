"""Pins of the price-space oracle (the paper's own grid and operators,
Secs. 3-4): closed forms, exactness on polynomials, direct summation, and
Table 4, which the paper computed with this very discretisation."""
import math

import numpy as np
import pytest
from scipy import integrate

from conftest import paper_sets, read_table
from oracle.price_space import (PriceGrid, PriceScheme, PriceSpaceOperators, fd_matrices, lagrange_matrix,
                                put_avg_cell_integral, sinh_c)

# (name, x_max / K, z_max^III) of Sec. 4
SETS = {"VG1": (5.0, 2.1410), "NIG1": (7.0, 0.8807), "NIG0": (6.0, 0.4172), "VG0": (57.0, 11.5010)}


def test_sinh_grid_shape():
    """Uniform on [0, x_int] with step c * dxi, sinh-stretched beyond; the
    limit fraction of points in [0, x_int] is F = 0.65."""
    pg = PriceGrid(400, 100.0, 500.0, 2.141)
    x = pg.x
    assert x[0] == 0.0 and x[-1] == 500.0 and np.all(np.diff(x) > 0)
    h = np.diff(x)
    inner = x[1:] <= 250.0
    assert np.ptp(h[inner]) < 1e-9 * h[0]
    assert abs(inner.sum() / 400 - 0.65) < 2.0 / 400
    assert np.all(np.diff(h[~inner]) > 0)
    # F(c) of Sec. 4 solved for c: VG0's printed c (x_max = 57 K) is reproduced
    assert abs(sinh_c(250.0, 5700.0, 0.65) - 21.6164) < 2e-3 * 21.6164


def test_y_grids_cover_the_x_domain_and_in_is_7_smooth():
    pg = PriceGrid(40, 100.0, 500.0, 2.141)
    assert pg.y_out[0] <= pg.x[1] and pg.y_out[-1] >= pg.x[-1]
    n = pg.n_in
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    assert n == 1
    assert pg.y_in.size == pg.n_in


def test_put_cell_integral_closed_form():
    K = 100.0
    for (a1, b1, a2, b2) in [(95, 105, 92, 101), (0, 10, 190, 210), (-3, 3, 195, 199), (40, 60, 40, 60)]:
        # nested adaptive quadrature split at the kink x1 + x2 = 2K
        def inner(x1):
            k = 2 * K - x1
            pts = [k] if a2 < k < b2 else None
            return integrate.quad(lambda x2: max(K - 0.5 * (x1 + x2), 0.0), a2, b2, points=pts,
                                  epsabs=1e-13, epsrel=1e-13, limit=200)[0]
        brk = [v for v in (2 * K - b2, 2 * K - a2) if a1 < v < b1]
        ref = integrate.quad(inner, a1, b1, points=brk or None, epsabs=1e-12, epsrel=1e-13, limit=200)[0]
        assert abs(put_avg_cell_integral(K, a1, b1, a2, b2) - ref) < 1e-10 * max(1.0, abs(ref))


def test_lagrange_interpolation_exact_on_cubics_and_linear_extrapolation():
    pg = PriceGrid(64, 100.0, 500.0, 2.141)
    x = pg.x
    t = np.linspace(0.0, 500.0, 777)
    T = lagrange_matrix(x, t, "linear")
    p = lambda s: 2.0 - 0.3 * s + 1e-3 * s * s - 2e-6 * s ** 3
    assert np.max(np.abs(T @ p(x) - p(t))) < 1e-9 * np.max(np.abs(p(t)))
    te = np.array([-5.0, 520.0])
    Te = lagrange_matrix(x, te, "linear")
    lin = lambda s: 3.0 + 0.7 * s
    assert np.allclose(Te @ lin(x), lin(te), rtol=0, atol=1e-9)
    Tz = lagrange_matrix(x, np.array([600.0]), "zero")
    assert Tz.nnz == 0


def test_finite_differences_exact_on_quadratics_with_boundary_rows():
    pg = PriceGrid(50, 100.0, 600.0, 0.4172)
    x = pg.x
    D1, D2 = fd_matrices(x)
    q = 1.0 + 0.2 * x - 3e-4 * x * x
    inner = slice(1, -1)
    assert np.allclose((D1 @ q)[inner], (0.2 - 6e-4 * x)[inner], rtol=0, atol=1e-10)
    assert np.allclose((D2 @ q)[inner], -6e-4, rtol=0, atol=1e-10)
    assert (D1 @ q)[0] == 0.0 and (D2 @ q)[0] == 0.0 and (D2 @ q)[-1] == 0.0
    assert abs((D1 @ q)[-1] - (q[-1] - q[-2]) / (x[-1] - x[-2])) < 1e-12


def test_price_space_correlation_equals_direct_summation():
    """The circulant product of size #in (eq. 3.13) keeps exactly the direct
    cross-correlation sum (eq. 3.12) on y_out."""
    mo, _ = paper_sets()["VG1"]
    pg = PriceGrid(12, 100.0, 500.0, 2.141)
    ops = PriceSpaceOperators(mo, pg)
    rng = np.random.Generator(np.random.PCG64(4))
    V = rng.uniform(0, 50, size=(pg.x.size, pg.x.size))
    got = ops.jump(V)
    A = np.asarray(ops.Tin @ V @ ops.Tin.T)
    n_out = pg.ny_minus + pg.ny_plus + 1
    om = ops.pre.omega
    L = om.shape[0]
    By = np.zeros((n_out, n_out))
    for m2 in range(n_out):
        for m1 in range(n_out):
            By[m2, m1] = np.sum(om * A[m2:m2 + L, m1:m1 + L])
    ref = np.asarray(ops.Tout @ By @ ops.Tout.T)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["VG1", "NIG1"])
def test_table4_with_the_papers_discretisation(name):
    """Table 4 (N_x = 800 in the paper) approached from N_x = 40 and 80 with
    the paper's grid, operators and time stepping: the error shrinks and is
    below 0.04 at N_x = 80 at the three diagonal points."""
    mo, co = paper_sets()[name]
    xm, ziii = SETS[name]
    col = {"VG1": 1, "NIG1": 3}[name]
    table = {(float(r[0]), float(r[1])): float(r[2 + col]) for r in read_table("table4_prices.txt")}
    errs = []
    for n in (40, 80):
        pg = PriceGrid(n, co.strike, xm * co.strike, ziii)
        res = PriceScheme(mo, pg, co, n // 2, tol=1e-7).solve()
        errs.append(max(abs(res.price_at(a, a) - table[(a, a)]) for a in (90.0, 100.0, 110.0)))
    assert errs[1] < errs[0] and errs[1] < 0.04, errs


@pytest.mark.parametrize("name,xm,ziii,n", [("VG1", 5.0, 2.1410, 160), ("NIG1", 7.0, 0.8807, 80),
                                            ("VG0", 57.0, 11.5010, 40)])
def test_c_abi_sinh_grid_matches_oracle_grid(name, xm, ziii, n):
    """pide2d_price_sinh_grid (host code of the library, no GPU) builds the same
    Sec. 4 grid as the oracle's PriceGrid: nodes to 1e-12 relative, the same
    z-lattice, and the unpadded y_out range (the oracle pads #in to a 7-smooth
    length, the CUDA path's FFT length is a power of two)."""
    import math
    from paper_2511_02700_gb300 import binding as B
    from paper_2511_02700_gb300 import build
    build.build()
    K = 100.0
    pg = PriceGrid(n, K, xm * K, ziii)
    x, n_z, h_z, nym, nyp = B.price_sinh_grid(n, K, xm * K, ziii)
    assert np.max(np.abs(x - pg.x) / np.maximum(pg.x, 1.0)) <= 1e-12
    assert n_z == pg.n_z and h_z == pytest.approx(pg.h_z, rel=1e-15)
    assert nym == math.ceil(-math.log(pg.x[1]) / pg.h_z) and nyp == math.ceil(math.log(pg.x_max) / pg.h_z)
    assert pg.ny_minus - nym == pg.ny_plus - nyp >= 0
    with pytest.raises(B.PideError):
        B.price_sinh_grid(3, K, xm * K, ziii)
