"""CPU checks of two numerical methods the CUDA path relies on, restated here
in NumPy from their mathematical definitions (they are not oracle code and
share nothing with the kernels):

* the column solve of the diffusion preconditioner: for the constant-
  coefficient matrix T = c tridiag(-1, 2 + s, -1) with Dirichlet ends, the LU
  pivots u_i = (c/q) psi_{i+1}/psi_i (q + 1/q = 2 + s, psi_m = 1 - q^{2m})
  turn both substitutions into recursions with the constant multiplier q;
  it must equal a banded LU solve and the DST-I eigen-solve of the same matrix;
* the density's ln(e^x K_nu(x)) read from a table on the lattice 0.01 Z in
  u = ln x by 8-point Lagrange interpolation (nodes base .. base + 7 around u):
  within 1e-13 of scipy's kve over the x range the weights need.
"""
import numpy as np
import pytest
from scipy.fft import dst
from scipy.linalg import solve_banded
from scipy.special import kve


def scaled_lu_solve(s, c, b):
    """T x = b, T = c tridiag(-1, 2 + s, -1) on rows 1..N-1 (b = b_1..b_{N-1})."""
    n1 = len(b)
    N = n1 + 1
    th = 2.0 * np.arcsinh(np.sqrt(s) / 2.0)
    q = np.exp(-th)
    psi = -np.expm1(-2.0 * th * np.arange(N + 1))          # psi_m, m = 0..N
    bb = np.zeros(N + 1)
    bb[1:N] = b
    z = np.zeros(N + 1)
    for i in range(1, N):
        z[i] = psi[i] * bb[i] + q * z[i - 1]
    t = np.zeros(N + 1)
    for i in range(N - 1, 0, -1):
        t[i] = (q / c) * z[i] / (psi[i] * psi[i + 1]) + q * t[i + 1]
    return psi[1:N] * t[1:N]


def banded_solve(s, c, b):
    n = len(b)
    ab = np.zeros((3, n))
    ab[0, 1:] = -c
    ab[1] = c * (2.0 + s)
    ab[2, :-1] = -c
    return solve_banded((1, 1), ab, b)


@pytest.mark.parametrize("N", [8, 16, 64, 512])
@pytest.mark.parametrize("s,c", [(0.25, 3.9), (1.0 / 64.0, 64.0), (100.0, 0.01), (1e-6, 1000.0)])
def test_scaled_lu_column_solve_equals_banded_lu(N, s, c):
    rng = np.random.default_rng(N)
    b = rng.standard_normal(N - 1)
    x = scaled_lu_solve(s, c, b)
    ref = banded_solve(s, c, b)
    # backward stable: error of the order of the condition number times eps
    cond = (4.0 + s) / s
    assert np.abs(x - ref).max() <= 50 * cond * 2.2e-16 * np.abs(ref).max()


def test_scaled_lu_column_solve_equals_dst_eigen_solve():
    """The eigenvalues of tridiag(-1, 2, -1) with Dirichlet ends are
    4 sin^2(pi k / 2N), its eigenvectors the DST-I modes."""
    N, c, s = 64, 2.0, 0.65
    rng = np.random.default_rng(5)
    b = rng.standard_normal(N - 1)
    k = np.arange(1, N)
    lam = c * (s + 4.0 * np.sin(np.pi * k / (2 * N)) ** 2)
    x_dst = dst(dst(b, type=1) / lam, type=1) / (2 * N)
    assert np.abs(scaled_lu_solve(s, c, b) - x_dst).max() <= 1e-13 * np.abs(x_dst).max()


def lagrange8(tab, u0, du, u):
    f = (u - u0) / du
    base = int(np.floor(f)) - 3
    t = f - base
    val = 0.0
    for a in range(8):
        la = 1.0
        for b in range(8):
            if b != a:
                la *= (t - b) / (a - b)
        val += la * tab[base + a]
    return val


@pytest.mark.parametrize("nu", [1.0, 1.1, 1.25, 1.5, 1.75])
def test_log_bessel_table_interpolation(nu):
    du = 0.01
    lo, hi = np.log(1e-8), np.log(200.0)
    u0 = du * np.floor(lo / du - 5.0)
    n = int(np.ceil((hi - lo) / du)) + 14
    nodes = u0 + du * np.arange(n)
    tab = np.log(kve(nu, np.exp(nodes)))
    rng = np.random.default_rng(int(nu * 100))
    us = rng.uniform(lo, hi, 400)
    err = max(abs(lagrange8(tab, u0, du, u) - np.log(kve(nu, np.exp(u)))) for u in us)
    # scipy's kve is itself accurate to a few 1e-15 relative
    assert err <= 1e-13, err
