"""The paper's own discretisation in price space (Sec. 3-4): a plain FP64 CPU
restatement, used as the oracle of the price-space jump operator and to
reproduce Table 4 with the paper's grid.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* x-grid      x_m = phi(phi^-1(0) + m (phi^-1(x_max) - phi^-1(0)) / N_x), m = 0..N_x,
              phi(xi) = c xi on [0, xi_int], x_int + c sinh(xi - xi_int) beyond
              (Sec. 4); c from the fraction F = max(0.65, x_int / x_max) of
              points in [0, x_int], x_int = 5K/2.
* z-grid      N_z = 2 N_x, h_z = z_III / N_z; weights, R_I moment and rates as
              in the log-grid oracle (eqs. 3.3, 3.5, 3.6).
* y-grids     y_out_m = e^{m h_z}, m = -N_y^- .. N_y^+;
              y_in_m = e^{(m + 1/2) h_z}, m = -N_z - N_y^- .. N_z + N_y^+ - 1;
              N_y^- = ceil(-ln(x_1)/h_z) + N_y*, N_y^+ = ceil(ln(x_max)/h_z) + N_y*,
              N_y* the least integer making #in = N_y^- + N_y^+ + 2 N_z 7-smooth.
* B_w V       T_out I~ C T_in V (eqs. 3.12-3.17): cubic Lagrange in price from
              the x-grid to y_in (v = 0 outside R_x), the cross-correlation with
              Omega on the y-lattice, cubic Lagrange from y_out back to the
              x-grid, linear extrapolation where x lies below y_out.
* D           second-order central differences on the non-uniform grid with
              the x^2 / x x factors of the price-space diffusion (Sec. 3.2.1);
              the rows at x = 0 vanish, at x_max the second difference is zero
              and the first difference one-sided (backward).
* SL          departure points x e^{kappa_w h_t} (Sec. 3.3), cubic Lagrange on
              the x-grid, linear extrapolation beyond x_max.
* time loop   eq. 3.23 with theta = 1/2, the first step damped (four theta = 1
              steps of h_t/4), fixed-point iteration (3.24)-(3.25) from the
              extrapolated start (3.26); each implicit solve is exact (sparse LU)
              where the paper uses BiCGSTAB + ILU to 1e-14.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.optimize import brentq

from .levy import NTSModel
from .scheme import Contract, Grid, precompute

# --------------------------------------------------------------------------
# grids (Sec. 4)
# --------------------------------------------------------------------------


def sinh_c(x_int: float, x_max: float, frac: float) -> float:
    """c such that xi_int / xi_max = frac (Sec. 4: F = (1 + c/x_int asinh((x_max - x_int)/c))^-1)."""
    def F(c):
        return 1.0 / (1.0 + c / x_int * math.asinh((x_max - x_int) / c)) - frac
    return brentq(F, 1e-6 * x_int, 1e6 * x_max, xtol=1e-14, rtol=1e-15, maxiter=500)


@dataclass
class PriceGrid:
    n: int                 # N_x
    strike: float
    x_max: float
    z_iii: float           # z_max^III
    frac: float = 0.65
    x: np.ndarray = field(init=False)
    c: float = field(init=False)
    h_z: float = field(init=False)
    n_z: int = field(init=False)
    ny_minus: int = field(init=False)
    ny_plus: int = field(init=False)
    n_in: int = field(init=False)

    def __post_init__(self):
        x_int = 2.5 * self.strike
        F = max(self.frac, x_int / self.x_max)
        self.c = sinh_c(x_int, self.x_max, F) if F < 1.0 else float("inf")
        xi_int = x_int / self.c
        xi_max = xi_int + math.asinh((self.x_max - x_int) / self.c)
        xi = np.arange(self.n + 1) * (xi_max / self.n)
        self.x = np.where(xi <= xi_int, self.c * xi, x_int + self.c * np.sinh(xi - xi_int))
        self.x[-1] = self.x_max
        self.n_z = 2 * self.n
        self.h_z = self.z_iii / self.n_z
        base_m = math.ceil(-math.log(self.x[1]) / self.h_z)
        base_p = math.ceil(math.log(self.x_max) / self.h_z)
        star = 0
        while max_prime_factor(base_m + base_p + 2 * self.n_z + 2 * star) > 7:
            star += 1
        self.ny_minus = base_m + star
        self.ny_plus = base_p + star
        self.n_in = self.ny_minus + self.ny_plus + 2 * self.n_z

    @property
    def y_out(self) -> np.ndarray:
        return np.exp(np.arange(-self.ny_minus, self.ny_plus + 1) * self.h_z)

    @property
    def y_in(self) -> np.ndarray:
        return np.exp((np.arange(-self.n_z - self.ny_minus, self.n_z + self.ny_plus) + 0.5) * self.h_z)

    def z_grid(self) -> Grid:
        """A log-grid object whose z-lattice is this scheme's (h = h_z, n_z = N_z), for the weights."""
        return Grid(2 * self.n_z, half_width=self.n_z * self.h_z)


def max_prime_factor(n: int) -> int:
    p, m, best = 2, n, 1
    while p * p <= m:
        while m % p == 0:
            best, m = p, m // p
        p += 1
    return max(best, m) if m > 1 else best


# --------------------------------------------------------------------------
# interpolation (cubic Lagrange, Sec. 4)
# --------------------------------------------------------------------------


def lagrange_matrix(nodes: np.ndarray, targets: np.ndarray, outside: str) -> sp.csr_matrix:
    """Rows: cubic Lagrange weights of `targets` on the increasing `nodes`,
    four consecutive nodes around each target (shifted inside at the ends).
    outside = 'zero': targets beyond the last node get an empty row;
    outside = 'linear': targets outside [nodes[0], nodes[-1]] are linearly
    extrapolated from the two nearest nodes."""
    n = nodes.size
    rows, cols, vals = [], [], []
    for i, t in enumerate(targets):
        if t > nodes[-1] or t < nodes[0]:
            if outside == "zero" and t > nodes[-1]:
                continue
            if outside == "linear" or t < nodes[0]:
                j = 0 if t < nodes[0] else n - 2
                a, b = nodes[j], nodes[j + 1]
                rows += [i, i]
                cols += [j, j + 1]
                vals += [(b - t) / (b - a), (t - a) / (b - a)]
                continue
        k = int(np.searchsorted(nodes, t, side="right")) - 1
        k = min(max(k, 0), n - 2)
        s = min(max(k - 1, 0), n - 4)
        pts = nodes[s:s + 4]
        for q in range(4):
            w = 1.0
            for r in range(4):
                if r != q:
                    w *= (t - pts[r]) / (pts[q] - pts[r])
            rows.append(i)
            cols.append(s + q)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(targets.size, n))


# --------------------------------------------------------------------------
# the jump operator B_w = T_out I~ C T_in (eqs. 3.12-3.17) and D (Sec. 3.2.1)
# --------------------------------------------------------------------------


class PriceSpaceOperators:
    def __init__(self, model: NTSModel, pg: PriceGrid):
        self.pg = pg
        self.pre = precompute(model, pg.z_grid())
        x = pg.x
        self.Tin = lagrange_matrix(x, pg.y_in, "zero")            # x -> y_in (per axis)
        self.Tout = lagrange_matrix(pg.y_out, x, "linear")         # y_out -> x (per axis)
        self.D1, self.D2 = fd_matrices(x)

    def jump(self, V: np.ndarray) -> np.ndarray:
        """B_w V on the (N_x+1)^2 x-grid; V[m2, m1]."""
        pg = self.pg
        A = self.Tin @ V @ self.Tin.T                               # [y_in m2, y_in m1] (tensor product)
        A = np.asarray(A)
        n_in, nz = pg.n_in, pg.n_z
        # circulant of size #in: first row = vec([Omega 0; 0 0]) -> cross-correlation (eq. 3.13)
        Wpad = np.zeros((n_in, n_in))
        Wpad[:2 * nz, :2 * nz] = self.pre.omega
        Cy = np.fft.irfft2(np.conj(np.fft.rfft2(Wpad)) * np.fft.rfft2(A), s=A.shape)
        n_out = pg.ny_minus + pg.ny_plus + 1
        By = Cy[:n_out, :n_out]                                     # I~: the kept outputs
        return np.asarray(self.Tout @ By @ self.Tout.T)

    def diffusion(self) -> sp.csr_matrix:
        """D on all (N_x+1)^2 nodes, m1 fastest (Sec. 3.2.1)."""
        a = self.pre.a
        x = self.pg.x
        n1 = x.size
        I = sp.identity(n1, format="csr")
        Ix = sp.diags(x)
        return (0.5 * a[0, 0] * sp.kron(I, Ix @ Ix @ self.D2) + a[0, 1] * sp.kron(Ix @ self.D1, Ix @ self.D1)
                + 0.5 * a[1, 1] * sp.kron(Ix @ Ix @ self.D2, I)).tocsr()


def fd_matrices(x: np.ndarray):
    """First and second central differences on the non-uniform grid; row 0
    zero; at x_max the second difference is zero and the first is backward."""
    n1 = x.size
    h = np.diff(x)                      # h[m-1] = x_m - x_{m-1}
    r1, c1, v1, r2, c2, v2 = [], [], [], [], [], []
    for m in range(1, n1 - 1):
        hm, hp = h[m - 1], h[m]
        r1 += [m, m, m]
        c1 += [m - 1, m, m + 1]
        v1 += [-hp / (hm * (hm + hp)), (hp - hm) / (hm * hp), hm / (hp * (hm + hp))]
        r2 += [m, m, m]
        c2 += [m - 1, m, m + 1]
        v2 += [2.0 / (hm * (hm + hp)), -2.0 / (hm * hp), 2.0 / (hp * (hm + hp))]
    m = n1 - 1
    r1 += [m, m]
    c1 += [m - 1, m]
    v1 += [-1.0 / h[-1], 1.0 / h[-1]]
    D1 = sp.csr_matrix((v1, (r1, c1)), shape=(n1, n1))
    D2 = sp.csr_matrix((v2, (r2, c2)), shape=(n1, n1))
    return D1, D2


# --------------------------------------------------------------------------
# initial values with cell averaging (Sec. 3.2.3) and the time loop (Sec. 3.3)
# --------------------------------------------------------------------------


def _H(t):
    return np.maximum(t, 0.0) ** 3 / 6.0


def put_avg_cell_integral(K, a1, b1, a2, b2):
    """int_{a1}^{b1} int_{a2}^{b2} max(K - (x1 + x2)/2, 0) dx2 dx1 in closed form
    (two integrations of the positive part of an affine function)."""
    return 4.0 * (_H(K - a1 / 2 - a2 / 2) - _H(K - a1 / 2 - b2 / 2) - _H(K - b1 / 2 - a2 / 2) + _H(K - b1 / 2 - b2 / 2))


def initial_values_price(pg: PriceGrid, contract: Contract) -> np.ndarray:
    """phi at the nodes, replaced by the cell average on cells that meet the
    kink x1 + x2 = 2K (put or call on the average)."""
    from .scheme import CALL_AVG, PUT_AVG
    x, K = pg.x, contract.strike
    n1 = x.size
    mid = 0.5 * (x[1:] + x[:-1])
    lo = np.concatenate(([-mid[0]], mid))                       # x_{m-1/2}
    hi = np.concatenate((mid, [2 * x[-1] - mid[-1]]))           # x_{m+1/2}
    X1, X2 = np.meshgrid(x, x)
    put = np.maximum(K - 0.5 * (X1 + X2), 0.0)
    A1, A2 = np.meshgrid(lo, lo)
    B1, B2 = np.meshgrid(hi, hi)
    s_min, s_max = A1 + A2, B1 + B2
    kink = (s_min < 2 * K) & (s_max > 2 * K)
    avg = put_avg_cell_integral(K, A1, B1, A2, B2) / ((B1 - A1) * (B2 - A2))
    put = np.where(kink, avg, put)
    if contract.payoff == PUT_AVG:
        return put
    if contract.payoff == CALL_AVG:
        centre = 0.25 * (A1 + B1 + A2 + B2)                      # average of the affine part over the cell
        lin = np.where(kink, centre, 0.5 * (X1 + X2)) - K
        return put + lin
    raise ValueError("price-space oracle: put or call on the average")


@dataclass
class PriceResult:
    V: np.ndarray
    price_at: callable
    iters: list


class PriceScheme:
    """Algorithm 1 in price space on the paper's grid (see the module docstring)."""

    def __init__(self, model: NTSModel, pg: PriceGrid, contract: Contract, n_steps: int, theta: float = 0.5,
                 tol: float = 1e-7, damping: bool = True, kmax: int = 100):
        self.model, self.pg, self.contract = model, pg, contract
        self.n_steps, self.theta, self.tol, self.damping, self.kmax = n_steps, theta, tol, damping, kmax
        self.ops = PriceSpaceOperators(model, pg)
        self.D = self.ops.diffusion()
        self.r_w = self.ops.pre.r_w
        self.kappa = self.ops.pre.kappa_w
        self._lu = {}
        self._sl = {}

    def lu(self, ht, theta):
        key = (ht, theta)
        if key not in self._lu:
            k = self.pg.x.size ** 2
            A = (sp.identity(k) * (1.0 + ht * theta * self.r_w) - ht * theta * self.D).tocsc()
            self._lu[key] = spla.splu(A)
        return self._lu[key]

    def sl(self, ht):
        if ht not in self._sl:
            x = self.pg.x
            self._sl[ht] = (lagrange_matrix(x, x * math.exp(self.kappa[0] * ht), "linear"),
                            lagrange_matrix(x, x * math.exp(self.kappa[1] * ht), "linear"))
        return self._sl[ht]

    def theta_step(self, V, BV, start, ht, theta):
        n1 = self.pg.x.size
        Dv = (self.D @ V.ravel()).reshape(n1, n1)
        Z = V + ht * (1.0 - theta) * (Dv - self.r_w * V + BV)
        T1, T2 = self.sl(ht)
        W = np.asarray(T2 @ Z @ T1.T)
        lu = self.lu(ht, theta)
        Y = start.copy()
        for k in range(1, self.kmax + 1):
            BY = self.ops.jump(Y)
            Ynew = lu.solve((ht * theta * BY + W).ravel()).reshape(n1, n1)
            err = float(np.max(np.abs(Ynew - Y) / np.maximum(1.0, np.abs(Ynew))))
            Y = Ynew
            if err < self.tol:
                break
        else:
            raise RuntimeError("price-space fixed point did not converge")
        return Y, self.ops.jump(Y), k

    def solve(self) -> PriceResult:
        T = self.contract.maturity
        ht = T / self.n_steps
        V0 = initial_values_price(self.pg, self.contract)
        iters = []
        hist = [V0]
        V, BV = V0, self.ops.jump(V0)
        first = 1
        if self.damping:
            for j in range(4):
                V, BV, k = self.theta_step(V, BV, V, ht / 4.0, 1.0)
                iters.append(k)
            hist.append(V)
            first = 2
        for step in range(first, self.n_steps + 1):
            h_ = hist[::-1]
            if len(h_) == 1:
                Y0 = h_[0]
            elif len(h_) == 2:
                Y0 = 2.0 * h_[0] - h_[1]
            elif len(h_) == 3:
                Y0 = 3.0 * h_[0] - 3.0 * h_[1] + h_[2]
            else:
                Y0 = 4.0 * h_[0] - 6.0 * h_[1] + 4.0 * h_[2] - h_[3]
            V, BV, k = self.theta_step(V, BV, Y0, ht, self.theta)
            iters.append(k)
            hist.append(V)
            if len(hist) > 4:
                hist.pop(0)
        x = self.pg.x

        def price_at(x1, x2, V=V):
            """Bicubic interpolation of V at (x1, x2) (cubic Lagrange on the x-grid)."""
            w1 = lagrange_matrix(x, np.array([x1]), "linear")
            w2 = lagrange_matrix(x, np.array([x2]), "linear")
            return float((w2 @ V @ w1.T)[0, 0])

        return PriceResult(V=V, price_at=price_at, iters=iters)
