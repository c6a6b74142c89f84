"""Oracle: the paper's discretisation of the 2D exponential-Levy PIDE, FP64, CPU.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

It follows Sec. 3 and Algorithm 1 of the paper step by step, on a uniform
log-price grid (the readings of the paper used here are listed, with
reasons, in the repository's design notes):

* grid        s_m = s_lo + m h, h = 2L/N, m = 0..N (node N is the upper
              Dirichlet boundary, not stored by the GPU path); unknowns are
              the interior nodes m in [1, N-1]^2; ln S0 is node N/2.
* z-grid      z_l = (l + 1/2) h_z, l = -N_z..N_z-1, h_z = h (Sec. 3.1).
* zones       z_I = 2 h_z, z_II = h_z ceil(sqrt(0.1) z_III/h_z - 1/2),
              z_III = N_z h_z (Sec. 4 scheme parameters).
* weights     eq. (3.5): 0 in R_I, ||z_l||^-2 int_{R_l} ||z||^2 l(dz) in R_II
              (Euclidean norm, Prop. 3.1), l(z_l) h_z^2 in R_III.
* rates       eq. (3.6): r_w = r + sum w, kappa_w^i = r - sum w (e^{z^i} - 1),
              sigma_w sigma_w^T = sigma sigma^T + int_{R_I} z z^T l(dz) (eq. 3.3).
* jump term   eqs. (3.10)-(3.17): cubic-Lagrange midpoint interpolation T_in
              (weights -1, 9, 9, -1 over 16 per axis), cross-correlation with
              Omega via zero-padded FFT with the conjugated weight spectrum
              (eq. 3.13); T_out is the identity on the log grid.  A direct
              summation version exists for small grids.
* diffusion   eq. (3.9) with the log-space generator: D = a11/2 d11 + a12 d1 d2
              + a22/2 d22, second-order central differences; first-order
              terms go into the semi-Lagrangian departure point.
* time        eq. (3.23) theta-scheme with semi-Lagrangian departure
              s + (kappa_w - a_ii/2) h_t; first step replaced by four steps
              of h_t/4 with theta = 1 (Sec. 3.3); fixed-point iteration
              eq. (3.24) with stopping rule eq. (3.25) and extrapolated start
              eq. (3.26); the linear system of eq. (3.24) is solved exactly
              (sparse LU), which is what BiCGSTAB+ILU at 1e-14 approximates.
* far field   nodes outside the interior carry g(s, tau), the discounted
              intrinsic value (exact solution where the payoff is linear).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import integrate

from .levy import NTSModel, levy_density

PUT_AVG = 0
CALL_AVG = 1
PUT_ASSET1 = 2

# cubic Lagrange weights at the midpoint of [j, j+1] from nodes j-1..j+2
MID_W = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
@dataclass
class Grid:
    n: int                      # N: nodes 0..N per axis, interior 1..N-1
    s_center: tuple = (math.log(100.0), math.log(100.0))
    half_width: float = 2.5     # L
    n_z: int | None = None      # N_z, default N/2 (z_III = L)

    def __post_init__(self):
        if self.n_z is None:
            self.n_z = self.n // 2

    @property
    def h(self) -> float:
        return 2.0 * self.half_width / self.n

    def s(self, axis: int, m):
        return self.s_center[axis] - self.half_width + np.asarray(m, dtype=np.float64) * self.h


@dataclass
class Contract:
    payoff: int = PUT_AVG
    strike: float = 100.0
    maturity: float = 1.0


def zones(grid: Grid):
    """Sec. 4 choices: z_I = 2 h_z, z_II = h_z ceil(sqrt(0.1) z_III/h_z - 1/2),
    z_III = N_z h_z.  Returned as integer multiples of h_z: (2, M, N_z)."""
    m2 = int(math.ceil(math.sqrt(0.1) * grid.n_z - 0.5))
    return 2, m2, grid.n_z


# --------------------------------------------------------------------------
# Gauss-Legendre nodes (library routine)
# --------------------------------------------------------------------------
def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def cell_integral_r2(model: NTSModel, c1: np.ndarray, c2: np.ndarray, h: float, order: int = 20):
    """int over [c1-h/2, c1+h/2] x [c2-h/2, c2+h/2] of ||z||_2^2 l(z) dz by
    tensor Gauss-Legendre (the 'common numerical integrator' of Sec. 3.1);
    vectorised over cells."""
    x, w = _gl(order)
    off = 0.5 * h * x
    W = np.outer(w, w) * (0.25 * h * h)
    out = np.zeros(c1.shape, dtype=np.float64)
    for a in range(order):
        for b in range(order):
            z1 = c1 + off[a]
            z2 = c2 + off[b]
            out += W[a, b] * (z1 * z1 + z2 * z2) * levy_density(model, z1, z2)
    return out


def r1_moment(model: NTSModel, H: float, order: int = 96) -> np.ndarray:
    """int_{[-H,H]^2} z z^T l(z) dz (eq. 3.3 with R_I = {||z||_inf <= H}).
    The square is split into four triangles with apex at the origin; in the
    triangle touching the edge z1 = +H, z = rho (1, t), rho in [0, H],
    t in [-1, 1], dz = rho drho dt (and likewise for the other three edges).
    The integrand behaves like rho^(1-2 alpha) at the apex: the rho integral
    is Gauss-Jacobi with exactly that weight (library nodes), the edge
    integral Gauss-Legendre."""
    from scipy.special import roots_jacobi
    a = model.alpha
    # Gauss-Jacobi on [-1,1] with weight (1-x)^0 (1+x)^(1-2a); map x -> rho = H (1+x)/2
    xj, wj = roots_jacobi(order, 0.0, 1.0 - 2.0 * a)
    rho = 0.5 * H * (1.0 + xj)
    wr = wj * (0.5 * H) ** (2.0 - 2.0 * a)       # d rho and (rho)^(1-2a) rescaling
    xt, wt = _gl(order)
    out = np.zeros((2, 2))
    edges = [((1.0, 0.0), (0.0, 1.0)), ((-1.0, 0.0), (0.0, 1.0)),
             ((0.0, 1.0), (1.0, 0.0)), ((0.0, -1.0), (1.0, 0.0))]
    R, T = np.meshgrid(rho, xt, indexing="ij")
    Wgt = np.outer(wr, wt)
    for (e1, e2), (f1, f2) in edges:
        d1 = e1 + T * f1
        d2 = e2 + T * f2
        # rho^3 d_i d_j l(rho d) / rho^(1-2a) = rho^(2+2a) d_i d_j l(rho d)
        gbase = R ** (2.0 + 2.0 * a) * levy_density(model, R * d1, R * d2)
        out[0, 0] += np.sum(Wgt * gbase * d1 * d1)
        out[0, 1] += np.sum(Wgt * gbase * d1 * d2)
        out[1, 1] += np.sum(Wgt * gbase * d2 * d2)
    out[1, 0] = out[0, 1]
    return out


@dataclass
class Precomputed:
    omega: np.ndarray          # [l2 + N_z, l1 + N_z], shape (2N_z, 2N_z)
    zone: np.ndarray           # 1 = R_I, 2 = R_II, 3 = R_III (same shape)
    a: np.ndarray              # sigma_w sigma_w^T (2x2)
    r_w: float
    kappa_w: np.ndarray        # (2,)
    b: np.ndarray              # SL drift kappa_w - a_ii/2 (2,)
    sum_w: float


def precompute(model: NTSModel, grid: Grid, r2_order: int = 20) -> Precomputed:
    """Weights (eq. 3.5), artificial diffusion (eq. 3.3) and rates (eq. 3.6)."""
    h = grid.h
    nz = grid.n_z
    zI, zII, zIII = zones(grid)
    l = np.arange(-nz, nz)
    L1, L2 = np.meshgrid(l, l)          # [l2, l1]
    c1 = (L1 + 0.5) * h
    c2 = (L2 + 0.5) * h
    inf_idx = np.maximum(np.abs(L1 + 0.5), np.abs(L2 + 0.5))   # ||z_l||_inf / h
    zone = np.where(inf_idx <= zI, 1, np.where(inf_idx <= zII, 2, 3))
    omega = np.zeros_like(c1)
    m3 = zone == 3
    omega[m3] = levy_density(model, c1[m3], c2[m3]) * h * h
    m2 = zone == 2
    omega[m2] = (cell_integral_r2(model, c1[m2], c2[m2], h, r2_order)
                 / (c1[m2] ** 2 + c2[m2] ** 2))
    a = model.sigma_matrix + r1_moment(model, zI * h)
    sum_w = float(omega.sum())
    r_w = model.r + sum_w
    kappa_w = np.array([model.r - float((omega * np.expm1(c1)).sum()),
                        model.r - float((omega * np.expm1(c2)).sum())])
    b = kappa_w - 0.5 * np.diag(a)
    return Precomputed(omega=omega, zone=zone, a=a, r_w=r_w, kappa_w=kappa_w, b=b, sum_w=sum_w)


# --------------------------------------------------------------------------
# payoff, far field, cell averaging
# --------------------------------------------------------------------------
def payoff(contract: Contract, S1, S2):
    K = contract.strike
    if contract.payoff == PUT_AVG:
        return np.maximum(K - 0.5 * (S1 + S2), 0.0)
    if contract.payoff == CALL_AVG:
        return np.maximum(0.5 * (S1 + S2) - K, 0.0)
    if contract.payoff == PUT_ASSET1:
        return np.maximum(K - S1 + 0.0 * S2, 0.0)
    raise ValueError("unknown payoff")


def far_field(contract: Contract, r: float, s1, s2, tau: float):
    """g(s, tau): the payoff with the strike discounted by e^{-r tau}."""
    c = Contract(contract.payoff, contract.strike * math.exp(-r * tau), contract.maturity)
    return payoff(c, np.exp(s1), np.exp(s2))


def _inner_put_avg(c, a, b):
    """int_a^b max(c - e^{s}/2, 0) ds  (c = K - e^{s2}/2)."""
    if c <= 0.0:
        return 0.0
    up = min(b, math.log(2.0 * c))
    if up <= a:
        return 0.0
    return c * (up - a) - 0.5 * (math.exp(up) - math.exp(a))


def _inner_call_avg(c, a, b):
    """int_a^b max(e^{s}/2 - c, 0) ds  (c = K - e^{s2}/2)."""
    if c <= 0.0:
        return 0.5 * (math.exp(b) - math.exp(a)) - c * (b - a)
    lo = max(a, math.log(2.0 * c))
    if lo >= b:
        return 0.0
    return 0.5 * (math.exp(b) - math.exp(lo)) - c * (b - lo)


def cell_average(contract: Contract, a1, b1, a2, b2) -> float:
    """eq. (3.18) in log coordinates: (1/h^2) int int phi(e^{s1}, e^{s2}) ds
    over the cell; inner integral in s1 in closed form, outer integral in s2
    adaptive with the kink crossings as break points."""
    K = contract.strike
    area = (b1 - a1) * (b2 - a2)
    if contract.payoff == PUT_ASSET1:
        up = min(b1, math.log(K))
        v = 0.0 if up <= a1 else K * (up - a1) - (math.exp(up) - math.exp(a1))
        return v * (b2 - a2) / area
    inner = _inner_put_avg if contract.payoff == PUT_AVG else _inner_call_avg
    pts = []
    for s in (a1, b1):
        q = 2.0 * K - math.exp(s)
        if q > 0.0:
            t = math.log(q)
            if a2 < t < b2:
                pts.append(t)
    v, _ = integrate.quad(lambda s2: inner(K - 0.5 * math.exp(s2), a1, b1), a2, b2,
                          points=pts or None, epsabs=1e-14 * area, epsrel=1e-13, limit=200)
    return v / area


def initial_values(contract: Contract, grid: Grid) -> np.ndarray:
    """V^0 on nodes [0, N]^2, array [m2, m1]: pointwise payoff, replaced by
    the cell average (eq. 3.18) at interior nodes whose cell meets the kink."""
    n = grid.n
    s1 = grid.s(0, np.arange(n + 1))
    s2 = grid.s(1, np.arange(n + 1))
    S1, S2 = np.meshgrid(np.exp(s1), np.exp(s2))
    V = payoff(contract, S1, S2)
    h = grid.h
    K = contract.strike
    for m2 in range(1, n):
        for m1 in range(1, n):
            a1, b1 = s1[m1] - 0.5 * h, s1[m1] + 0.5 * h
            a2, b2 = s2[m2] - 0.5 * h, s2[m2] + 0.5 * h
            if contract.payoff == PUT_ASSET1:
                crosses = math.exp(a1) < K < math.exp(b1)
            else:
                crosses = (math.exp(a1) + math.exp(a2) < 2.0 * K < math.exp(b1) + math.exp(b2))
            if crosses:
                V[m2, m1] = cell_average(contract, a1, b1, a2, b2)
    return V


# --------------------------------------------------------------------------
# jump operator (Sec. 3.2.2)
# --------------------------------------------------------------------------
def extend(grid: Grid, contract: Contract, r: float, Y_int: np.ndarray, tau: float,
           far: bool = True) -> np.ndarray:
    """U_ext on nodes m in [-N_z-1, N+N_z]^2 (array index m + N_z + 1):
    interior nodes from Y_int ((N-1)x(N-1), [m2-1, m1-1]); every other node
    carries g(s, tau) (or 0 when far=False)."""
    n, nz = grid.n, grid.n_z
    m = np.arange(-nz - 1, n + nz + 1)
    if far:
        S1, S2 = np.meshgrid(grid.s(0, m), grid.s(1, m))
        U = far_field(contract, r, S1, S2, tau)
    else:
        U = np.zeros((m.size, m.size))
    o = nz + 1
    U[o + 1:o + n, o + 1:o + n] = Y_int
    return U


def midpoints(U: np.ndarray) -> np.ndarray:
    """T_in: tensor cubic-Lagrange values at the cell midpoints j + 1/2 of the
    node lattice (eqs. 3.14, 3.16).  Input nodes index 0..M-1 give midpoints
    between nodes 1 and 2 .. M-3 and M-2 (M-3 values per axis)."""
    M = U.shape[0]
    A = sum(MID_W[b] * U[:, b:M - 3 + b] for b in range(4))          # along m1
    return sum(MID_W[b] * A[b:M - 3 + b, :] for b in range(4))       # along m2


def circulant_product(first: np.ndarray, a: np.ndarray) -> np.ndarray:
    """eq. (3.13): C a = ifft(conj(fft(C_1)) o fft(a)) for the block-circulant
    C whose first row is vec(first); with the vec ordering of eq. (3.7)
    (first index fastest) this is the 2D cyclic cross-correlation
    (C a)[p] = sum_k first[k] a[(p + k) mod P]."""
    s = a.shape
    return np.fft.irfft2(np.conj(np.fft.rfft2(first)) * np.fft.rfft2(a), s=s)


def jump_fft(grid: Grid, omega: np.ndarray, U: np.ndarray) -> np.ndarray:
    """(B_w V) at interior nodes by eq. (3.17): ifft(conj(fft(C_1)) o fft(T_in V)),
    i.e. a zero-padded 2D cross-correlation out[m] = sum_l w_l Umid[m + l].
    Padded size P = 2N per axis: the T_in output has N + 2 N_z - 1 <= 2N - 1
    points, so no kept output wraps around."""
    n, nz = grid.n, grid.n_z
    P = 2 * n
    Um = midpoints(U)                    # midpoints j = -N_z .. N+N_z-2
    A = np.zeros((P, P))
    A[:Um.shape[0], :Um.shape[1]] = Um
    Wpad = np.zeros((P, P))
    Wpad[:2 * nz, :2 * nz] = omega
    out = circulant_product(Wpad, A)
    return out[1:n, 1:n]


def jump_direct(grid: Grid, omega: np.ndarray, U: np.ndarray) -> np.ndarray:
    """The same sum as eq. (3.10) by direct summation: O(N^2 N_z^2)."""
    n, nz = grid.n, grid.n_z
    Um = midpoints(U)
    out = np.zeros((n - 1, n - 1))
    # Um index q corresponds to midpoint j = q - N_z; node m + l -> q = m + l + N_z
    for i2 in range(2 * nz):
        for i1 in range(2 * nz):
            w = omega[i2, i1]
            if w != 0.0:
                out += w * Um[1 + i2:n + i2, 1 + i1:n + i1]
    return out


# --------------------------------------------------------------------------
# diffusion (Sec. 3.2.1) and the semi-Lagrangian interpolation (Sec. 3.3)
# --------------------------------------------------------------------------
def diffusion_matrix(grid: Grid, a: np.ndarray) -> sp.csr_matrix:
    """D on the interior unknowns (m1 fastest, eq. 3.7 ordering):
    a11/2 I(x)d11 + a12 d1(x)d1 + a22/2 d22(x)I (eq. 3.9, log-space form)."""
    n, h = grid.n, grid.h
    k = n - 1
    I = sp.identity(k, format="csr")
    T2 = sp.diags([np.ones(k - 1), -2.0 * np.ones(k), np.ones(k - 1)], [-1, 0, 1]) / (h * h)
    T1 = sp.diags([-np.ones(k - 1), np.ones(k - 1)], [-1, 1]) / (2.0 * h)
    return (0.5 * a[0, 0] * sp.kron(I, T2) + a[0, 1] * sp.kron(T1, T1)
            + 0.5 * a[1, 1] * sp.kron(T2, I)).tocsr()


def apply_diffusion(grid: Grid, a: np.ndarray, V: np.ndarray) -> np.ndarray:
    """D applied to a full node array V ([0,N]^2), evaluated at interior nodes."""
    h = grid.h
    c = V[1:-1, 1:-1]
    d11 = (V[1:-1, 2:] - 2.0 * c + V[1:-1, :-2]) / (h * h)
    d22 = (V[2:, 1:-1] - 2.0 * c + V[:-2, 1:-1]) / (h * h)
    d12 = (V[2:, 2:] - V[:-2, 2:] - V[2:, :-2] + V[:-2, :-2]) / (4.0 * h * h)
    return 0.5 * a[0, 0] * d11 + a[0, 1] * d12 + 0.5 * a[1, 1] * d22


def solve_nonmixed(grid: Grid, a: np.ndarray, r_w: float, ht: float, theta: float,
                   rhs: np.ndarray) -> np.ndarray:
    """X with ((1 + ht theta r_w) I - ht theta (a11/2 d11 + a22/2 d22)) X = rhs on
    the interior nodes ((N-1) x (N-1), zero Dirichlet ring): the matrix of
    eq. (3.24) without the mixed term a12 d1 d2 (Sec. 3.2.1 differences).  The
    operator is diagonal in the 2D sine basis sin(pi k m / N), with
    eigenvalues 1 + ht theta (r_w + a11/2 l_k1 + a22/2 l_k2),
    l_k = (2 - 2 cos(pi k / N)) / h^2; the type-I DST of scipy is used as a
    library step.  (Used to check the CUDA path's inner solve kernel by kernel;
    the scheme itself solves eq. (3.24) with the full matrix.)"""
    from scipy.fft import dstn, idstn
    n, h = grid.n, grid.h
    k = np.arange(1, n)
    lk = (2.0 - 2.0 * np.cos(np.pi * k / n)) / (h * h)
    lam = 1.0 + ht * theta * (r_w + 0.5 * a[0, 0] * lk[None, :] + 0.5 * a[1, 1] * lk[:, None])
    return idstn(dstn(rhs, type=1) / lam, type=1)


def sl_weights(shift_cells: float, order: int):
    """Lagrange weights for evaluating at node + shift (|shift| < 1 cell).
    Returns (first tap offset, weights).  order 1: linear on [o, o+1];
    order 3: cubic on o-1..o+2, o = floor(shift)."""
    o = math.floor(shift_cells)
    f = shift_cells - o
    if order == 1:
        return o, np.array([1.0 - f, f])
    if order == 3:
        return o - 1, np.array([-f * (f - 1.0) * (f - 2.0) / 6.0,
                                (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0,
                                -(f + 1.0) * f * (f - 2.0) / 2.0,
                                (f + 1.0) * f * (f - 1.0) / 6.0])
    raise ValueError("order must be 1 or 3")


def sl_interpolate(Zx: np.ndarray, pad: int, n: int, shift: tuple, order: int) -> np.ndarray:
    """T_SL: values at interior nodes m + shift (in cells) from the node array
    Zx covering [-pad, N+pad]^2.  Tensor-product Lagrange (eq. 3.22)."""
    o1, w1 = sl_weights(shift[0], order)
    o2, w2 = sl_weights(shift[1], order)
    out = np.zeros((n - 1, n - 1))
    for b, wb in enumerate(w2):
        for a_, wa in enumerate(w1):
            r0 = pad + 1 + o2 + b
            c0 = pad + 1 + o1 + a_
            out += wb * wa * Zx[r0:r0 + n - 1, c0:c0 + n - 1]
    return out


# --------------------------------------------------------------------------
# Greeks (Sec. 4: second-order central differences on the grid)
# --------------------------------------------------------------------------
def greeks(grid: Grid, V: np.ndarray) -> dict:
    """Delta_i = dV/dS_i and Gamma_ij = d2V/dS_i dS_j at the interior nodes by
    central differences in log price: dV/dS = V_s / S,
    d2V/dS^2 = (V_ss - V_s) / S^2, d2V/dS1 dS2 = V_s1s2 / (S1 S2)."""
    h = grid.h
    n = grid.n
    S1 = np.exp(grid.s(0, np.arange(1, n)))[None, :]
    S2 = np.exp(grid.s(1, np.arange(1, n)))[:, None]
    c = V[1:-1, 1:-1]
    v1 = (V[1:-1, 2:] - V[1:-1, :-2]) / (2 * h)
    v2 = (V[2:, 1:-1] - V[:-2, 1:-1]) / (2 * h)
    v11 = (V[1:-1, 2:] - 2 * c + V[1:-1, :-2]) / (h * h)
    v22 = (V[2:, 1:-1] - 2 * c + V[:-2, 1:-1]) / (h * h)
    v12 = (V[2:, 2:] - V[:-2, 2:] - V[2:, :-2] + V[:-2, :-2]) / (4 * h * h)
    return {"delta1": v1 / S1, "delta2": v2 / S2, "gamma11": (v11 - v1) / (S1 * S1),
            "gamma12": v12 / (S1 * S2), "gamma22": (v22 - v2) / (S2 * S2)}


# --------------------------------------------------------------------------
# time stepping (Sec. 3.3, Algorithm 1)
# --------------------------------------------------------------------------
@dataclass
class SolveResult:
    V: np.ndarray                  # final values on [0, N]^2, [m2, m1]
    price: float                   # V at node (N/2, N/2)
    iters: list = field(default_factory=list)   # fixed-point iterations per (sub)step
    resid: list = field(default_factory=list)
    pre: Precomputed | None = None


class Scheme:
    """Algorithm 1 on the log grid.  ``jump`` selects 'fft' (eq. 3.17) or
    'direct' (eq. 3.10)."""

    def __init__(self, model: NTSModel, grid: Grid, contract: Contract, n_steps: int,
                 theta: float = 0.5, tol: float = 1e-10, sl_order: int = 1,
                 damping: bool = True, kmax: int = 100, jump: str = "fft",
                 pre: Precomputed | None = None):
        self.model, self.grid, self.contract = model, grid, contract
        self.n_steps, self.theta, self.tol = n_steps, theta, tol
        self.sl_order, self.damping, self.kmax = sl_order, damping, kmax
        self.jump = jump_fft if jump == "fft" else jump_direct
        self.pre = pre if pre is not None else precompute(model, grid)
        self.Dint = diffusion_matrix(grid, self.pre.a)
        self._lu = {}
        n = grid.n
        self.s1 = grid.s(0, np.arange(n + 1))
        self.s2 = grid.s(1, np.arange(n + 1))

    # far field on the full node set [0,N]^2
    def g_nodes(self, tau):
        S1, S2 = np.meshgrid(self.s1, self.s2)
        return far_field(self.contract, self.model.r, S1, S2, tau)

    def B(self, Y_int, tau):
        U = extend(self.grid, self.contract, self.model.r, Y_int, tau)
        return self.jump(self.grid, self.pre.omega, U)

    def lu(self, ht, theta):
        key = (ht, theta)
        if key not in self._lu:
            k = (self.grid.n - 1) ** 2
            A = (sp.identity(k) * (1.0 + ht * theta * self.pre.r_w) - ht * theta * self.Dint).tocsc()
            self._lu[key] = spla.splu(A)
        return self._lu[key]

    def explicit_part(self, Vfull, BV, ht, theta, tau_prev):
        """Z = (I + h_t(1-theta)(D - r_w)) V + h_t (1-theta) B V at interior
        nodes; g(s, tau_{n-1}) at every other node (pad 2 around [0,N])."""
        n = self.grid.n
        pad = 2
        m = np.arange(-pad, n + pad + 1)
        S1, S2 = np.meshgrid(self.grid.s(0, m), self.grid.s(1, m))
        Zx = far_field(self.contract, self.model.r, S1, S2, tau_prev)
        Vi = Vfull[1:-1, 1:-1]
        Z = Vi + ht * (1.0 - theta) * (apply_diffusion(self.grid, self.pre.a, Vfull)
                                       - self.pre.r_w * Vi + BV)
        Zx[pad + 1:pad + n, pad + 1:pad + n] = Z
        return Zx, pad

    def theta_step(self, Vfull, BV, start_int, tau_prev, tau, ht, theta):
        """One step of eq. (3.23) by the fixed-point iteration (3.24)-(3.25)
        from time level tau_prev to tau = tau_prev + ht.
        Returns (V^n full, B V^n, iterations, last increment)."""
        n = self.grid.n
        shift = (self.pre.b[0] * ht / self.grid.h, self.pre.b[1] * ht / self.grid.h)
        Zx, pad = self.explicit_part(Vfull, BV, ht, theta, tau_prev)
        W = sl_interpolate(Zx, pad, n, shift, self.sl_order)
        gfull = self.g_nodes(tau)
        gring = gfull.copy()
        gring[1:-1, 1:-1] = 0.0
        Wb = W + ht * theta * apply_diffusion(self.grid, self.pre.a, gring)
        lu = self.lu(ht, theta)
        Y = start_int.copy()
        err = np.inf
        for k in range(1, self.kmax + 1):
            BY = self.B(Y, tau)
            rhs = ht * theta * BY + Wb
            Ynew = lu.solve(rhs.ravel()).reshape(n - 1, n - 1)
            err = float(np.max(np.abs(Ynew - Y) / np.maximum(1.0, np.abs(Ynew))))
            Y = Ynew
            if err < self.tol:
                break
        else:
            raise RuntimeError("fixed-point iteration did not converge")
        Vn = gfull
        Vn[1:-1, 1:-1] = Y
        return Vn, self.B(Y, tau), k, err

    def iterate(self):
        """Algorithm 1 time loop as a generator: yields (step, iterations)
        after every time step (the damped first step yields once, with the
        iterations of its four substeps summed); the final state is left in
        ``self.result``."""
        T = self.contract.maturity
        ht = T / self.n_steps
        n = self.grid.n
        V0 = self.g_nodes(0.0)
        V0[1:-1, 1:-1] = initial_values(self.contract, self.grid)[1:-1, 1:-1]
        res = SolveResult(V=None, price=float("nan"), pre=self.pre)
        self.result = res
        hist = [V0]
        V = V0
        BV = self.B(V0[1:-1, 1:-1], 0.0)
        if self.damping:
            hq = ht / 4.0
            ktot = 0
            for j in range(4):
                V, BV, k, e = self.theta_step(V, BV, V[1:-1, 1:-1], j * hq, (j + 1) * hq, hq, 1.0)
                res.iters.append(k)
                res.resid.append(e)
                ktot += k
            hist.append(V)
            first = 2
            res.V = V
            yield 1, ktot
        else:
            first = 1
        for step in range(first, self.n_steps + 1):
            h_ = [x[1:-1, 1:-1] for x in hist[::-1]]   # V^{n-1}, V^{n-2}, ...
            if len(h_) == 1:
                Y0 = h_[0]
            elif len(h_) == 2:
                Y0 = 2.0 * h_[0] - h_[1]
            elif len(h_) == 3:
                Y0 = 3.0 * h_[0] - 3.0 * h_[1] + h_[2]
            else:
                Y0 = 4.0 * h_[0] - 6.0 * h_[1] + 4.0 * h_[2] - h_[3]
            V, BV, k, e = self.theta_step(V, BV, Y0, (step - 1) * ht, step * ht, ht, self.theta)
            res.iters.append(k)
            res.resid.append(e)
            hist.append(V)
            if len(hist) > 4:
                hist.pop(0)
            res.V = V
            yield step, k
        res.price = float(V[n // 2, n // 2])

    def solve(self) -> SolveResult:
        for _ in self.iterate():
            pass
        return self.result
