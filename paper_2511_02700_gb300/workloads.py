"""Seeded synthetic workloads: the input generators shared by the tests, the
benchmark and the oracle checks.  Only parameters and random draws live
here -- none of the method's arithmetic.

The five workloads restate the benchmark configurations of the build: a
put on the average of two assets, K = 100, S0 = (100, 100), r = 0.03,
bivariate NTS jumps from a unit-mean tempered-stable subordinator with
variance kappa, Brownian drift beta, volatilities sigma and correlation corr,
on a uniform log grid ln 100 +- 2.5 with N nodes per axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    steps: int
    alpha: float
    kappa: float = 0.5
    beta: tuple = (-0.10, -0.05)
    sigma: tuple = (0.20, 0.25)
    corr: float = 0.3
    r: float = 0.03
    strike: float = 100.0
    maturity: float = 1.0
    theta: float = 0.5
    tol: float = 1e-10
    precision: str = "fp64"        # "fp64" or "fp32"
    sl_order: int = 3
    half_width: float = 2.5


# plain FP64 pricing, 128^2 grid, 32 steps, tol 1e-10
PLAIN_FP64_128 = Workload("plain_fp64_128", n=128, steps=32, alpha=0.25, tol=1e-10, precision="fp64")


def convergence_sweep(precision: str):
    """alpha in {0.25, 0.5, 0.75} x N in {256, 512, 1024}, steps N/4, tol 1e-8."""
    return [Workload(f"sweep_a{a}_n{n}_{precision}", n=n, steps=n // 4, alpha=a, tol=1e-8,
                     precision=precision)
            for a in (0.25, 0.5, 0.75) for n in (256, 512, 1024)]


# large single solve: 4096^2 grid (8192^2 padded transforms), alpha 0.5, 1024 steps, tol 1e-7
LARGE_FP32_4096 = Workload("large_fp32_4096", n=4096, steps=1024, alpha=0.5, tol=1e-7, precision="fp32")


# adjoint: 1024^2 grid, 256 steps, FP64, tol 1e-10, checkpoints every 16 steps (alpha 0.25 and 0.5)
ADJOINT_FP64_1024 = Workload("adjoint_fp64_1024", n=1024, steps=256, alpha=0.25, tol=1e-10, precision="fp64")
ADJOINT_INTERVAL = 16


def batch_draw(count: int = 512, seed: int = 2511027):
    """Independent pricings with seed-drawn parameters (uniform ranges):
    alpha [0.1, 0.45], kappa [0.2, 1], sigma_i [0.1, 0.4], corr [-0.6, 0.6],
    beta_i [-0.2, 0.2], K [80, 120], T [0.1, 2]; N from {128, 256, 512} with
    N/4 steps; FP32-bulk, fixed-point tol 1e-8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        a = float(rng.uniform(0.1, 0.45))
        kap = float(rng.uniform(0.2, 1.0))
        s = (float(rng.uniform(0.1, 0.4)), float(rng.uniform(0.1, 0.4)))
        c = float(rng.uniform(-0.6, 0.6))
        b = (float(rng.uniform(-0.2, 0.2)), float(rng.uniform(-0.2, 0.2)))
        K = float(rng.uniform(80.0, 120.0))
        T = float(rng.uniform(0.1, 2.0))
        n = int(rng.choice([128, 256, 512]))
        out.append(Workload(f"batch_{i}", n=n, steps=n // 4, alpha=a, kappa=kap, beta=b, sigma=s, corr=c,
                            strike=K, maturity=T, tol=1e-8, precision="fp32"))
    return out


def random_field(n: int, seed: int, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    """(n+1) x (n+1) FP64 field, uniform in [lo, hi], for operator checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(n + 1, n + 1))


def with_(w: Workload, **kw) -> Workload:
    return replace(w, **kw)


# The paper's own parameter sets (Table 2: NTS alpha, lambda, delta, eta, the
# matrix rho as (rho11, rho12, rho22), r, T, K; sigma = 0), the price-space
# domains of its Sec. 4 experiments (x_max / K and z_max^III), and its Table 4
# price at (K, K) (N_x = 800; 400 for NIG0).  Printed values, cited data only.
@dataclass(frozen=True)
class PaperSet:
    name: str
    alpha: float
    lam: float
    delta: float
    eta: tuple
    rho: tuple
    r: float
    maturity: float
    strike: float
    x_max_over_k: float
    z_max_iii: float
    table4_at_k: float


PAPER_SETS = {
    "VG0": PaperSet("VG0", 0.0, 1.0, 1.0, (-0.1, -0.2), (0.09, 0.06, 0.16), 0.05, 1.0, 100.0, 57.0, 11.5010,
                    8.8020),
    "VG1": PaperSet("VG1", 0.0, 6.0, 6.0, (-0.1, -0.2), (0.01, 0.0, 0.0225), 0.0, 0.5, 100.0, 5.0, 2.1410, 2.9029),
    "NIG0": PaperSet("NIG0", 0.5, 20766.4, 0.77576, (-37.688, -2.224), (3.984, 3.160, 3.512), 0.0, 0.5, 100.0,
                     6.0, 0.4172, 5.1186),
    "NIG1": PaperSet("NIG1", 0.5, 57.1108, 4.26367, (-0.295846, -0.292984), (0.037021, 0.026574, 0.054613), 0.0,
                     0.5, 100.0, 7.0, 0.8807, 5.3956),
}
