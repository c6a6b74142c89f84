"""Price sensitivities of the oracle scheme by central finite differences.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The gradient of the discrete price V^{N_t}(S0) with respect to the
subordinated-Brownian-motion parameters (sigma_1, sigma_2, corr, kappa,
beta_1, beta_2) of the workloads (the Table A5 subordinator with unit mean
and variance kappa; Brownian drift beta and covariance built from sigma and
corr).  Each component is (P(p + e) - P(p - e)) / (2 e) with the oracle's
FP64 scheme (Algorithm 1) run to a tight fixed-point tolerance, so the
truncation error is O(e^2) and the fixed-point noise O(tol / e).
"""
from __future__ import annotations

from .levy import model_from_subordinated_bm
from .scheme import Contract, Grid, Scheme

PARAMS = ("sigma1", "sigma2", "corr", "kappa", "beta1", "beta2")


def _price(alpha, kappa, beta, sigma, corr, r, grid: Grid, contract: Contract, n_steps, theta, tol, sl_order):
    m = model_from_subordinated_bm(alpha, kappa, beta, sigma, corr, r)
    return Scheme(m, grid, contract, n_steps, theta=theta, tol=tol, sl_order=sl_order).solve().price


def price_gradient_fd(alpha, kappa, beta, sigma, corr, r, grid: Grid, contract: Contract, n_steps: int,
                      theta: float = 0.5, tol: float = 1e-13, sl_order: int = 3, eps: float = 1e-4) -> dict:
    """Central differences of the oracle price in each workload parameter."""
    base = {"sigma1": sigma[0], "sigma2": sigma[1], "corr": corr, "kappa": kappa,
            "beta1": beta[0], "beta2": beta[1]}

    def price_at(vals):
        return _price(alpha, vals["kappa"], (vals["beta1"], vals["beta2"]), (vals["sigma1"], vals["sigma2"]),
                      vals["corr"], r, grid, contract, n_steps, theta, tol, sl_order)

    out = {}
    for p in PARAMS:
        up = dict(base)
        dn = dict(base)
        up[p] += eps
        dn[p] -= eps
        out[p] = (price_at(up) - price_at(dn)) / (2.0 * eps)
    return out
