"""Oracle computations that the GPU parity tests run in worker processes
(started with the spawn method, so no worker inherits a CUDA context).  Only
the oracle and the seeded input generators are used here."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2511_02700_gb300.workloads import Workload, random_field


def _inputs(w):
    m = O.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    return m, O.Grid(w.n, half_width=w.half_width), O.Contract(O.PUT_AVG, w.strike, w.maturity)


def solve(w: Workload):
    """Algorithm 1 for the workload's model, grid and contract: (price, V)."""
    m, g, c = _inputs(w)
    res = O.Scheme(m, g, c, w.steps, theta=w.theta, tol=w.tol, sl_order=w.sl_order).solve()
    return res.price, res.V


def probe_residual(n: int, seed: int) -> np.ndarray:
    """The residual field handed to one fixed-point iteration: uniform in
    [-1, 1] at the interior nodes, zero on the ring."""
    r = random_field(n, seed, -1.0, 1.0)
    r[0, :] = r[-1, :] = r[:, 0] = r[:, -1] = 0.0
    return r


def iteration_reference(w: Workload, seed: int, ht: float, theta: float, r2_order: int = 20):
    """One iteration of the increment loop from Y = 0 on the residual of
    probe_residual: delta solves the eq. (3.24) matrix without its mixed term,
    bdelta = B_w delta with a zero far field (eq. 3.17), and the eq. (3.25)
    quantity max |delta| / max(1, |delta|).  Returns (delta, bdelta, stop,
    sum of the weights) on the interior nodes."""
    m, g, c = _inputs(w)
    pre = O.precompute(m, g, r2_order=r2_order)
    r = probe_residual(w.n, seed)
    delta = O.solve_nonmixed(g, pre.a, pre.r_w, ht, theta, r[1:-1, 1:-1])
    bdelta = O.jump_fft(g, pre.omega, O.extend(g, c, m.r, delta, 0.0, far=False))
    stop = float(np.max(np.abs(delta) / np.maximum(1.0, np.abs(delta))))
    return delta, bdelta, stop, pre.sum_w
