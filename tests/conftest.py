import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than ~20 s on the CPU")


def read_table(name):
    """Rows of a whitespace table under tests/golden (comment lines skipped)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def paper_sets():
    """Table 2 parameter sets as oracle models and contracts."""
    from oracle import Contract, NTSModel, PUT_AVG
    out = {}
    for r in read_table("table2_parameter_sets.txt"):
        name = r[0]
        v = [float(x) for x in r[1:]]
        m = NTSModel(alpha=v[0], lam=v[1], delta=v[2], eta=(v[3], v[4]),
                     rho=(v[5], v[6], v[7]), r=v[8])
        out[name] = (m, Contract(PUT_AVG, v[10], v[9]))
    return out


def oracle_inputs(w):
    """Oracle model/grid/contract for a workloads.Workload."""
    import oracle as O
    m = O.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    g = O.Grid(w.n, half_width=w.half_width)
    c = O.Contract(O.PUT_AVG, w.strike, w.maturity)
    return m, g, c


def gpu_solver(w, payoff=0, **kw):
    """CUDA-path Solver (through the C ABI) for a workloads.Workload."""
    from paper_2511_02700_gb300 import binding as B
    prec = B.PIDE2D_FP64 if w.precision == "fp64" else B.PIDE2D_FP32_BULK
    grid = B.make_grid(w.n, prec, w.sl_order, half_width=w.half_width)
    model = B.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    contract = B.make_contract(payoff, w.strike, w.maturity)
    return B.Solver(grid, model, contract, w.steps, theta=w.theta, tol=w.tol, **kw)


def gpu_job(w, payoff=0):
    """pide2d_job (C ABI batch entry) for a workloads.Workload."""
    from paper_2511_02700_gb300 import binding as B
    prec = B.PIDE2D_FP64 if w.precision == "fp64" else B.PIDE2D_FP32_BULK
    grid = B.make_grid(w.n, prec, w.sl_order, half_width=w.half_width)
    model = B.model_from_subordinated_bm(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    contract = B.make_contract(payoff, w.strike, w.maturity)
    return B.make_job(grid, model, contract, w.steps, theta=w.theta, tol=w.tol)

