"""pide2d_adjoint: the discrete adjoint of the time loop.

The gradient of V^{N_t}(S0) with respect to (sigma1, sigma2, corr, kappa,
beta1, beta2) is checked against central finite differences of the CUDA
path's own prices (FP64 mode, step 1e-4) and against the FP64 oracle's
central-difference gradient; checkpoint intervals must not change it, the
final values must survive it, and the torch.autograd wrapper must return
it.
"""
import math

import numpy as np
import pytest

from conftest import gpu_solver, oracle_inputs
from paper_2511_02700_gb300.workloads import Workload, with_

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PARAMS = ("sigma1", "sigma2", "corr", "kappa", "beta1", "beta2")


def _params(w):
    return {"sigma1": w.sigma[0], "sigma2": w.sigma[1], "corr": w.corr, "kappa": w.kappa,
            "beta1": w.beta[0], "beta2": w.beta[1]}


def _with_params(w, p):
    return with_(w, sigma=(p["sigma1"], p["sigma2"]), corr=p["corr"], kappa=p["kappa"],
                 beta=(p["beta1"], p["beta2"]))


def adjoint_gradient(w, interval=4, payoff=0, **kw):
    from paper_2511_02700_gb300 import binding as B
    s = gpu_solver(w, payoff=payoff, **kw)
    s.record(interval=interval, ndirs=6)
    price, V, _, st = s.solve(values=True)
    assert st == 0
    dirs = B.subordinated_bm_directions(w.alpha, w.kappa, w.beta, w.sigma, w.corr)
    g, ast = s.adjoint(dirs)
    V_after = s.values()
    s.close()
    assert ast == 0
    return dict(zip(PARAMS, g)), price, V, V_after


def gpu_fd_gradient(w, eps=1e-4, payoff=0, **kw):
    base = _params(w)
    out = {}
    for p in PARAMS:
        up, dn = dict(base), dict(base)
        up[p] += eps
        dn[p] -= eps
        pu = gpu_solver(_with_params(w, up), payoff=payoff, **kw).solve()[0]
        pd = gpu_solver(_with_params(w, dn), payoff=payoff, **kw).solve()[0]
        out[p] = (pu - pd) / (2 * eps)
    return out


def _close(a, b, rel, floor):
    scale = max(abs(v) for v in b.values())
    for p in PARAMS:
        assert abs(a[p] - b[p]) <= rel * abs(b[p]) + floor * scale, (p, a[p], b[p], a, b)


@pytest.mark.parametrize("alpha,sl", [(0.25, 3), (0.5, 1)])
def test_adjoint_matches_finite_differences_fp64(alpha, sl):
    w = Workload("adj", n=32, steps=8, alpha=alpha, tol=1e-13, precision="fp64", sl_order=sl)
    g, price, V, V_after = adjoint_gradient(w)
    fd = gpu_fd_gradient(w)
    _close(g, fd, 1e-5, 1e-7)
    assert torch.equal(V, V_after)          # the final values are put back


def test_adjoint_without_damping_and_theta_half_first_step():
    """No damped start: the first theta step has an explicit part, so the
    payoff V^0 enters the gradient through B V^0 and D V^0."""
    w = Workload("adj_nd", n=32, steps=6, alpha=0.25, tol=1e-13, precision="fp64")
    g, _, _, _ = adjoint_gradient(w, damping=False)
    fd = gpu_fd_gradient(w, damping=False)
    _close(g, fd, 1e-5, 1e-7)


def test_adjoint_matches_oracle_gradient():
    import oracle as O
    w = Workload("adj_or", n=32, steps=8, alpha=0.25, tol=1e-13, precision="fp64")
    g, _, _, _ = adjoint_gradient(w)
    _, grid, c = oracle_inputs(w)
    ref = O.price_gradient_fd(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r, grid, c, w.steps, theta=w.theta,
                              tol=1e-13, sl_order=w.sl_order, eps=1e-4)
    _close(g, ref, 1e-5, 1e-7)


def test_checkpoint_interval_does_not_change_the_gradient():
    w = Workload("adj_ck", n=32, steps=10, alpha=0.5, tol=1e-12, precision="fp64")
    ref, _, _, _ = adjoint_gradient(w, interval=1)
    for interval in (3, 16):
        g, _, _, _ = adjoint_gradient(w, interval=interval)
        assert g == ref, (interval, g, ref)


def test_fp32_bulk_adjoint_close_to_fp64():
    w = Workload("adj32", n=64, steps=16, alpha=0.25, tol=1e-10, precision="fp64")
    g64, _, _, _ = adjoint_gradient(w)
    g32, _, _, _ = adjoint_gradient(with_(w, precision="fp32", tol=1e-8))
    _close(g32, g64, 1e-4, 1e-5)


def test_single_asset_gradient_ignores_asset_two():
    w = Workload("adj_sa", n=32, steps=8, alpha=0.25, tol=1e-13, precision="fp64")
    g, _, _, _ = adjoint_gradient(w, payoff=2)
    for p in ("sigma2", "corr", "beta2"):
        assert abs(g[p]) < 0.01 * abs(g["sigma1"]), g


def test_autograd_function_returns_the_adjoint_gradient():
    from paper_2511_02700_gb300 import binding as B
    w = Workload("adj_ag", n=32, steps=8, alpha=0.25, tol=1e-13, precision="fp64")
    g, price, _, _ = adjoint_gradient(w, interval=16)
    grid = B.make_grid(w.n, B.PIDE2D_FP64, w.sl_order, half_width=w.half_width)
    contract = B.make_contract(0, w.strike, w.maturity)
    p = torch.tensor([w.sigma[0], w.sigma[1], w.corr, w.kappa, w.beta[0], w.beta[1]], dtype=torch.float64,
                     requires_grad=True)
    Price = B.price_function()
    v = Price.apply(p, w.alpha, w.r, grid, contract, w.steps, w.theta, w.tol, 16)
    v.backward()
    assert float(v.detach()) == price
    assert np.allclose(p.grad.numpy(), [g[k] for k in PARAMS], rtol=0, atol=0)


def test_adjoint_requires_tape_and_finished_solve():
    from paper_2511_02700_gb300 import binding as B
    w = Workload("adj_err", n=16, steps=4, alpha=0.25, tol=1e-12, precision="fp64")
    dirs = B.subordinated_bm_directions(w.alpha, w.kappa, w.beta, w.sigma, w.corr)
    s = gpu_solver(w)
    s.solve()
    with pytest.raises(B.PideError) as e:
        s.adjoint(dirs)
    assert "tape" in str(e.value)
    s2 = gpu_solver(w)
    s2.step()
    with pytest.raises(B.PideError):
        s2.record()
    s3 = gpu_solver(w)
    s3.record(interval=2, ndirs=2)
    with pytest.raises(B.PideError) as e:
        s3.adjoint(dirs[:2])
    assert "finished" in str(e.value)
    s3.solve()
    with pytest.raises(B.PideError):
        s3.adjoint(dirs)                       # more directions than the tape holds
    g, st = s3.adjoint(dirs[:2])
    assert st == 0 and all(math.isfinite(x) for x in g)


def test_workload_adjoint_entry_equals_composed_directions():
    """pide2d_adjoint_workload (the Table A5 tangents inside the library)
    against pide2d_adjoint along tangents composed here by hand from the
    mapping lambda = (1 - alpha)/kappa, delta = lambda^(1-alpha)/Gamma(1-alpha),
    eta = beta, rho = [[s1^2, c s1 s2], [c s1 s2, s2^2]]."""
    from paper_2511_02700_gb300 import binding as B
    w = Workload("adjw", n=32, steps=8, alpha=0.5, tol=1e-13, precision="fp64")
    s = gpu_solver(w)
    s.record(interval=4, ndirs=6)
    s.solve()
    lam = (1.0 - w.alpha) / w.kappa
    delta = lam ** (1.0 - w.alpha) / math.gamma(1.0 - w.alpha)
    s1, s2, c = w.sigma[0], w.sigma[1], w.corr
    z = (0.0, 0.0)
    dirs = [B.make_model(0.0, 0.0, 0.0, z, (2 * s1, c * s2, 0.0), 0.0),
            B.make_model(0.0, 0.0, 0.0, z, (0.0, c * s1, 2 * s2), 0.0),
            B.make_model(0.0, 0.0, 0.0, z, (0.0, s1 * s2, 0.0), 0.0),
            B.make_model(0.0, -(1.0 - w.alpha) * delta / w.kappa, -lam / w.kappa, z, (0.0, 0.0, 0.0), 0.0),
            B.make_model(0.0, 0.0, 0.0, (1.0, 0.0), (0.0, 0.0, 0.0), 0.0),
            B.make_model(0.0, 0.0, 0.0, (0.0, 1.0), (0.0, 0.0, 0.0), 0.0)]
    g_ref, _ = s.adjoint(dirs)
    wl = B.make_workload(w.alpha, w.kappa, w.beta, w.sigma, w.corr, w.r)
    g, st = s.adjoint_workload(wl)
    assert st == 0
    scale = max(abs(x) for x in g_ref)
    assert max(abs(a - b) for a, b in zip(g, g_ref)) <= 1e-12 * scale, (g, g_ref)
    # a workload that is not the handle's model is refused
    other = B.make_workload(w.alpha, w.kappa * 1.01, w.beta, w.sigma, w.corr, w.r)
    with pytest.raises(B.PideError) as e:
        s.adjoint_workload(other)
    assert "ERR_ARG" in str(e.value)
    s.close()
