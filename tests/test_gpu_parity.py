"""GPU parity: the CUDA path, called through the C ABI, against the FP64
CPU oracle on the same seeded inputs.

Tolerances: FP64 mode 1e-10 relative (at the valuation node and in
max-norm over the region of interest, relative to the max-norm of the
oracle there); FP32-bulk mode 1e-5 relative.  Operator checks (weights,
jump sum) use bounds derived from the arithmetic: FP64 quadrature of the
weights agrees to ~1e-13, the FP64 FFT correlation to ~1e-13 of
sum(w) max|U|, the FP32 one to ~1e-6 of it.
"""
import math

import numpy as np
import pytest

from conftest import gpu_solver, oracle_inputs
from paper_2511_02700_gb300.workloads import PLAIN_FP64_128, Workload, random_field, with_

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402


def roi_mask(n, half_width=2.5):
    s = math.log(100.0) - half_width + np.arange(n + 1) * (2 * half_width / n)
    S = np.exp(s)
    m1 = (S <= 300.0)
    M = np.outer(m1, m1)
    M[0, :] = M[-1, :] = M[:, 0] = M[:, -1] = False
    return M


@pytest.mark.parametrize("n,alpha", [(16, 0.25), (64, 0.5), (128, 0.25), (128, 0.75), (1024, 0.75)])
def test_weights_and_rates_match_oracle(n, alpha):
    w = Workload("w", n=n, steps=n // 4, alpha=alpha)
    s = gpu_solver(w)
    om, rates = s.weights()
    om = om.cpu().numpy()
    m, g, _ = oracle_inputs(w)
    pre = O.precompute(m, g)
    nz = pre.omega != 0
    assert np.array_equal(om != 0, nz)
    assert np.max(np.abs(om[nz] / pre.omega[nz] - 1.0)) < 1e-11
    ref = [pre.sum_w, pre.r_w, pre.kappa_w[0], pre.kappa_w[1], pre.a[0, 0], pre.a[0, 1], pre.a[1, 1],
           pre.b[0], pre.b[1]]
    r = rates.numpy()
    for a, b in zip(r, ref):
        assert abs(a - b) <= 1e-11 * max(abs(b), 1e-3), (r, ref)


@pytest.mark.parametrize("precision,n", [("fp64", 8), ("fp64", 16), ("fp64", 64), ("fp64", 256),
                                         ("fp32", 16), ("fp32", 128), ("fp32", 512)])
@pytest.mark.parametrize("far", [1, 0])
def test_jump_operator_matches_oracle(precision, n, far):
    w = Workload("j", n=n, steps=4, alpha=0.5, precision=precision)
    s = gpu_solver(w)
    U = random_field(n, seed=n + 7 * far)
    tau = 0.37
    B_gpu = s.apply_jump(torch.from_numpy(U), tau, far_field=bool(far)).cpu().numpy()[1:-1, 1:-1]
    m, g, c = oracle_inputs(w)
    pre = O.precompute(m, g)
    Ue = O.extend(g, c, m.r, U[1:-1, 1:-1], tau, far=bool(far))
    B_ref = O.jump_fft(g, pre.omega, Ue)
    scale = pre.sum_w * np.abs(Ue).max()
    tol = 1e-13 if precision == "fp64" else 2e-6
    err = np.abs(B_gpu - B_ref).max()
    assert err <= tol * scale, (err, scale)


@pytest.mark.parametrize("n,alpha,sl", [(16, 0.25, 3), (16, 0.75, 1), (32, 0.5, 3), (64, 0.25, 1),
                                        (64, 0.75, 3)])
def test_fp64_solve_matches_oracle(n, alpha, sl):
    w = Workload("s", n=n, steps=max(4, n // 4), alpha=alpha, tol=1e-13, sl_order=sl)
    s = gpu_solver(w)
    price, V, stats, st = s.solve(values=True)
    assert st == 0
    V = V.cpu().numpy()
    m, g, c = oracle_inputs(w)
    ref = O.Scheme(m, g, c, w.steps, theta=w.theta, tol=w.tol, sl_order=sl).solve()
    scale = np.abs(ref.V).max()
    assert np.abs(V - ref.V).max() <= 1e-10 * scale
    assert abs(price - ref.price) <= 1e-10 * abs(ref.price)


def test_plain_fp64_128_workload():
    """The 128^2, 32-step, tol 1e-10 FP64 workload: price and ROI max-norm."""
    w = PLAIN_FP64_128
    s = gpu_solver(w)
    price, V, stats, st = s.solve(values=True)
    V = V.cpu().numpy()
    m, g, c = oracle_inputs(w)
    ref = O.Scheme(m, g, c, w.steps, theta=w.theta, tol=w.tol, sl_order=w.sl_order).solve()
    roi = roi_mask(w.n)
    scale = np.abs(ref.V[roi]).max()
    assert abs(price - ref.price) <= 1e-10 * abs(ref.price), (price, ref.price)
    assert np.abs(V - ref.V)[roi].max() <= 1e-10 * scale
    assert stats.steps_done == w.steps


@pytest.mark.parametrize("n,alpha,sl", [(64, 0.25, 3), (128, 0.5, 3), (64, 0.5, 1)])
def test_fp32_bulk_solve_matches_oracle(n, alpha, sl):
    """FP32-bulk solves against the FP64 oracle, with the cubic and the linear
    departure interpolation (the preparation's two-node windows of 4 x 5 and
    2 x 3 taps)."""
    w = Workload("f", n=n, steps=n // 4, alpha=alpha, tol=1e-10, precision="fp32", sl_order=sl)
    s = gpu_solver(w)
    price, V, stats, st = s.solve(values=True)
    V = V.cpu().numpy()
    m, g, c = oracle_inputs(w)
    ref = O.Scheme(m, g, c, w.steps, theta=w.theta, tol=w.tol, sl_order=w.sl_order).solve()
    roi = roi_mask(n)
    scale = np.abs(ref.V[roi]).max()
    assert abs(price - ref.price) <= 1e-5 * abs(ref.price), (price, ref.price)
    assert np.abs(V - ref.V)[roi].max() <= 1e-5 * scale


@pytest.mark.parametrize("payoff", [1, 2])
def test_other_payoffs_fp64(payoff):
    w = Workload("p", n=32, steps=8, alpha=0.5, tol=1e-13)
    s = gpu_solver(w, payoff=payoff)
    price, V, stats, st = s.solve(values=True)
    m, g, _ = oracle_inputs(w)
    c = O.Contract(payoff, w.strike, w.maturity)
    ref = O.Scheme(m, g, c, w.steps, tol=w.tol, sl_order=w.sl_order).solve()
    assert np.abs(V.cpu().numpy() - ref.V).max() <= 1e-10 * np.abs(ref.V).max()


def test_step_api_and_state_errors():
    from paper_2511_02700_gb300 import binding as B
    w = Workload("st", n=16, steps=3, alpha=0.25, tol=1e-12)
    s = gpu_solver(w)
    k1, r1, st1 = s.step()      # damped first step: four substeps
    assert st1 == 0 and k1 >= 4 and r1 < w.tol
    for _ in range(2):
        k, r, st = s.step()
        assert st == 0 and 1 <= k < 100
    with pytest.raises(B.PideError) as e:
        s.step()
    assert "ERR_STATE" in str(e.value)


@pytest.mark.parametrize("n,alpha", [(512, 0.5), (1024, 0.25), (1024, 0.75)])
def test_fp32_bulk_matches_fp64_on_large_grids(n, alpha):
    """Convergence-sweep sizes (tol 1e-8, N/4 steps): the FP32-bulk solve
    agrees with the FP64 solve (itself oracle-pinned on smaller grids) to
    1e-5 relative at S0 and in max-norm over the region of interest."""
    w64 = Workload("big", n=n, steps=n // 4, alpha=alpha, tol=1e-8, precision="fp64")
    p64, V64, _, _ = gpu_solver(w64).solve(values=True)
    p32, V32, _, _ = gpu_solver(with_(w64, precision="fp32")).solve(values=True)
    V64, V32 = V64.cpu().numpy(), V32.cpu().numpy()
    roi = roi_mask(n)
    assert abs(p32 - p64) <= 1e-5 * abs(p64), (p32, p64)
    assert np.abs(V32 - V64)[roi].max() <= 1e-5 * np.abs(V64[roi]).max()


@pytest.mark.slow
def test_jump_operator_full_size_sampled():
    """4096^2 grid, 8192^2 transforms, FP32-bulk -- the launch configuration of
    the benchmark: B_w U at 16 sampled interior nodes against the oracle's
    direct sums (eq. 3.10) with the oracle's weights (8-point cell rule)."""
    n = 4096
    w = Workload("full", n=n, steps=1024, alpha=0.5, precision="fp32")
    s = gpu_solver(w)
    U = random_field(n, seed=4096)
    tau = 0.25
    B_gpu = s.apply_jump(torch.from_numpy(U), tau, far_field=True).cpu().numpy()
    m, g, c = oracle_inputs(w)
    pre = O.precompute(m, g, r2_order=8)
    Ue = O.extend(g, c, m.r, U[1:-1, 1:-1], tau)          # nodes -N/2-1 .. N+N/2
    rng = np.random.default_rng(11)
    nodes = [(int(a), int(b)) for a, b in rng.integers(1, n, size=(16, 2))] + [(1, 1), (n - 1, n - 1), (n // 2, n // 2)]
    wsum = pre.sum_w
    for (m1, m2) in nodes:
        # midpoints j = m + l, l in [-N/2, N/2): nodes j-1..j+2 -> ext index j - 1 + N/2 + 1 ..
        o = n // 2 + 1
        lo1, lo2 = m1 - n // 2, m2 - n // 2
        blk = Ue[lo2 - 1 + o: lo2 + n + 2 + o, lo1 - 1 + o: lo1 + n + 2 + o]
        mid = O.midpoints(blk)                               # (n) x (n) midpoints m + l
        ref = float(np.sum(pre.omega * mid))
        assert abs(B_gpu[m2, m1] - ref) <= 2e-6 * wsum * np.abs(Ue).max(), (m1, m2, B_gpu[m2, m1], ref)


def test_greeks_match_oracle():
    """Delta/Gamma fields (Sec. 4 central differences) of the FP64 solve."""
    w = Workload("g", n=64, steps=16, alpha=0.5, tol=1e-13)
    s = gpu_solver(w)
    s.solve()
    G = {k: v.cpu().numpy()[1:-1, 1:-1] for k, v in s.greeks().items()}
    m, g, c = oracle_inputs(w)
    ref = O.Scheme(m, g, c, w.steps, tol=w.tol, sl_order=w.sl_order).solve()
    R = O.greeks(g, ref.V)
    for k in R:
        assert np.abs(G[k] - R[k]).max() <= 1e-9 * (np.abs(R[k]).max() + 1e-12), k


def test_vg0_wide_domain_fp64_matches_oracle():
    """VG0 (alpha = 0, z_max^III = 11.5): half-width 11.5 log units."""
    from conftest import paper_sets
    from paper_2511_02700_gb300 import binding as B
    mo, co = paper_sets()["VG0"]
    n = 64
    grid = B.make_grid(n, B.PIDE2D_FP64, 3, half_width=11.5)
    model = B.make_model(mo.alpha, mo.delta, mo.lam, mo.eta, mo.rho, mo.r)
    s = B.Solver(grid, model, B.make_contract(0, co.strike, co.maturity), n // 4, tol=1e-13)
    price, V, _, _ = s.solve(values=True)
    ref = O.Scheme(mo, O.Grid(n, half_width=11.5), co, n // 4, tol=1e-13, sl_order=3).solve()
    assert np.abs(V.cpu().numpy() - ref.V).max() <= 1e-10 * np.abs(ref.V).max()


@pytest.mark.slow
@pytest.mark.parametrize("name,col,half_width", [("VG0", 0, 11.5), ("VG1", 1, 2.5), ("NIG0", 2, 2.5),
                                                 ("NIG1", 3, 2.5)])
def test_table4_prices_on_fine_grids(name, col, half_width):
    """Table 4 (nine points near (K, K)) through the CUDA path: 2048^2 log
    grid, FP32-bulk, N/2 time steps (the paper's N_t = N_x/2), cubic SL, values
    off the grid by bicubic interpolation of the log-grid solution.  Bands: 4e-3
    (8e-3 for NIG0) -- the printed values carry the paper's own grid error."""
    from conftest import paper_sets, read_table
    from paper_2511_02700_gb300 import binding as B
    from scipy.interpolate import RectBivariateSpline
    mo, co = paper_sets()[name]
    n = 2048
    grid = B.make_grid(n, B.PIDE2D_FP32_BULK, 3, half_width=half_width)
    model = B.make_model(mo.alpha, mo.delta, mo.lam, mo.eta, mo.rho, mo.r)
    s = B.Solver(grid, model, B.make_contract(0, co.strike, co.maturity), n // 2, tol=1e-8)
    price, V, _, _ = s.solve(values=True)
    V = V.cpu().numpy()
    sg = math.log(100.0) - half_width + np.arange(n + 1) * (2 * half_width / n)
    spl = RectBivariateSpline(sg, sg, V.T, kx=3, ky=3)     # V is [m2, m1]
    # the paper prints NIG0 from a 400-point grid (the others from 800 points,
    # Sec. 4), so its own discretisation error allows a wider band there
    tol = 8e-3 if name == "NIG0" else 4e-3
    dev = []
    for row in read_table("table4_prices.txt"):
        x1, x2 = float(row[0]), float(row[1])
        got = float(spl.ev(math.log(x1), math.log(x2)))
        dev.append((x1, x2, round(got, 5), float(row[2 + col]), round(got - float(row[2 + col]), 5)))
    assert max(abs(d[-1]) for d in dev) < tol, (name, dev)
