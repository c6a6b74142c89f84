"""The price-space jump operator through the CUDA path against the
price-space oracle (the paper's own grid and transfers, Secs. 3.2.2, 4):
weights and rates on the z-lattice, and B_w V = T_out I~ C T_in V on random
fields and on the payoff, FP64 to 1e-10 and FP32-bulk to 1e-5 relative (at
the nodes below y_out, which the paper fills by linear extrapolation, the
bound carries that extrapolation's amplification)."""
import numpy as np
import pytest

from conftest import paper_sets
from oracle.price_space import PriceGrid, PriceSpaceOperators

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SETS = {"VG1": (5.0, 2.1410), "NIG1": (7.0, 0.8807), "NIG0": (6.0, 0.4172)}


def _operator(name, n, precision):
    from paper_2511_02700_gb300 import binding as B
    mo, co = paper_sets()[name]
    xm, ziii = SETS[name]
    pg = PriceGrid(n, co.strike, xm * co.strike, ziii)
    model = B.make_model(mo.alpha, mo.delta, mo.lam, mo.eta, mo.rho, mo.r)
    prec = B.PIDE2D_FP64 if precision == "fp64" else B.PIDE2D_FP32_BULK
    pj = B.PriceJump(pg.x, pg.n_z, pg.h_z, pg.ny_minus, pg.ny_plus, model, precision=prec)
    return pg, PriceSpaceOperators(mo, pg), pj


@pytest.mark.parametrize("name", ["VG1", "NIG1"])
def test_price_space_weights_match_oracle(name):
    pg, ops, pj = _operator(name, 24, "fp64")
    om, rates = pj.weights()
    om = om.cpu().numpy()
    ref = ops.pre.omega
    nz = ref != 0
    assert np.array_equal(om != 0, nz)
    assert np.max(np.abs(om[nz] / ref[nz] - 1.0)) < 1e-11
    pre = ops.pre
    want = [pre.sum_w, pre.r_w, pre.kappa_w[0], pre.kappa_w[1], pre.a[0, 0], pre.a[0, 1], pre.a[1, 1],
            pre.b[0], pre.b[1]]
    for a, b in zip(rates, want):
        assert abs(a - b) <= 1e-11 * max(abs(b), 1e-3), (rates, want)
    pj.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("name,n", [("VG1", 24), ("NIG1", 40), ("NIG0", 16)])
def test_price_space_jump_matches_oracle(name, n, precision, tol):
    pg, ops, pj = _operator(name, n, precision)
    rng = np.random.Generator(np.random.PCG64(n))
    for V in (rng.uniform(0.0, 100.0, size=(n + 1, n + 1)),
              np.maximum(100.0 - 0.5 * (pg.x[None, :] + pg.x[:, None]), 0.0)):
        got = pj.apply(torch.from_numpy(V)).cpu().numpy()
        ref = ops.jump(V)
        scale = np.max(np.abs(ref))
        # nodes below y_out (x = 0) are linear extrapolations from y_out_0, y_out_1 (Sec. 4), which
        # amplify the transform's rounding by (y1 + y0 - 2x) / (y1 - y0) per axis
        y0, y1 = pg.y_out[0], pg.y_out[1]
        f = np.where(pg.x < y0, (y1 + y0 - 2 * pg.x) / (y1 - y0), 1.0)
        bound = tol * scale * np.outer(f, f)
        err = np.abs(got - ref)
        assert np.all(err <= bound), (name, n, precision, np.max(err / bound))
        inner = np.outer(f == 1.0, f == 1.0)
        assert np.max(err[inner]) <= tol * scale
    pj.close()


def test_price_space_rejects_bad_grids():
    from paper_2511_02700_gb300 import binding as B
    mo, _ = paper_sets()["VG1"]
    model = B.make_model(mo.alpha, mo.delta, mo.lam, mo.eta, mo.rho, mo.r)
    with pytest.raises(B.PideError):
        B.PriceJump(np.array([0.0, 1.0, 0.5, 2.0, 3.0]), 4, 0.1, 2, 10, model)      # not increasing
    with pytest.raises(B.PideError):
        B.PriceJump(np.array([1.0, 2.0, 3.0, 4.0, 5.0]), 4, 0.1, 2, 10, model)      # x[0] != 0


@pytest.mark.parametrize("name,n,precision,tol", [("VG1", 24, "fp64", 1e-8), ("NIG1", 32, "fp64", 1e-8),
                                                  ("VG1", 24, "fp32", 1e-5)])
def test_price_space_solve_matches_oracle(name, n, precision, tol):
    """Algorithm 1 in price space through the CUDA path against the oracle's
    PriceScheme on the same grid: the oracle solves each implicit system
    exactly, the CUDA path by BiCGSTAB to 1e-13, both iterate to tol 1e-12."""
    from oracle.price_space import PriceScheme
    from paper_2511_02700_gb300 import binding as B
    pg, ops, pj = _operator(name, n, precision)
    mo, co = paper_sets()[name]
    steps = n // 4
    V, st, status = pj.solve(B.make_contract(0, co.strike, co.maturity), steps, tol=1e-12)
    assert status == 0 and st.steps_done == steps
    ref = PriceScheme(mo, pg, co, steps, tol=1e-12).solve().V
    got = V.cpu().numpy()
    err = np.abs(got - ref) / np.max(np.abs(ref))
    # as for B_w V alone, the rounding of an FP32 transform is amplified at the nodes below
    # y_out (x = 0), which are linear extrapolations (Sec. 4)
    y0, y1 = pg.y_out[0], pg.y_out[1]
    f = np.where(pg.x < y0, (y1 + y0 - 2 * pg.x) / (y1 - y0), 1.0)
    inner = np.outer(f == 1.0, f == 1.0)
    msg = (name, n, precision, float(np.max(err)), float(np.max(err[inner])), float(np.max(err / np.outer(f, f))))
    assert np.max(err[inner]) <= tol, msg
    assert np.all(err <= tol * np.outer(f, f)), msg
    pj.close()


@pytest.mark.parametrize("name,col", [("VG1", 1), ("NIG1", 3)])
def test_price_space_solve_table4_fine_grid(name, col):
    """Table 4 (the paper's N_x = 800) from the CUDA path at N_x = 160 with the
    paper's grid and scheme: within 0.02 at the nine printed points."""
    from conftest import read_table
    from oracle.price_space import lagrange_matrix
    from paper_2511_02700_gb300 import binding as B
    n = 160
    pg, _, pj = _operator(name, n, "fp64")
    mo, co = paper_sets()[name]
    V, st, status = pj.solve(B.make_contract(0, co.strike, co.maturity), n // 2, tol=1e-7)
    assert status == 0
    V = V.cpu().numpy()
    dev = []
    for row in read_table("table4_prices.txt"):
        x1, x2 = float(row[0]), float(row[1])
        w1 = lagrange_matrix(pg.x, np.array([x1]), "linear")
        w2 = lagrange_matrix(pg.x, np.array([x2]), "linear")
        got = float((w2 @ V @ w1.T)[0, 0])
        dev.append(got - float(row[2 + col]))
    assert max(abs(d) for d in dev) < 0.02, (name, dev)
    pj.close()
