"""pide2d_batch_solve: many independent pricings (uneven grids) on one GPU.

Jobs of one geometry run in lockstep through the multi-job kernels, which
share their bodies with the single-solve kernels, so the batch prices must
equal the single-solve prices exactly; one small job is also checked against
the oracle at the FP32-bulk tolerance.
"""
import pytest

from conftest import gpu_job, gpu_solver, oracle_inputs
from paper_2511_02700_gb300.workloads import batch_draw, with_


def test_batch_workspace_bytes_and_arguments():
    from paper_2511_02700_gb300 import binding as B
    from paper_2511_02700_gb300 import build
    build.build()
    jobs = [gpu_job(with_(w, n=n)) for w, n in zip(batch_draw(3), (64, 256, 128))]
    one = B.pide2d_workspace_bytes(jobs[1].grid)
    nb = B.pide2d_batch_workspace_bytes(jobs, 2)
    # two lanes + the multi-job argument arrays of every theta step of the longest job (64 steps + 3)
    assert nb >= 2 * one and nb < 2 * one + 1024 * 1024
    assert B.pide2d_batch_workspace_bytes(jobs, 8) == B.pide2d_batch_workspace_bytes(jobs, 3)
    with pytest.raises(B.PideError):
        B.pide2d_batch_workspace_bytes(jobs, 0)
    bad = gpu_job(with_(batch_draw(1)[0], n=100))
    with pytest.raises(B.PideError):
        B.pide2d_batch_workspace_bytes(jobs + [bad], 2)


def _small_batch(count=24):
    out = []
    for i, w in enumerate(batch_draw(count, seed=77)):
        n = (32, 64, 128)[i % 3]
        w = with_(w, n=n, steps=n // 8)
        if i % 4 == 0:
            w = with_(w, sl_order=1)          # a second group of the same size
        out.append(w)
    return out


@pytest.mark.gpu
def test_batch_equals_single_solves():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02700_gb300 import binding as B
    ws = _small_batch()
    prices, sts, stats = B.solve_batch([gpu_job(w) for w in ws], lanes=6)
    assert all(s == 0 for s in sts), sts
    assert stats.jobs_done == len(ws) and stats.failures == 0
    cells = 0.0
    for w, p in zip(ws, prices):
        s = gpu_solver(w)
        p1, _, st1, _ = s.solve()
        s.close()
        assert p == p1, (w.name, p, p1)
        cells += st1.cell_iters
    assert stats.cell_iters == cells


@pytest.mark.gpu
def test_batch_job_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_2511_02700_gb300 import binding as B
    w = with_(batch_draw(1, seed=5)[0], n=64, steps=16)
    prices, sts, _ = B.solve_batch([gpu_job(w), gpu_job(with_(w, n=32, steps=8))], lanes=2)
    m, g, c = oracle_inputs(w)
    ref = O.Scheme(m, g, c, w.steps, theta=w.theta, tol=w.tol, sl_order=w.sl_order).solve().price
    assert sts == [0, 0]
    assert abs(prices[0] - ref) <= 1e-5 * abs(ref), (prices[0], ref)


@pytest.mark.gpu
def test_batch_reports_iteration_cap_per_job():
    """kmax = 20 with an unreachable tolerance for half of the jobs: those
    report NOT_CONVERGED (4) with the same prices as single solves under the
    same cap; the others converge normally."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02700_gb300 import binding as B
    ws = [with_(w, n=32, steps=4, tol=(1e-30 if i % 2 else 1e-8)) for i, w in enumerate(batch_draw(6, seed=9))]
    prices, sts, stats = B.solve_batch([gpu_job(w) for w in ws], lanes=4, kmax=20)
    assert sts == [0, 4, 0, 4, 0, 4], sts
    assert stats.failures == 3 and stats.jobs_done == 6
    for w, p in zip(ws, prices):
        s = gpu_solver(w, kmax=20, host_loop=True)
        p1, _, _, st1 = s.solve()
        s.close()
        assert p == p1 and st1 == (4 if w.tol < 1e-20 else 0)



@pytest.mark.gpu
def test_batch_fp32_bulk_prices_within_1e5_of_fp64():
    """The benchmark's batch workload (its first 16 draws: N in {128, 256, 512},
    N/4 steps, tol 1e-8) in FP32-bulk through the batch path, against the same
    jobs solved one by one in FP64 (itself at parity with the oracle to 1e-10):
    every price within the FP32-bulk bound of 1e-5 relative."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02700_gb300 import binding as B
    ws = batch_draw(512)[:16]
    prices, sts, _ = B.solve_batch([gpu_job(w) for w in ws], lanes=16)
    assert all(s == 0 for s in sts), sts
    errs = []
    for w, p32 in zip(ws, prices):
        s = gpu_solver(with_(w, precision="fp64"))
        p64, _, st, _ = s.solve()
        s.close()
        errs.append(abs(p32 - p64) / abs(p64))
    assert max(errs) <= 1e-5, [(w.name, e) for w, e in zip(ws, errs) if e > 1e-5]


@pytest.mark.gpu
def test_batch_launch_shape_trials_report_and_keep_prices():
    """The timed trials pick a launch shape per geometry group (FFT units per
    block, jobs per chunk) and report it; the shape changes how FFT units
    share blocks, not what they compute, so the prices agree with the fixed
    single-job shapes (up to a stop decision at the rounding level)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02700_gb300 import binding as B
    ws = [with_(w, n=(64, 128)[i % 2], steps=8) for i, w in enumerate(batch_draw(40, seed=21))]
    jobs = [gpu_job(w) for w in ws]
    p_fixed, s_fixed, st_fixed = B.solve_batch(jobs, lanes=40, fixed_shapes=True)
    p_tuned, s_tuned, st_tuned = B.solve_batch(jobs, lanes=40)
    assert all(x == 0 for x in s_fixed + s_tuned)
    assert st_fixed.tuned == 0
    tun = st_tuned.tuning()
    assert st_tuned.tuned == 2 and sorted(t["n"] for t in tun) == [64, 128]
    for t in tun:
        assert t["units_per_block"] >= 1 and 1 <= t["lanes"] <= 20 and t["us_per_job_column_pass"] > 0
    for a, b in zip(p_fixed, p_tuned):
        assert abs(a - b) <= 1e-10 * abs(b), (a, b)
