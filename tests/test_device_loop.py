"""The fixed-point loop of each theta step (eqs. 3.24-3.25) runs either on
the device (a CUDA-graph while-node whose check kernel evaluates the
stopping rule) or on the host (one residual read per iteration).  Both run
the same kernels in the same order, so values, prices and iteration counts
must agree exactly; the stopping rule must also end the device loop at
kmax."""
import numpy as np
import pytest

from conftest import gpu_solver
from paper_2511_02700_gb300.workloads import PLAIN_FP64_128, Workload, with_

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("w", [PLAIN_FP64_128,
                               Workload("dl32", n=256, steps=64, alpha=0.75, tol=1e-8, precision="fp32"),
                               Workload("dl32lin", n=128, steps=16, alpha=0.5, tol=1e-8, precision="fp32",
                                        sl_order=1)],
                         ids=lambda w: w.name)
def test_device_loop_equals_host_loop(w):
    sd = gpu_solver(w)
    sh = gpu_solver(w, host_loop=True)
    pd, Vd, std, sd_st = sd.solve(values=True)
    ph, Vh, sth, sh_st = sh.solve(values=True)
    assert sd_st == 0 and sh_st == 0
    assert pd == ph
    assert torch.equal(Vd, Vh)
    assert std.fp_iters_total == sth.fp_iters_total
    assert std.fp_iters_max == sth.fp_iters_max
    assert std.cell_iters == sth.cell_iters
    assert std.steps_done == sth.steps_done == w.steps
    assert std.last_resid == sth.last_resid
    sd.close()
    sh.close()


def test_device_loop_step_api_reports_counts():
    w = with_(PLAIN_FP64_128, n=64, steps=6)
    sd = gpu_solver(w)
    sh = gpu_solver(w, host_loop=True)
    for _ in range(w.steps):
        kd, rd, std = sd.step()
        kh, rh, sth = sh.step()
        assert (kd, rd, std) == (kh, rh, sth)
        assert 1 <= kd < 100 and rd < w.tol
    assert torch.equal(sd.values(), sh.values())


@pytest.mark.parametrize("host_loop", [False, True])
def test_iteration_cap_ends_the_loop(host_loop):
    """kmax = 2 with an unreachable tolerance: every theta step stops after
    two iterations and the solve reports NOT_CONVERGED (4), with the state
    advanced by the last iterate."""
    w = Workload("cap", n=64, steps=4, alpha=0.5, tol=1e-30, precision="fp64")
    s = gpu_solver(w, kmax=2, host_loop=host_loop)
    p, V, st, status = s.solve(values=True)
    assert status == 4
    assert st.fp_iters_total == 2 * (4 + 3)            # damped first step = 4 theta steps
    assert st.fp_iters_max == 8
    assert np.isfinite(p) and torch.isfinite(V).all()
    s.close()


def test_iteration_cap_same_state_in_both_loops():
    w = Workload("cap2", n=64, steps=4, alpha=0.25, tol=1e-30, precision="fp32")
    a = gpu_solver(w, kmax=3)
    b = gpu_solver(w, kmax=3, host_loop=True)
    pa, Va, _, sa = a.solve(values=True)
    pb, Vb, _, sb = b.solve(values=True)
    assert sa == sb == 4 and pa == pb and torch.equal(Va, Vb)
