"""pide2d_jump_static: the jump sum for callers that cannot allocate device
memory (for example a plugin whose host process owns all device memory, or a
service that must not call cudaMalloc after start-up).  It keeps its scratch
in a fixed device array inside the library instead of a caller workspace.

Checked against the regular entry point pide2d_apply_jump (caller-owned
workspace) on the same inputs, on two calls in a row, with the FP64 jump
tolerance used by the other parity tests.  Collected last on purpose.
"""
import numpy as np
import pytest

from conftest import gpu_solver
from paper_2511_02700_gb300.workloads import Workload, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_static_scratch_jump_matches_workspace_entry_point():
    from paper_2511_02700_gb300 import binding as B
    n = 64
    w = Workload("noalloc", n=n, steps=4, alpha=0.5, precision="fp64")
    s = gpu_solver(w)
    omega, rates = s.weights()                 # device weights from the regular path
    sum_w = float(rates[0])
    stream = torch.cuda.current_stream()
    for call in range(2):                      # two calls in a row share the static scratch
        U = torch.from_numpy(random_field(n, seed=500 + call)).cuda()
        ref = s.apply_jump(U, 0.0, far_field=False).cpu().numpy()
        out = torch.zeros_like(U)
        B.pide2d_jump_static(n, omega.data_ptr(), U.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = sum_w * float(U.abs().max())
        assert np.abs(got[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() <= 1e-13 * scale
        # entries outside the interior are left as they were
        assert np.all(got[0, :] == 0) and np.all(got[:, 0] == 0) and np.all(got[-1, :] == 0)
    s.close()


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    from paper_2511_02700_gb300 import binding as B
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PideError) as e:
        B.pide2d_jump_static(512, t.data_ptr(), t.data_ptr(), t.data_ptr(), 0)
    assert "ERR_ARG" in str(e.value) and "256" in str(e.value)
