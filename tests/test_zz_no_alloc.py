"""pide2d_jump_static: the jump sum for callers that cannot allocate device
memory (for example a plugin whose host process owns all device memory, or a
service that must not call cudaMalloc after start-up).  It keeps its scratch
in a fixed device array inside the library instead of a caller workspace.

Checked on two calls in a row (the calls share the static scratch) at the
smallest size, a middle size and the largest size (n = 256 fills the whole
scratch), with the FP64 jump tolerance of the other parity tests:
* against the FP64 CPU oracle's FFT correlation with a zero far field, both
  sides using the oracle's weights;
* against the regular entry point pide2d_apply_jump (caller-owned workspace),
  both sides using the weights the GPU precompute produced.
Collected last on purpose.
"""
import numpy as np
import pytest

from conftest import gpu_solver, oracle_inputs
from paper_2511_02700_gb300.workloads import Workload, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402


@pytest.mark.parametrize("n", [8, 64, 256])
def test_static_scratch_jump_matches_oracle_and_workspace_entry_point(n):
    from paper_2511_02700_gb300 import binding as B
    w = Workload("noalloc", n=n, steps=4, alpha=0.5, precision="fp64")
    s = gpu_solver(w)
    omega_gpu, rates = s.weights()             # device weights from the regular path
    m, g, c = oracle_inputs(w)
    pre = O.precompute(m, g)
    omega_ref = torch.from_numpy(pre.omega).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):                      # two calls in a row share the static scratch
        Uh = random_field(n, seed=500 + 10 * n + call)
        U = torch.from_numpy(Uh).cuda()
        # against the oracle, with the oracle's weights on both sides
        out = torch.zeros_like(U)
        B.pide2d_jump_static(n, omega_ref.data_ptr(), U.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = O.jump_fft(g, pre.omega, O.extend(g, c, m.r, Uh[1:-1, 1:-1], 0.0, far=False))
        scale = pre.sum_w * float(np.abs(Uh).max())
        assert np.abs(got[1:-1, 1:-1] - ref).max() <= 1e-13 * scale
        # entries outside the interior are left as they were
        assert np.all(got[0, :] == 0) and np.all(got[:, 0] == 0) and np.all(got[-1, :] == 0)
        assert np.all(got[:, -1] == 0)
        # against the workspace entry point, with the GPU's weights on both sides
        out2 = torch.zeros_like(U)
        B.pide2d_jump_static(n, omega_gpu.data_ptr(), U.data_ptr(), out2.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        ref2 = s.apply_jump(U, 0.0, far_field=False).cpu().numpy()
        got2 = out2.cpu().numpy()
        assert np.abs(got2[1:-1, 1:-1] - ref2[1:-1, 1:-1]).max() <= 1e-13 * float(rates[0]) * float(np.abs(Uh).max())
    s.close()


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    from paper_2511_02700_gb300 import binding as B
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PideError) as e:
        B.pide2d_jump_static(512, t.data_ptr(), t.data_ptr(), t.data_ptr(), 0)
    assert "ERR_ARG" in str(e.value) and "256" in str(e.value)
