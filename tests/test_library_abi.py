"""CPU checks of the C ABI: the library builds/loads, exports every entry
point include/pide2d.h declares, and rejects bad arguments before touching
the GPU."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(pide2d_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2511_02700_gb300 import build, binding
    build.build()
    return binding.lib()


def test_header_declares_the_api():
    names = declared_symbols()
    for n in ("pide2d_create", "pide2d_step", "pide2d_solve", "pide2d_destroy", "pide2d_workspace_bytes",
              "pide2d_last_error", "pide2d_apply_jump", "pide2d_get_values", "pide2d_get_weights"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_workspace_bytes_and_argument_checks(lib):
    from paper_2511_02700_gb300 import binding as B
    g = B.make_grid(128, B.PIDE2D_FP64)
    nb = B.pide2d_workspace_bytes(g)
    assert nb > 128 * 128 * 8 * 10
    g32 = B.make_grid(4096, B.PIDE2D_FP32_BULK)
    assert B.pide2d_workspace_bytes(g32) < 4 * 1024 ** 3
    with pytest.raises(B.PideError):
        B.pide2d_workspace_bytes(B.make_grid(100))          # not a power of two
    # FP64 mode runs every size up to 4096 (8192-point FP64 transforms)
    assert B.pide2d_workspace_bytes(B.make_grid(4096, B.PIDE2D_FP64)) < 8 * 1024 ** 3
    with pytest.raises(B.PideError):
        B.pide2d_workspace_bytes(B.make_grid(8192, B.PIDE2D_FP64))
    model = B.model_from_subordinated_bm(0.25, 0.5, (-0.1, -0.05), (0.2, 0.25), 0.3, 0.03)
    contract = B.make_contract()
    bad = B.model_from_subordinated_bm(0.25, 0.5, (-0.1, -0.05), (0.2, 0.25), 0.3, 0.03)
    bad.rho[1] = 1.0                                        # not positive definite
    for args, msg in [((g, bad, contract, 0.5, 1 / 32, 1e-10), "positive definite"),
                      ((g, model, contract, 0.2, 1 / 32, 1e-10), "theta"),
                      ((g, model, contract, 0.5, 0.3, 1e-10), "integer"),
                      ((g, model, contract, 0.5, 1 / 32, -1.0), "positive")]:
        with pytest.raises(B.PideError) as e:
            B.pide2d_create(*args, None, 0, nb, 0)
        assert msg in str(e.value)
    # a NULL workspace is rejected before any device call
    with pytest.raises(B.PideError) as e:
        B.pide2d_create(g, model, contract, 0.5, 1 / 32, 1e-10, None, 0, nb, 0)
    assert "ERR_WORKSPACE" in str(e.value)


def test_workload_mapping_matches_oracle_and_its_tangents(lib):
    """pide2d_model_from_workload (Table A5 in the library) against the
    oracle's mapping, and pide2d_workload_directions against central
    differences of the library's own mapping (host-only calls, no GPU)."""
    import oracle as O
    from paper_2511_02700_gb300 import binding as B
    for alpha in (0.0, 0.25, 0.5, 0.75):
        args = (alpha, 0.5, (-0.10, -0.05), (0.20, 0.25), 0.3, 0.03)
        m = B.model_from_subordinated_bm(*args)
        o = O.model_from_subordinated_bm(*args)
        assert abs(m.delta - o.delta) <= 1e-14 * o.delta and abs(m.lambda_ - o.lam) <= 1e-14 * o.lam
        assert tuple(m.eta) == tuple(o.eta) and m.r == o.r
        assert max(abs(a - b) for a, b in zip(m.rho, o.rho)) <= 1e-16
        dirs = B.subordinated_bm_directions(*args[:5])
        base = dict(sigma1=0.20, sigma2=0.25, corr=0.3, kappa=0.5, beta1=-0.10, beta2=-0.05)
        eps = 1e-6
        for k, name in enumerate(B.SUBORDINATED_BM_PARAMS):
            pu, pd = dict(base), dict(base)
            pu[name] += eps
            pd[name] -= eps
            mu = B.model_from_subordinated_bm(alpha, pu["kappa"], (pu["beta1"], pu["beta2"]),
                                              (pu["sigma1"], pu["sigma2"]), pu["corr"], 0.03)
            md = B.model_from_subordinated_bm(alpha, pd["kappa"], (pd["beta1"], pd["beta2"]),
                                              (pd["sigma1"], pd["sigma2"]), pd["corr"], 0.03)
            for f, get in (("delta", lambda x: x.delta), ("lambda", lambda x: x.lambda_),
                           ("eta0", lambda x: x.eta[0]), ("eta1", lambda x: x.eta[1]),
                           ("rho0", lambda x: x.rho[0]), ("rho1", lambda x: x.rho[1]), ("rho2", lambda x: x.rho[2])):
                fd = (get(mu) - get(md)) / (2 * eps)
                assert abs(get(dirs[k]) - fd) <= 1e-7 * max(1.0, abs(fd)), (alpha, name, f, get(dirs[k]), fd)
    for bad in [(1.0, 0.5, (0, 0), (0.2, 0.2), 0.0, 0.0), (0.5, 0.0, (0, 0), (0.2, 0.2), 0.0, 0.0),
                (0.5, 0.5, (0, 0), (0.0, 0.2), 0.0, 0.0), (0.5, 0.5, (0, 0), (0.2, 0.2), 1.0, 0.0)]:
        with pytest.raises(B.PideError) as e:
            B.model_from_subordinated_bm(*bad)
        assert "ERR_ARG" in str(e.value)
