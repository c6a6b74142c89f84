"""Thin ctypes binding of the pide2d C ABI (include/pide2d.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names; ``Solver`` is a convenience
wrapper that takes its device workspace from PyTorch and runs on a PyTorch
stream.  If the library has not been built, ``lib()`` raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpide2d.so")

PIDE2D_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_WORKSPACE", 4: "ERR_NOT_CONVERGED",
          5: "ERR_STATE", 6: "ERR_UNSUPPORTED"}
PIDE2D_PUT_AVG, PIDE2D_CALL_AVG, PIDE2D_PUT_ASSET1 = 0, 1, 2
PIDE2D_FP64, PIDE2D_FP32_BULK = 0, 1


class pide2d_grid(ctypes.Structure):
    _fields_ = [("n", c_int), ("n_z", c_int), ("s_center", c_double * 2), ("half_width", c_double),
                ("sl_order", c_int), ("precision", c_int)]


class pide2d_model(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("delta", c_double), ("lambda_", c_double), ("eta", c_double * 2),
                ("rho", c_double * 3), ("r", c_double), ("sigma_cov", c_double * 3)]


class pide2d_contract(ctypes.Structure):
    _fields_ = [("payoff", c_int), ("strike", c_double), ("maturity", c_double)]


class pide2d_options(ctypes.Structure):
    _fields_ = [("kmax", c_int), ("damping", c_int), ("host_loop", c_int), ("fixed_shapes", c_int)]


class pide2d_stats(ctypes.Structure):
    _fields_ = [("steps_done", c_int), ("fp_iters_total", c_int), ("fp_iters_max", c_int),
                ("last_resid", c_double), ("cell_iters", c_double)]


class pide2d_kernel_times(ctypes.Structure):
    _fields_ = [("launches", c_int * 16), ("ms", c_double * 16)]


class pide2d_workload(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("kappa", c_double), ("beta", c_double * 2), ("sigma", c_double * 2),
                ("corr", c_double), ("r", c_double)]


class pide2d_job(ctypes.Structure):
    _fields_ = [("grid", pide2d_grid), ("model", pide2d_model), ("contract", pide2d_contract),
                ("theta", c_double), ("dt", c_double), ("fp_tol", c_double)]


class pide2d_batch_stats(ctypes.Structure):
    _fields_ = [("jobs_done", c_int), ("failures", c_int), ("fp_iters_total", c_int), ("cell_iters", c_double),
                ("tuned", c_int), ("tune_n", c_int * 8), ("tune_units", c_int * 8), ("tune_lanes", c_int * 8),
                ("tune_us_per_job", c_double * 8), ("create_s", c_double), ("tune_s", c_double),
                ("loop_s", c_double)]

    def tuning(self):
        """The launch shapes the batch picked, one dict per tuned geometry group."""
        return [{"n": self.tune_n[i], "units_per_block": self.tune_units[i], "lanes": self.tune_lanes[i],
                 "us_per_job_column_pass": self.tune_us_per_job[i]} for i in range(min(self.tuned, 8))]


class pide2d_price_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("x", c_void_p), ("n_z", c_int), ("h_z", c_double), ("ny_minus", c_int),
                ("ny_plus", c_int), ("precision", c_int)]


class PideError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"pide2d CUDA library missing ({LIB_PATH}); "
                               "build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.pide2d_workspace_bytes.argtypes = [POINTER(pide2d_grid), POINTER(c_size_t)]
        L.pide2d_create.argtypes = [POINTER(pide2d_grid), POINTER(pide2d_model), POINTER(pide2d_contract),
                                    c_double, c_double, c_double, POINTER(pide2d_options), c_void_p, c_size_t,
                                    c_void_p, POINTER(c_void_p)]
        L.pide2d_step.argtypes = [c_void_p, POINTER(c_int), POINTER(c_double)]
        L.pide2d_solve.argtypes = [c_void_p, POINTER(c_double), c_void_p, POINTER(pide2d_stats)]
        L.pide2d_get_values.argtypes = [c_void_p, c_void_p]
        L.pide2d_get_weights.argtypes = [c_void_p, c_void_p, c_void_p]
        L.pide2d_apply_jump.argtypes = [c_void_p, c_void_p, c_double, c_int, c_void_p]
        L.pide2d_iteration_probe.argtypes = [c_void_p, c_void_p, c_double, c_double, c_void_p, c_void_p,
                                             POINTER(c_double)]
        L.pide2d_last_error.argtypes = [c_void_p]
        L.pide2d_last_error.restype = ctypes.c_char_p
        L.pide2d_profile.argtypes = [c_void_p, c_int]
        L.pide2d_profile_read.argtypes = [c_void_p, POINTER(pide2d_kernel_times)]
        L.pide2d_jump_static.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_void_p]
        L.pide2d_greeks.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.pide2d_tape_bytes.argtypes = [c_void_p, c_int, c_int, POINTER(c_size_t)]
        L.pide2d_record.argtypes = [c_void_p, c_void_p, c_size_t, c_int, c_int]
        L.pide2d_adjoint.argtypes = [c_void_p, POINTER(pide2d_model), c_int, POINTER(c_double)]
        L.pide2d_model_from_workload.argtypes = [POINTER(pide2d_workload), POINTER(pide2d_model)]
        L.pide2d_workload_directions.argtypes = [POINTER(pide2d_workload), POINTER(pide2d_model)]
        L.pide2d_adjoint_workload.argtypes = [c_void_p, POINTER(pide2d_workload), POINTER(c_double)]
        L.pide2d_price_workspace_bytes.argtypes = [POINTER(pide2d_price_grid), POINTER(c_size_t)]
        L.pide2d_price_sinh_grid.argtypes = [c_int, c_double, c_double, c_double, c_double, c_void_p,
                                             POINTER(pide2d_price_grid)]
        L.pide2d_price_create.argtypes = [POINTER(pide2d_price_grid), POINTER(pide2d_model), c_void_p, c_size_t,
                                          c_void_p, POINTER(c_void_p)]
        L.pide2d_price_apply_jump.argtypes = [c_void_p, c_void_p, c_void_p]
        L.pide2d_price_get_weights.argtypes = [c_void_p, c_void_p, c_void_p]
        L.pide2d_price_solve.argtypes = [c_void_p, POINTER(pide2d_contract), c_double, c_int, c_double,
                                         POINTER(pide2d_options), c_void_p, POINTER(pide2d_stats)]
        L.pide2d_price_last_error.argtypes = [c_void_p]
        L.pide2d_price_last_error.restype = c_char_p
        L.pide2d_price_destroy.argtypes = [c_void_p]
        L.pide2d_price_destroy.restype = None
        L.pide2d_batch_workspace_bytes.argtypes = [POINTER(pide2d_job), c_int, c_int, POINTER(c_size_t)]
        L.pide2d_batch_solve.argtypes = [POINTER(pide2d_job), c_int, POINTER(pide2d_options), c_int, c_void_p,
                                         c_size_t, POINTER(c_double), POINTER(c_int), POINTER(pide2d_batch_stats)]
        L.pide2d_destroy.argtypes = [c_void_p]
        L.pide2d_destroy.restype = None
        for name in ("pide2d_workspace_bytes", "pide2d_create", "pide2d_step", "pide2d_solve",
                     "pide2d_get_values", "pide2d_get_weights", "pide2d_apply_jump", "pide2d_iteration_probe",
                     "pide2d_profile",
                     "pide2d_profile_read", "pide2d_jump_static", "pide2d_greeks", "pide2d_batch_workspace_bytes",
                     "pide2d_batch_solve", "pide2d_tape_bytes", "pide2d_record", "pide2d_adjoint",
                     "pide2d_model_from_workload", "pide2d_workload_directions", "pide2d_adjoint_workload",
                     "pide2d_price_workspace_bytes", "pide2d_price_create", "pide2d_price_apply_jump",
                     "pide2d_price_get_weights", "pide2d_price_solve", "pide2d_price_sinh_grid"):
            getattr(L, name).restype = c_int
        _LIB = L
    return _LIB


def _check(status, handle=None):
    if status != PIDE2D_OK and status != 4:
        raise PideError(status, lib().pide2d_last_error(handle).decode())
    return status


# ------------------------------------------------------------------ C names
def pide2d_workspace_bytes(grid: pide2d_grid) -> int:
    n = c_size_t(0)
    _check(lib().pide2d_workspace_bytes(byref(grid), byref(n)))
    return n.value


def pide2d_create(grid, model, contract, theta, dt, fp_tol, opts, workspace, workspace_bytes, stream):
    h = c_void_p(0)
    _check(lib().pide2d_create(byref(grid), byref(model), byref(contract), theta, dt, fp_tol,
                               byref(opts) if opts is not None else None, c_void_p(workspace),
                               workspace_bytes, c_void_p(stream), byref(h)))
    return h


def pide2d_step(h):
    k = c_int(0)
    r = c_double(0.0)
    st = _check(lib().pide2d_step(h, byref(k), byref(r)), h)
    return k.value, r.value, st


def pide2d_solve(h, values_out_ptr=None):
    price = c_double(0.0)
    stats = pide2d_stats()
    st = _check(lib().pide2d_solve(h, byref(price), c_void_p(values_out_ptr) if values_out_ptr else None,
                                   byref(stats)), h)
    return price.value, stats, st


def pide2d_get_values(h, dst_ptr):
    _check(lib().pide2d_get_values(h, c_void_p(dst_ptr)), h)


def pide2d_get_weights(h, omega_ptr, rates_ptr):
    _check(lib().pide2d_get_weights(h, c_void_p(omega_ptr) if omega_ptr else None,
                                    c_void_p(rates_ptr) if rates_ptr else None), h)


def pide2d_apply_jump(h, U_ptr, tau, far_field, out_ptr):
    _check(lib().pide2d_apply_jump(h, c_void_p(U_ptr), tau, int(far_field), c_void_p(out_ptr)), h)


def pide2d_iteration_probe(h, r_ptr, ht, theta, delta_ptr, bdelta_ptr):
    stop = c_double(0.0)
    _check(lib().pide2d_iteration_probe(h, c_void_p(r_ptr), ht, theta, c_void_p(delta_ptr) if delta_ptr else None,
                                        c_void_p(bdelta_ptr) if bdelta_ptr else None, byref(stop)), h)
    return stop.value


def pide2d_greeks(h, delta1, delta2, gamma11, gamma12, gamma22):
    _check(lib().pide2d_greeks(h, *[c_void_p(p) if p else None for p in
                                    (delta1, delta2, gamma11, gamma12, gamma22)]), h)


def pide2d_profile(h, enable):
    _check(lib().pide2d_profile(h, int(enable)), h)


def pide2d_profile_read(h) -> pide2d_kernel_times:
    out = pide2d_kernel_times()
    _check(lib().pide2d_profile_read(h, byref(out)), h)
    return out


def pide2d_jump_static(n, omega_ptr, U_ptr, out_ptr, stream=0):
    """B_w U without device allocation (device pointers; n <= 256; async on stream)."""
    _check(lib().pide2d_jump_static(int(n), c_void_p(omega_ptr), c_void_p(U_ptr), c_void_p(out_ptr),
                                    c_void_p(stream)))


def pide2d_tape_bytes(h, interval, ndirs) -> int:
    n = c_size_t(0)
    _check(lib().pide2d_tape_bytes(h, interval, ndirs, byref(n)), h)
    return n.value


def pide2d_record(h, tape_ptr, nbytes, interval, ndirs):
    _check(lib().pide2d_record(h, c_void_p(tape_ptr), nbytes, interval, ndirs), h)


def pide2d_adjoint(h, dirs):
    """Returns (gradient list, status)."""
    k = len(dirs)
    arr = (pide2d_model * k)(*dirs)
    g = (c_double * k)()
    st = _check(lib().pide2d_adjoint(h, arr, k, g), h)
    return list(g), st


def pide2d_adjoint_workload(h, workload):
    """Returns (gradient in SUBORDINATED_BM_PARAMS order, status)."""
    g = (c_double * 6)()
    st = _check(lib().pide2d_adjoint_workload(h, byref(workload), g), h)
    return list(g), st


def pide2d_batch_workspace_bytes(jobs, lanes) -> int:
    arr = (pide2d_job * len(jobs))(*jobs)
    n = c_size_t(0)
    _check(lib().pide2d_batch_workspace_bytes(arr, len(jobs), lanes, byref(n)))
    return n.value


def pide2d_batch_solve(jobs, opts, lanes, workspace, workspace_bytes):
    """Returns (prices list, statuses list, stats, status)."""
    count = len(jobs)
    arr = (pide2d_job * count)(*jobs)
    prices = (c_double * count)()
    sts = (c_int * count)()
    stats = pide2d_batch_stats()
    st = lib().pide2d_batch_solve(arr, count, byref(opts) if opts is not None else None, lanes,
                                  c_void_p(workspace), workspace_bytes, prices, sts, byref(stats))
    if st not in (PIDE2D_OK, 4):
        raise PideError(st, lib().pide2d_last_error(None).decode())
    return list(prices), list(sts), stats, st


def make_job(grid, model, contract, n_steps, theta=0.5, tol=1e-10):
    j = pide2d_job()
    j.grid, j.model, j.contract = grid, model, contract
    j.theta, j.dt, j.fp_tol = theta, contract.maturity / n_steps, tol
    return j


def pide2d_last_error(h=None) -> str:
    return lib().pide2d_last_error(h).decode()


def pide2d_destroy(h):
    lib().pide2d_destroy(h)


# ------------------------------------------------------------------ helpers
def make_grid(n, precision=PIDE2D_FP64, sl_order=3, s0=(100.0, 100.0), half_width=2.5):
    g = pide2d_grid()
    g.n = n
    g.n_z = 0
    g.s_center[0] = math.log(s0[0])
    g.s_center[1] = math.log(s0[1])
    g.half_width = half_width
    g.sl_order = sl_order
    g.precision = precision
    return g


def make_model(alpha, delta, lam, eta, rho, r, sigma_cov=(0.0, 0.0, 0.0)):
    m = pide2d_model()
    m.alpha, m.delta, m.lambda_ = alpha, delta, lam
    m.eta[0], m.eta[1] = eta
    m.rho[0], m.rho[1], m.rho[2] = rho
    m.r = r
    m.sigma_cov[0], m.sigma_cov[1], m.sigma_cov[2] = sigma_cov
    return m


def make_workload(alpha, kappa, beta, sigma, corr, r):
    w = pide2d_workload()
    w.alpha, w.kappa = alpha, kappa
    w.beta[0], w.beta[1] = beta
    w.sigma[0], w.sigma[1] = sigma
    w.corr, w.r = corr, r
    return w


def model_from_subordinated_bm(alpha, kappa, beta, sigma, corr, r):
    """pide2d_model_from_workload: the NTS model of a unit-mean tempered-stable
    subordinator with variance kappa, Brownian drift beta, volatilities sigma
    and correlation corr (the mapping lives in the C library)."""
    m = pide2d_model()
    _check(lib().pide2d_model_from_workload(byref(make_workload(alpha, kappa, beta, sigma, corr, r)), byref(m)))
    return m


SUBORDINATED_BM_PARAMS = ("sigma1", "sigma2", "corr", "kappa", "beta1", "beta2")


def subordinated_bm_directions(alpha, kappa, beta, sigma, corr, r=0.0):
    """pide2d_workload_directions: the six model tangents for
    SUBORDINATED_BM_PARAMS, as pide2d_model directions for pide2d_adjoint."""
    dirs = (pide2d_model * 6)()
    _check(lib().pide2d_workload_directions(byref(make_workload(alpha, kappa, beta, sigma, corr, r)), dirs))
    return list(dirs)


def make_contract(payoff=PIDE2D_PUT_AVG, strike=100.0, maturity=1.0):
    c = pide2d_contract()
    c.payoff, c.strike, c.maturity = payoff, strike, maturity
    return c


class Solver:
    """One pricing: device workspace from PyTorch, kernels on a PyTorch stream."""

    def __init__(self, grid, model, contract, n_steps, theta=0.5, tol=1e-10, kmax=100, damping=True,
                 device="cuda", stream=None, host_loop=False):
        import torch
        self.torch = torch
        self.grid = grid
        self.n = grid.n
        nbytes = pide2d_workspace_bytes(grid)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        opts = pide2d_options()
        opts.kmax, opts.damping = kmax, 1 if damping else 0
        opts.host_loop = 1 if host_loop else 0
        self.h = pide2d_create(grid, model, contract, theta, contract.maturity / n_steps, tol, opts, base,
                               nbytes, self.stream.cuda_stream)
        self.workspace_bytes = nbytes

    def step(self):
        return pide2d_step(self.h)

    def solve(self, values=False):
        torch = self.torch
        out = None
        if values:
            out = torch.empty((self.n + 1, self.n + 1), dtype=torch.float64, device=self.ws.device)
        price, stats, status = pide2d_solve(self.h, out.data_ptr() if out is not None else None)
        return price, out, stats, status

    def values(self):
        out = self.torch.empty((self.n + 1, self.n + 1), dtype=self.torch.float64, device=self.ws.device)
        pide2d_get_values(self.h, out.data_ptr())
        return out

    def weights(self):
        torch = self.torch
        om = torch.empty((self.n, self.n), dtype=torch.float64, device=self.ws.device)
        rates = torch.empty(9, dtype=torch.float64)
        pide2d_get_weights(self.h, om.data_ptr(), rates.data_ptr())
        return om, rates

    def greeks(self):
        """Delta and Gamma fields of the current values (device tensors)."""
        torch = self.torch
        outs = [torch.zeros((self.n + 1, self.n + 1), dtype=torch.float64, device=self.ws.device) for _ in range(5)]
        pide2d_greeks(self.h, *[o.data_ptr() for o in outs])
        return dict(zip(("delta1", "delta2", "gamma11", "gamma12", "gamma22"), outs))

    def apply_jump(self, U, tau, far_field=True):
        torch = self.torch
        U = U.to(device=self.ws.device, dtype=torch.float64).contiguous()
        out = torch.zeros_like(U)
        pide2d_apply_jump(self.h, U.data_ptr(), tau, far_field, out.data_ptr())
        return out

    def iteration_probe(self, r, ht, theta=0.5):
        """pide2d_iteration_probe: (delta, B_w delta, stop) for a residual field r."""
        torch = self.torch
        r = r.to(device=self.ws.device, dtype=torch.float64).contiguous()
        d = torch.zeros_like(r)
        bd = torch.zeros_like(r)
        stop = pide2d_iteration_probe(self.h, r.data_ptr(), ht, theta, d.data_ptr(), bd.data_ptr())
        return d, bd, stop

    def record(self, interval=16, ndirs=6):
        """Checkpoint the time loop for pide2d_adjoint (before the first step)."""
        torch = self.torch
        nbytes = pide2d_tape_bytes(self.h, interval, ndirs)
        self.tape = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.ws.device)
        base = (self.tape.data_ptr() + 255) & ~255
        pide2d_record(self.h, base, nbytes, interval, ndirs)
        self.tape_bytes = nbytes

    def adjoint(self, dirs):
        return pide2d_adjoint(self.h, dirs)

    def adjoint_workload(self, workload):
        """Gradient with respect to SUBORDINATED_BM_PARAMS (pide2d_adjoint_workload)."""
        return pide2d_adjoint_workload(self.h, workload)

    def close(self):
        if self.h:
            pide2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(jobs, lanes=16, kmax=100, damping=True, device="cuda", host_loop=False, fixed_shapes=False):
    """Prices a list of pide2d_job through pide2d_batch_solve (workspace from
    PyTorch).  Returns (prices, statuses, stats)."""
    import torch
    lanes = max(1, min(lanes, len(jobs)))
    nbytes = pide2d_batch_workspace_bytes(jobs, lanes)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    base = (ws.data_ptr() + 255) & ~255
    opts = pide2d_options()
    opts.kmax, opts.damping = kmax, 1 if damping else 0
    opts.host_loop = 1 if host_loop else 0
    opts.fixed_shapes = 1 if fixed_shapes else 0
    torch.cuda.synchronize(device)
    prices, sts, stats, _ = pide2d_batch_solve(jobs, opts, lanes, base, nbytes)
    del ws
    return prices, sts, stats


def price_function():
    """torch.autograd.Function: price(params) with params = (sigma1, sigma2,
    corr, kappa, beta1, beta2) as a float64 tensor; the backward pass is the
    discrete adjoint (pide2d_adjoint).  Extra arguments of apply: alpha, r,
    grid, contract, n_steps, theta, tol, interval."""
    import torch

    class _Price(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, alpha, r, grid, contract, n_steps, theta=0.5, tol=1e-10, interval=16):
            p = [float(x) for x in params.detach().cpu().tolist()]
            wl = make_workload(alpha, p[3], (p[4], p[5]), (p[0], p[1]), p[2], r)
            model = pide2d_model()
            _check(lib().pide2d_model_from_workload(byref(wl), byref(model)))
            s = Solver(grid, model, contract, n_steps, theta=theta, tol=tol)
            s.record(interval=interval, ndirs=6)
            price, _, _, _ = s.solve()
            g, _ = s.adjoint_workload(wl)
            s.close()
            ctx.save_for_backward(torch.tensor(g, dtype=torch.float64))
            return torch.tensor(price, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return (grad_out * g, None, None, None, None, None, None, None, None)

    return _Price


def price_sinh_grid(nx, strike, x_max, z_iii, frac=0.65):
    """pide2d_price_sinh_grid: the paper's price grid (Sec. 4).  Returns
    (x, n_z, h_z, ny_minus, ny_plus) as PriceJump takes them."""
    import numpy as np
    x = np.empty(nx + 1, dtype=np.float64)
    g = pide2d_price_grid()
    _check(lib().pide2d_price_sinh_grid(nx, strike, x_max, z_iii, frac, x.ctypes.data, byref(g)))
    return x, g.n_z, g.h_z, g.ny_minus, g.ny_plus


class PriceJump:
    """The price-space jump operator B_w = T_out I~ C T_in on a non-uniform
    price grid (pide2d_price_*); workspace from PyTorch."""

    def __init__(self, x, n_z, h_z, ny_minus, ny_plus, model, precision=PIDE2D_FP64, device="cuda", stream=None):
        import numpy as np
        import torch
        self.torch = torch
        self._x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        g = pide2d_price_grid()
        g.nx = self._x.size - 1
        g.x = self._x.ctypes.data
        g.n_z, g.h_z, g.ny_minus, g.ny_plus, g.precision = n_z, h_z, ny_minus, ny_plus, precision
        self.grid = g
        n = c_size_t(0)
        _check(lib().pide2d_price_workspace_bytes(byref(g), byref(n)))
        self.ws = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        base = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = c_void_p()
        st = lib().pide2d_price_create(byref(g), byref(model), c_void_p(base), n.value,
                                       c_void_p(self.stream.cuda_stream), byref(h))
        if st != PIDE2D_OK:
            raise PideError(st, lib().pide2d_last_error(None).decode())
        self.h = h
        self.nx1 = g.nx + 1

    def apply(self, V):
        torch = self.torch
        V = V.to(device=self.ws.device, dtype=torch.float64).contiguous()
        out = torch.empty_like(V)
        st = lib().pide2d_price_apply_jump(self.h, c_void_p(V.data_ptr()), c_void_p(out.data_ptr()))
        if st != PIDE2D_OK:
            raise PideError(st, lib().pide2d_price_last_error(self.h).decode())
        return out

    def solve(self, contract, n_steps, theta=0.5, tol=1e-7, kmax=100, damping=True):
        """Algorithm 1 in price space on this grid; returns (V device tensor, stats, status)."""
        torch = self.torch
        V = torch.empty((self.nx1, self.nx1), dtype=torch.float64, device=self.ws.device)
        opts = pide2d_options()
        opts.kmax, opts.damping = kmax, 1 if damping else 0
        stats = pide2d_stats()
        st = lib().pide2d_price_solve(self.h, byref(contract), theta, n_steps, tol, byref(opts),
                                      c_void_p(V.data_ptr()), byref(stats))
        if st not in (PIDE2D_OK, 4):
            raise PideError(st, lib().pide2d_price_last_error(self.h).decode())
        return V, stats, st

    def weights(self):
        torch = self.torch
        nzz = 2 * self.grid.n_z
        om = torch.empty((nzz, nzz), dtype=torch.float64, device=self.ws.device)
        rates = (c_double * 9)()
        st = lib().pide2d_price_get_weights(self.h, c_void_p(om.data_ptr()), rates)
        if st != PIDE2D_OK:
            raise PideError(st, lib().pide2d_price_last_error(self.h).decode())
        return om, list(rates)

    def close(self):
        if getattr(self, "h", None):
            lib().pide2d_price_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

