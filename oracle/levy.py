"""Oracle: the bivariate Normal Tempered Stable (NTS) Levy model, FP64, CPU.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

Every function follows one formula of the paper (Moda, in 't Hout,
Vanmaele, Benth, "Numerical valuation of European options under two-asset
infinite-activity exponential Levy models", arXiv 2511.02700):

* ``levy_density``            -- Sec. 4, NTS Levy density (the closed form
                                 with K_{1+alpha}); equal to delta*Phi(z|alpha,0)
                                 of Table A6 / eq. (A.2) with d = 2.
* ``levy_density_subordinated`` -- Appendix A construction L = B(G) - ct:
                                 the Levy measure of a Brownian motion with
                                 drift eta and covariance rho, subordinated by
                                 the tempered stable subordinator of Table A5.
                                 Used only as an independent pin of the above.
* ``variance``                -- Table A6 variance (Appendix A form; the Sec. 4
                                 variance formula carries a typo, see the
                                 readings list in the design notes).
* ``char_exponent_1d``        -- Table A6 characteristic exponent with d = 1.
* ``subordinator_from_mean_variance`` -- Table A5 mean and variance solved for
                                 (lambda, delta) at unit mean and variance kappa.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import integrate
from scipy.special import gamma, kve


@dataclass
class NTSModel:
    """Paper notation (Sec. 4, Table 2): 0 <= alpha < 1, delta > 0, lam > 0,
    eta in R^2, rho symmetric positive definite (2x2), riskless rate r, and
    the extra Gaussian covariance sigma sigma^T of eq. (2.3) (zero in all the
    paper's experiments)."""

    alpha: float
    delta: float
    lam: float
    eta: tuple
    rho: tuple  # (rho11, rho12, rho22)
    r: float
    sigma_cov: tuple = (0.0, 0.0, 0.0)  # (a11, a12, a22) of sigma sigma^T

    @property
    def rho_matrix(self) -> np.ndarray:
        r11, r12, r22 = self.rho
        return np.array([[r11, r12], [r12, r22]], dtype=np.float64)

    @property
    def sigma_matrix(self) -> np.ndarray:
        a11, a12, a22 = self.sigma_cov
        return np.array([[a11, a12], [a12, a22]], dtype=np.float64)


def subordinator_from_mean_variance(alpha: float, kappa: float):
    """Table A5: E[G(1)] = delta Gamma(1-alpha) / lam^(1-alpha) and
    V[G(1)] = delta Gamma(2-alpha) / lam^(2-alpha).  Setting the mean to 1
    and the variance to kappa gives V/E = (1-alpha)/lam = kappa."""
    lam = (1.0 - alpha) / kappa
    delta = lam ** (1.0 - alpha) / gamma(1.0 - alpha)
    return lam, delta


def model_from_subordinated_bm(alpha, kappa, beta, sigma, corr, r) -> NTSModel:
    """Workload parameterisation: unit-mean TS subordinator with variance
    kappa, Brownian drift eta = beta and Brownian covariance
    rho = [[s1^2, c s1 s2], [c s1 s2, s2^2]] (Appendix A, B(t) = eta t +
    sqrt(rho) W(t)); no extra Gaussian diffusion (the paper takes sigma = 0)."""
    lam, delta = subordinator_from_mean_variance(alpha, kappa)
    s1, s2 = sigma
    return NTSModel(alpha=alpha, delta=delta, lam=lam, eta=(beta[0], beta[1]),
                    rho=(s1 * s1, corr * s1 * s2, s2 * s2), r=r)


def _rho_quantities(m: NTSModel):
    R = m.rho_matrix
    Ri = np.linalg.inv(R)
    eta = np.asarray(m.eta, dtype=np.float64)
    eta_rho2 = float(eta @ Ri @ eta)            # ||eta||_rho^2
    c1 = np.sqrt(eta_rho2 + 2.0 * m.lam)       # sqrt(||eta||_rho^2 + 2 lam)
    return R, Ri, eta, eta_rho2, c1


def levy_density(m: NTSModel, z1, z2):
    """Sec. 4 NTS Levy density
        l(z) = delta/pi * sqrt(c1^(2(1+alpha)) / det rho) * K_{1+alpha}(c1 ||z||_rho)
               * ||z||_rho^(-1-alpha) * exp(<eta, z>_rho),
    with <x,y>_rho = x^T rho^{-1} y and c1 = sqrt(||eta||_rho^2 + 2 lam).
    Evaluated in log form with the exponentially scaled Bessel function to
    avoid overflow/underflow far from the origin."""
    R, Ri, eta, _, c1 = _rho_quantities(m)
    z1 = np.asarray(z1, dtype=np.float64)
    z2 = np.asarray(z2, dtype=np.float64)
    zn = np.sqrt(Ri[0, 0] * z1 * z1 + 2.0 * Ri[0, 1] * z1 * z2 + Ri[1, 1] * z2 * z2)
    b = Ri @ eta
    nu = 1.0 + m.alpha
    logpref = np.log(m.delta / np.pi) + 0.5 * (2.0 * nu * np.log(c1) - np.log(np.linalg.det(R)))
    with np.errstate(divide="ignore"):
        logl = (logpref + np.log(kve(nu, c1 * zn)) - c1 * zn - nu * np.log(zn)
                + b[0] * z1 + b[1] * z2)
    return np.exp(logl)


def levy_density_subordinated(m: NTSModel, z1: float, z2: float) -> float:
    """Appendix A: the Levy measure of B(G(t)) is the mixture
        l(z) = int_0^inf N(z; eta t, rho t) * delta e^{-lam t} t^{-1-alpha} dt
    (Gaussian density of B(t) weighted by the Table A5 subordinator measure).
    Computed by adaptive 1D quadrature; used only to pin ``levy_density``."""
    R = m.rho_matrix
    Ri = np.linalg.inv(R)
    eta = np.asarray(m.eta, dtype=np.float64)
    z = np.array([z1, z2], dtype=np.float64)
    detR = np.linalg.det(R)

    def integrand(t):
        d = z - eta * t
        q = d @ Ri @ d
        gauss = np.exp(-0.5 * q / t) / (2.0 * np.pi * t * np.sqrt(detR))
        return gauss * m.delta * np.exp(-m.lam * t) * t ** (-1.0 - m.alpha)

    # the mass sits near t ~ ||z||_rho / c1; split there for the adaptive rule
    _, _, _, _, c1 = _rho_quantities(m)
    zn = np.sqrt(z @ Ri @ z)
    tc = max(zn / c1, 1e-12)
    pts = [tc * 1e-3, tc * 1e-1, tc, tc * 10.0, tc * 1e3]
    total = 0.0
    lo = 0.0
    for p in pts + [np.inf]:
        v, _ = integrate.quad(integrand, lo, p, epsabs=0.0, epsrel=1e-13, limit=400)
        total += v
        lo = p
    return total


def variance(m: NTSModel) -> np.ndarray:
    """Table A6: V[L(1)] = delta Gamma(2-alpha)/lam^(2-alpha)
                            * (rho lam/(1-alpha) + eta eta^T)."""
    eta = np.asarray(m.eta, dtype=np.float64)
    return (m.delta * gamma(2.0 - m.alpha) / m.lam ** (2.0 - m.alpha)
            * (m.rho_matrix * m.lam / (1.0 - m.alpha) + np.outer(eta, eta)))


def char_exponent_1d(m: NTSModel, asset: int, u):
    """Table A6 with d = 1 for the marginal L^{(i)} = B_i(G) - c_i t (drift
    eta_i, variance rho_ii), compensated so E[L(1)] = 0:
        alpha = 0:  -delta ln((lam - i u eta + u^2 rho/2)/lam) - i u c
        alpha > 0:  delta Gamma(-alpha) ((lam - i u eta + u^2 rho/2)^alpha - lam^alpha) - i u c
    with c = delta Gamma(1-alpha)/lam^(1-alpha) * eta.  E[exp(i u L(t))] =
    exp(t psi(u)).  Complex u is allowed (principal branch)."""
    u = np.asarray(u, dtype=np.complex128)
    eta = m.eta[asset]
    rho = m.rho[0] if asset == 0 else m.rho[2]
    c = m.delta * gamma(1.0 - m.alpha) / m.lam ** (1.0 - m.alpha) * eta
    q = m.lam - 1j * u * eta + 0.5 * u * u * rho
    if m.alpha == 0.0:
        psi = -m.delta * np.log(q / m.lam)
    else:
        psi = m.delta * gamma(-m.alpha) * (q ** m.alpha - m.lam ** m.alpha)
    return psi - 1j * u * c


def put_price_1d(m: NTSModel, asset: int, S0: float, K: float, T: float) -> float:
    """European put on one asset of the exponential Levy model of Sec. 2.1
    (eqs. 2.1-2.4 reduced to one coordinate): under Q,
        ln S_T = ln S0 + (r - psi(-i) - s^2/2) T + s W_T + L_T,
    where psi(-i) = int (e^z - 1 - z) l(dz) is the jump compensator and s^2
    the extra Gaussian variance.  Priced by Fourier inversion (Lewis' contour
    at Im = -1/2) of the call, then put-call parity:
        C = S0 - sqrt(S0 K) e^{-rT}/pi * int_0^inf Re[e^{i u k} phi(u - i/2)] / (u^2 + 1/4) du,
    with k = ln(S0/K) and phi the characteristic function of ln(S_T/S0)
    (the pole of the call transform at zeta = i gives the S0 term)."""
    s2 = m.sigma_cov[0] if asset == 0 else m.sigma_cov[2]
    comp = float(np.real(char_exponent_1d(m, asset, -1j)))  # psi(-i), real

    def phi(u):
        u = np.asarray(u, dtype=np.complex128)
        drift = (m.r - comp - 0.5 * s2) * T
        return np.exp(1j * u * drift + T * (char_exponent_1d(m, asset, u) - 0.5 * s2 * u * u))

    k = np.log(S0 / K)

    def integrand(u):
        return float(np.real(np.exp(1j * u * k) * phi(u - 0.5j))) / (u * u + 0.25)

    val, _ = integrate.quad(integrand, 0.0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=2000)
    call = S0 - np.sqrt(S0 * K) * np.exp(-m.r * T) / np.pi * val
    return call - S0 + K * np.exp(-m.r * T)
