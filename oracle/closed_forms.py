"""Closed-form solutions that pin the oracle (test infrastructure only).

Each function is a textbook solution of the continuous or discrete problem the
paper's equations reduce to in a special case:

* ``erfc_1d``        -- 1D conduction into a half space after a step change of
                        the boundary temperature (Eq. 2 with q = 0), or the
                        same for head diffusion (Eq. 1, D = K / S_s).
* ``ogata_banks``    -- 1D advection-diffusion with a step inflow boundary
                        (Eq. 2 with a uniform Darcy flux).
* ``q1_mode_factor`` -- per-step amplification of the discrete sine mode for
                        Q1 elements with consistent mass and backward Euler
                        (Eq. 3 / Eq. 4 on a uniform mesh).
* ``line_source_e1`` -- continuous infinite line source in a still medium
                        (exponential integral E1).
* ``moving_line_source`` -- the same line source in a uniform groundwater flow
                        (the moving infinite line source of Diao, Li and Fang,
                        2004), and its steady limit with the modified Bessel
                        function K0.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def erfc_1d(x, t, D, dT):
    """u(x, t) = dT * erfc(x / (2 sqrt(D t)))."""
    return dT * special.erfc(np.asarray(x) / (2.0 * math.sqrt(D * t)))


def ogata_banks(x, t, v, D, dT):
    """Ogata & Banks (1961): u_t + v u_x = D u_xx on x > 0, u(0, t) = dT,
    u(x, 0) = 0."""
    x = np.asarray(x, dtype=np.float64)
    s = 2.0 * math.sqrt(D * t)
    a = special.erfc((x - v * t) / s)
    # exp(v x / D) erfc((x + v t)/s) written with erfcx for stability
    arg = (x + v * t) / s
    b = np.exp(v * x / D - arg * arg) * special.erfcx(arg)
    return 0.5 * dT * (a + b)


def q1_mode_mu(H, L):
    """Generalised eigenvalue of the 1D Q1 stiffness/mass pair for the mode
    sin(pi x / L) on a uniform mesh of spacing H:
    mu = 6 (1 - cos theta) / (H^2 (2 + cos theta)), theta = pi H / L."""
    th = math.pi * H / L
    return 6.0 * (1.0 - math.cos(th)) / (H * H * (2.0 + math.cos(th)))


def q1_mode_factor(dt, diff, Hs, Ls):
    """Backward-Euler amplification 1 / (1 + dt * diff * sum_d mu_d)."""
    return 1.0 / (1.0 + dt * diff * sum(q1_mode_mu(H, L) for H, L in zip(Hs, Ls)))


def line_source_e1(r, t, ql, lam, a):
    """dT = q_l / (4 pi lambda) * E1(r^2 / (4 a t)) for a continuous infinite
    line source of strength q_l (W/m) switched on at t = 0."""
    return ql / (4.0 * math.pi * lam) * special.exp1(np.asarray(r) ** 2 / (4.0 * a * t))


def moving_line_source(x, y, t, ql, lam, a, U):
    """dT(x, y, t) = q_l / (4 pi lambda) exp(U x / (2 a))
    * int_{r^2/(4 a t)}^inf exp(-psi - U^2 r^2 / (16 a^2 psi)) / psi dpsi,
    r^2 = x^2 + y^2, for a line source at the origin switched on at t = 0 in
    a medium of diffusivity a whose heat moves at U along +x (U = c_w q / c_T
    for a Darcy flux q).  With U = 0 it is line_source_e1."""
    from scipy import integrate
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    out = np.empty(np.broadcast(x, y).shape)
    for k, (xx, yy) in enumerate(np.broadcast(x, y)):
        r2 = xx * xx + yy * yy
        c = U * U * r2 / (16.0 * a * a)
        val, _ = integrate.quad(lambda s: math.exp(-s - c / s) / s, r2 / (4.0 * a * t), np.inf,
                                epsabs=0.0, epsrel=1e-12, limit=200)
        out.flat[k] = ql / (4.0 * math.pi * lam) * math.exp(U * xx / (2.0 * a)) * val
    return out


def moving_line_source_steady(x, y, ql, lam, a, U):
    """t -> infinity limit: q_l / (2 pi lambda) exp(U x / (2 a)) K0(U r / (2 a))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = np.sqrt(x * x + y * y)
    return ql / (2.0 * math.pi * lam) * np.exp(U * x / (2.0 * a)) * special.k0(U * r / (2.0 * a))
