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
