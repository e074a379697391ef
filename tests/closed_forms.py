"""Closed-form references used as pins (no oracle or CUDA code)."""
import math

import numpy as np


def rlc_closed_form(cfg, t):
    """q(t) of L q'' + R q' + q/C = s V0 (1 - cos w t) e^{-t/tau} / 2, q(0)=q'(0)=0."""
    L, R, C = cfg["L"], cfg["R"], cfg["C"]
    s, V0, w, tau = cfg["polarity"], cfg["V0"], 2 * math.pi * cfg["f"], cfg["tau"]
    Z = lambda a: L * a * a + R * a + 1.0 / C
    a0 = -1.0 / tau
    a1 = complex(-1.0 / tau, w)
    amp = s * V0 / 2.0
    qp = lambda tt: amp * (np.exp(a0 * tt) / Z(a0) - np.real(np.exp(a1 * tt) / Z(a1)))
    dqp = lambda tt: amp * (a0 * np.exp(a0 * tt) / Z(a0) - np.real(a1 * np.exp(a1 * tt) / Z(a1)))
    alpha = R / (2 * L)
    wd = math.sqrt(1.0 / (L * C) - alpha * alpha)
    c1 = -qp(0.0)
    c2 = (alpha * c1 - dqp(0.0)) / wd
    return qp(t) + np.exp(-alpha * t) * (c1 * np.cos(wd * t) + c2 * np.sin(wd * t))
