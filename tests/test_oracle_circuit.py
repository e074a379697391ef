"""Pins of the oracle's circuit and coupled solve on a particle-free gap.

With no particles and A = C d / eps0, the gap is exactly the capacitor C, so
the strict scheme integrates L q'' + R q' + q/C = s V_s(t) (q = circuit
charge, V_gap = q / C).  That ODE has a closed form: particular solutions
for the exponential forcing terms of V_s plus the damped homogeneous part
with q(0) = q'(0) = 0.  BDF2 (App. A) must reproduce it with second-order
error in dt; the weak scheme (Sec. 2.4.3) must coincide with the strict one
when no plasma charge is present.
"""
import math

import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W
from closed_forms import rlc_closed_form


def particle_free(dt, steps, mode, orc):
    cfg = W.scaled(W.gap_1d_fp64(), dt=dt, beam_per_step=0)
    g = orc.OracleGap(cfg)
    assert g.step(mode, steps) == orc.OK
    h = g.history()
    g.close()
    return cfg, h


def test_particle_free_gap_matches_closed_form_rlc(orc):
    T = 300e-9
    errs = []
    for dt in (2e-11, 1e-11):
        cfg, h = particle_free(dt, int(round(T / dt)), orc.STRICT, orc)
        q_exact = rlc_closed_form(cfg, h["t"])
        V_exact = q_exact / cfg["C"]
        scale = np.max(np.abs(V_exact))
        assert scale > 1e3  # the source has grown to tens of kV
        err = np.max(np.abs(h["V_gap"] - V_exact)) / scale
        errs.append(err)
        # the gap is the capacitor: V_gap = Q_circ / C and Q_surf = Q_circ
        np.testing.assert_allclose(h["V_gap"], h["Q_circ"] / cfg["C"], rtol=1e-10,
                                   atol=1e-12 * scale)
        np.testing.assert_allclose(h["Q_surf"], h["Q_circ"], rtol=1e-10,
                                   atol=1e-12 * np.max(np.abs(h["Q_circ"])))
        # current is the BDF2 derivative of the charge; compare with q'(t)
        assert np.all(h["residual"] <= 1e-12)
    assert errs[1] < 2e-5
    order = math.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.2, (errs, order)


def test_strict_and_weak_coincide_without_plasma(orc):
    cfg, hs = particle_free(1e-11, 5000, orc.STRICT, orc)
    _, hw = particle_free(1e-11, 5000, orc.WEAK, orc)
    scale = np.max(np.abs(hs["V_gap"]))
    np.testing.assert_allclose(hw["V_gap"], hs["V_gap"], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(hw["I_circ"], hs["I_circ"], rtol=0,
                               atol=1e-8 * np.max(np.abs(hs["I_circ"])))


def test_source_waveform_special_values(orc):
    cfg = W.gap_1d_fp64()
    assert orc.source(cfg, 0.0) == 0.0
    # peak of (1 - cos) at half a period: V0 exp(-1/(2 f tau))
    th = 0.5 / cfg["f"]
    assert orc.source(cfg, th) == pytest.approx(cfg["V0"] * math.exp(-th / cfg["tau"]), rel=1e-14)
    # starts quadratically: V_s(t) ~ V0 (2 pi f t)^2 / 4
    t = 1e-12
    assert orc.source(cfg, t) == pytest.approx(cfg["V0"] * (2 * math.pi * cfg["f"] * t) ** 2 / 4,
                                               rel=1e-6)
