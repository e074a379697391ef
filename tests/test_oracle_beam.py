"""Pins of the oracle's ion beam (ions entering the gap at x = d).

The beam of the workloads enters at the grounded electrode and flies
toward the driven one (the paper's ion injection, Sec. 3.2; the workloads
replace its Gaussian pulse by a steady beam).  What is checked is physics,
not a restatement of the oracle's formulas:

* every injected ion carries the beam energy: m_i v^2 / 2 = E (mono), or an
  energy uniform in [E_min, E_max] (mean and variance within 5 sigma over
  10^5 draws, Kolmogorov-Smirnov);
* it enters during the step: its position lies within one step's flight
  of x = d, and the flown fraction is uniform on (0, 1);
* ion ids are the loaded ions' followed by step * B + k;
* in a field-free gap an ion reaches x = 0 after d / (v dt) steps on
  average: the first arrivals come floor(d / (v dt)) pushes after the first
  injection and arrivals then average B per step.
"""
import math

import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W


def beam_only(orc, mode, B, steps, **over):
    """A gap with nothing in it but the beam, at negligible weight (no field)."""
    cfg = W.scaled(W.gap_1d_fp64(seed=5), beam_per_step=B, beam_mode=mode, circuit=orc.OPEN,
                   weight=1e-30, see_scale=0.0, **over)
    g = orc.OracleGap(cfg)
    assert g.step(orc.STRICT, steps) == orc.OK
    return cfg, g


def energies_eV(cfg, u):
    dx = cfg["d"] / cfg["n_cells"]
    v = u * dx / cfg["dt"]
    return 0.5 * cfg["m_i"] * v * v / cfg["e"]


def test_mono_beam_energy_entry_and_ids(orc):
    B = 100_000
    cfg, g = beam_only(orc, 0, B, 1)
    xi, u, ids = g.particles(orc.IONS)
    g.close()
    N = cfg["n_cells"]
    assert xi.size == B
    np.testing.assert_array_equal(np.sort(ids), np.arange(B, dtype=np.uint32))
    assert np.all(u < 0)  # toward the driven electrode
    E = energies_eV(cfg, u)
    np.testing.assert_allclose(E, cfg["beam_E_eV"], rtol=1e-13)
    frac = (N - xi) / np.abs(u)  # the fraction of the step already flown
    assert np.all(frac > 0) and np.all(frac < 1)
    assert abs(frac.mean() - 0.5) < 5 * math.sqrt(1 / 12 / B)
    assert abs(frac.var() - 1 / 12) < 5 * 0.0745 / math.sqrt(B)
    from scipy.stats import kstest
    assert kstest(frac, "uniform").pvalue > 1e-4


def test_uniform_beam_spectrum(orc):
    B = 100_000
    cfg, g = beam_only(orc, 1, B, 1)
    xi, u, _ = g.particles(orc.IONS)
    g.close()
    lo, hi = cfg["beam_Emin_eV"], cfg["beam_Emax_eV"]
    E = energies_eV(cfg, u)
    assert np.all(E >= lo * (1 - 1e-13)) and np.all(E <= hi * (1 + 1e-13))
    w = hi - lo
    assert abs(E.mean() - (lo + hi) / 2) < 5 * w / math.sqrt(12 * B)
    assert abs(E.var() - w * w / 12) < 5 * 0.0745 * w * w / math.sqrt(B)
    from scipy.stats import kstest
    assert kstest((E - lo) / w, "uniform").pvalue > 1e-4
    frac = (cfg["n_cells"] - xi) / np.abs(u)
    assert np.all(frac > 0) and np.all(frac < 1)


def test_ids_continue_after_the_loaded_ions(orc):
    cfg = W.scaled(W.gap_1d_fp64(seed=2), beam_per_step=7, weight=1e-30, see_scale=0.0,
                   circuit=orc.OPEN)
    g = orc.OracleGap(cfg)
    loaded = np.array([3, 11, 40], dtype=np.uint32)
    g.set_particles(orc.IONS, np.array([100.5, 120.25, 130.0]), np.zeros(3), loaded)
    assert g.step(orc.STRICT, 3) == orc.OK
    _, _, ids = g.particles(orc.IONS)
    g.close()
    want = np.concatenate([loaded, 41 + np.arange(3 * 7, dtype=np.uint32)])
    np.testing.assert_array_equal(np.sort(ids), np.sort(want))


def test_field_free_transit_time(orc):
    """Arrivals at x = 0 follow the flight time d / v of the beam ions."""
    B = 40
    cfg = W.gap_1d_fp64(seed=5)
    dx = cfg["d"] / cfg["n_cells"]
    v = math.sqrt(2 * cfg["beam_E_eV"] * cfg["e"] / cfg["m_i"])
    a = cfg["d"] / (v * cfg["dt"])  # flight time in steps
    T = int(2 * a) + 20
    cfg, g = beam_only(orc, 0, B, T)
    h = g.history()
    g.close()
    arr = h["absorbed"][:, 0, 1]  # row n: arrivals in the push from level n-1
    assert h["absorbed"][:, 1, 1].sum() == 0  # nothing leaves through x = d
    # cohort injected by push m (row m+1) arrives floor(a) or floor(a)+1 pushes later
    first = int(np.nonzero(arr)[0][0])
    assert first == 1 + math.floor(a), (first, a)
    # from then on every push delivers a cohort's worth on average: the running
    # total differs from B per row by less than one cohort
    r0 = first + 2
    tot = arr[r0:].sum()
    assert abs(tot - B * (len(arr) - r0)) <= B


def test_absorbed_ion_energy_tally(orc):
    """The energy of the ions absorbed at x = 0 (a feature of the learned
    weak scheme, from the impact velocity m_i v^2 / 2) equals the sum of the
    ions' kinetic energies within the tally's rounding (1/512 eV per ion)."""
    cfg = W.scaled(W.gap_1d_fp64(seed=4), beam_per_step=0, weight=1e-30, see_scale=0.0,
                   circuit=orc.OPEN)
    rng = np.random.default_rng(9)
    n = 5000
    N = cfg["n_cells"]
    dx = cfg["d"] / N
    E = rng.uniform(1e3, 6e4, n)  # eV
    u = -np.sqrt(2 * E * cfg["e"] / cfg["m_i"]) * cfg["dt"] / dx
    xi = rng.uniform(0.05, 0.95, n) * np.abs(u)  # every ion reaches x = 0 in its first push
    g = orc.OracleGap(cfg)
    g.set_particles(orc.IONS, xi, u)
    assert g.step(orc.STRICT, 1) == orc.OK
    h = g.history()
    g.close()
    assert h["absorbed"][1, 0, 1] == n
    # the first push kicks half a step in the (vanishing) field: impact speed = |u|
    want = float(energies_eV(cfg, u).sum())
    assert abs(h["ion_energy_eV"][1] - want) <= n / 512.0 + 1e-12 * want
