"""Seeded synthetic workloads shared by the CUDA path's callers and the tests.

This module holds parameter sets and seeded initial-condition draws only; it
contains none of the PIC/SEE/circuit arithmetic.  Positions come out in cell
units (xi = x/dx in [0, N)) and velocities in cells per step (u = v dt/dx),
the representation both the CUDA path and the oracle take.

Workloads (all synthetic; the paper's measured waveforms, SEY fits and
injection profile are not available, so these parameter sets stand in):

* ``gap_1d_fp64``: 5 mm planar vacuum gap, 256 cells, 1e4 electron/H+ pairs at
  1 eV, n0 = 1e14 m^-3, 20 keV H+ beam of 50 macroparticles/step entering at
  x = d, SEE yield min(0.05 sqrt(E/1 keV), 3), 2 eV emitted electrons, source
  V0 (1-cos 2 pi f t) exp(-t/tau)/2 with V0 = 100 kV, f = 1 MHz, tau = 2 us into
  R = 50 Ohm, L = 1 uH, C = 100 pF; dt = 1 ps, 5000 steps; FP64 particles.
* ``gap_1d_fp32_large``: same gap with 4096 cells, 1e7 macroparticles (5e6
  pairs), 5000 beam macroparticles/step (mono 20 keV or uniform 5-50 keV
  depending on the seed), dt = 0.5 ps, 20000 steps; FP32 particles.
* ``gap_1d_fp32_thinned``: the same physics with `factor` times fewer
  macroparticles of `factor` times the weight (loaded pairs and beam alike):
  the predictor's training and evaluation runs.
* ``gap_2d``: 5 mm x 5 mm gap, periodic in y, 1024 x 1024 cells, 1e8
  macroparticles (5e7 pairs), a 20 keV H+ beam with a Gaussian transverse
  profile (sigma 0.5 mm, centred) at n_pairs/1000 ions per step, dt = 1 ps,
  2000 steps, FP32 particles; the electrode area (depth x 5 mm) keeps the
  gap capacitance at C.
* ``tesla_gap``: the paper's integrated configuration (Tables 3 and 4): an
  80 mm gap of 600 cells driven by the 5-loop Tesla transformer (C1 = 3.8 uF
  pre-charged to 3 kV, L1 = 47 uH, L2 = 0.13 H, k = 0.37, R1 = R2 = 5 Ohm,
  R3 = 100 MOhm, C2 = 2.8 pF, the gap being the load capacitor C3 = 0.2 pF),
  dt = 15 ns, Ti+ ions (7.95e-26 kg), electrons 1000 times heavier than
  physical (the paper's reduced mass ratio), superparticle weight 2.5e7; the
  paper's Gaussian ion pulse has no published profile, so a 100 eV Ti+ beam
  of 20 macroparticles per step enters at x = d, plus 500 pairs of 1 eV
  plasma.
* ``ensemble``: independent 5 mm gaps with cells log-uniform in 256-4096,
  initial macroparticles log-uniform in 1e4-2e6, V0 uniform in 50-200 kV,
  C uniform in 20-500 pF, SEE scale uniform in 0-2 (every 8th instance
  SEE-free), mono-energetic beam uniform in 5-50 keV at
  max(50, N_init/2000) ions per step, dt = 1 ps, FP32 particles.
"""
import math

import numpy as np

# CODATA 2018
E_CHARGE = 1.602176634e-19
M_E = 9.1093837015e-31
M_P = 1.67262192369e-27
EPS0 = 8.8541878128e-12

FP64, FP32 = 0, 1


def _base(n_cells, n_pairs, dt, steps, beam_per_step, precision, seed=0, n0=1e14):
    d = 5e-3
    C = 100e-12
    area = C * d / EPS0
    weight = n0 * d * area / n_pairs
    return dict(
        d=d, area=area, eps0=EPS0, e=E_CHARGE, m_e=M_E, m_i=M_P,
        R=50.0, L=1e-6, C=C, V0=100e3, f=1e6, tau=2e-6, polarity=-1.0,
        gamma_coef=0.05, gamma_max=3.0, E_ref_eV=1000.0, see_scale=1.0, T_emit_eV=2.0,
        # SEE laws: count 0 floor + Bernoulli, 1 Poisson; energy 0 half-Maxwellian of
        # T_emit, 1 lognormal.  The paper's lognormal parameters are not published:
        # mu = 1.0, sigma = 0.8 (ln eV) are placeholders (mode 1.4 eV, median 2.7 eV,
        # inside the below-20-eV regime the paper describes).
        see_count_law=0, see_energy_law=0, see_ln_mu=1.0, see_ln_sigma=0.8,
        beam_E_eV=20e3, beam_Emin_eV=5e3, beam_Emax_eV=50e3,
        dt=dt, weight=weight, sigma0=0.0, seed=seed,
        n_cells=n_cells, circuit=0, beam_per_step=beam_per_step, beam_mode=0,
        n_pairs=n_pairs, T_load_eV=1.0, n0=n0, steps=steps, precision=precision,
    )


def gap_1d_fp64(seed=0):
    """Small FP64 gap (256 cells, 1e4 pairs, 5000 steps)."""
    cfg = _base(256, 10_000, 1e-12, 5000, 50, FP64, seed)
    cfg["name"] = "gap_1d_fp64"
    return cfg


def gap_1d_fp32_large(seed=0):
    """Large FP32 gap (4096 cells, 1e7 macroparticles, 20000 steps)."""
    cfg = _base(4096, 5_000_000, 0.5e-12, 20000, 5000, FP32, seed)
    rng = np.random.default_rng([seed, 0xBEA])
    cfg["beam_mode"] = int(rng.integers(0, 2))  # mono-energetic or uniform 5-50 keV
    cfg["name"] = "gap_1d_fp32_large"
    return cfg


def gap_1d_fp32_thinned(seed=0, factor=25, steps=20000):
    """The large FP32 gap's distribution with factor x fewer, heavier macroparticles."""
    cfg = _base(4096, 5_000_000 // factor, 0.5e-12, steps, 5000 // factor, FP32, seed)
    rng = np.random.default_rng([seed, 0xBEA])
    cfg["beam_mode"] = int(rng.integers(0, 2))
    cfg["name"] = "gap_1d_fp32_thinned"
    return cfg


def tesla_circuit(dt):
    """The Tesla transformer of Table 3 (loop-charge parameters tR1..tV1)."""
    L1, L2, k = 47e-6, 0.13, 0.37
    return dict(dt=dt, circuit=2, tR1=5.0, tR2=5.0, tR3=100e6, tC1=3.8e-6, tC2=2.8e-12,
                tC3=0.2e-12, tL1=L1, tL2=L2, tM=k * math.sqrt(L1 * L2), tV1=3000.0)


def tesla_gap(seed=0, steps=575):
    """The paper's integrated configuration with the Tesla circuit (FP64)."""
    cfg = _base(600, 500, 15e-9, steps, 20, FP64, seed)
    cfg.update(tesla_circuit(15e-9))
    cfg["d"] = 0.08
    cfg["C"] = cfg["tC3"]
    cfg["area"] = cfg["tC3"] * cfg["d"] / EPS0  # the particle-free gap is C3
    cfg["m_i"] = 7.95e-26  # Ti+
    cfg["m_e"] = 1000.0 * M_E  # reduced mass ratio
    cfg["weight"] = 2.5e7
    cfg["beam_E_eV"] = 100.0
    # the paper's SEE sampling: Poisson counts, lognormal energies
    cfg["see_count_law"], cfg["see_energy_law"] = 1, 1
    cfg["see_scale"] = 8.0
    cfg["name"] = "tesla_gap"
    return cfg


def ensemble(n_inst=512, seed=0, steps=10000, thin=1, n_cells_max=4096):
    """Instances of the ensemble workload; `thin` divides every particle count
    (weights scaled up to keep the densities and beam currents)."""
    rng = np.random.default_rng([seed, 0xE75])
    out = []
    for i in range(n_inst):
        n_cells = int(round(math.exp(rng.uniform(math.log(256), math.log(n_cells_max)))))
        n_init = math.exp(rng.uniform(math.log(1e4), math.log(2e6)))
        n_pairs = max(16, int(n_init / 2 / thin))
        beam = max(1, int(max(50.0, n_init / 2000.0) / thin))
        cfg = _base(n_cells, n_pairs, 1e-12, steps, beam, FP32, seed=seed * 100003 + i)
        C = rng.uniform(20e-12, 500e-12)
        cfg["C"] = C
        cfg["area"] = C * cfg["d"] / EPS0
        cfg["weight"] = cfg["n0"] * cfg["d"] * cfg["area"] / n_pairs
        cfg["V0"] = rng.uniform(50e3, 200e3)
        scale = rng.uniform(0.0, 2.0)
        cfg["see_scale"] = 0.0 if i % 8 == 7 else scale
        cfg["beam_E_eV"] = rng.uniform(5e3, 50e3)
        cfg["beam_mode"] = 0
        cfg["name"] = "ensemble[%d]" % i
        out.append(cfg)
    return out


def gap_2d(seed=0, Nx=1024, Ny=1024, n_pairs=50_000_000, steps=2000, beam_per_step=None):
    """The 2D planar gap (x normal, y periodic)."""
    cfg = _base(Nx, n_pairs, 1e-12, steps, 0, FP32, seed)
    cfg["Ny"] = int(Ny)
    cfg["Ly"] = 5e-3
    cfg["beam_per_step"] = int(n_pairs // 1000 if beam_per_step is None else beam_per_step)
    cfg["beam_sigma"] = 0.5e-3
    cfg["beam_yc"] = 0.5 * cfg["Ly"]
    cfg["name"] = "gap_2d"
    return cfg


def load_pairs_2d(cfg, seed=None):
    """Co-located pairs uniform in the 2D gap, Maxwellian in both velocity
    components; returns (xi, eta, u_e, w_e, u_i, w_i) in cell units."""
    n = int(cfg["n_pairs"])
    Nx, Ny = int(cfg["n_cells"]), int(cfg["Ny"])
    rng = np.random.default_rng([int(cfg["seed"] if seed is None else seed), 0x2D10AD])
    xi = rng.random(n) * Nx
    xi = np.where(xi > 0.0, xi, 1e-9)
    eta = rng.random(n) * Ny
    dyx = (cfg["Ly"] / Ny) / (cfg["d"] / Nx)  # dy / dx
    ue = rng.standard_normal(n) * thermal_u(cfg, cfg["m_e"], cfg["T_load_eV"])
    we = rng.standard_normal(n) * thermal_u(cfg, cfg["m_e"], cfg["T_load_eV"]) / dyx
    ui = rng.standard_normal(n) * thermal_u(cfg, cfg["m_i"], cfg["T_load_eV"])
    wi = rng.standard_normal(n) * thermal_u(cfg, cfg["m_i"], cfg["T_load_eV"]) / dyx
    return xi, eta, ue, we, ui, wi


def scaled(cfg, **over):
    """Copy of a workload with some parameters replaced (weight kept unless given)."""
    out = dict(cfg)
    out.update(over)
    return out


def thermal_u(cfg, mass, T_eV):
    """Thermal speed sqrt(e T / m) expressed in cells per step."""
    dx = cfg["d"] / cfg["n_cells"]
    return math.sqrt(cfg["e"] * T_eV / mass) * cfg["dt"] / dx


def load_pairs(cfg, seed=None, n_pairs=None):
    """Co-located electron/ion pairs, uniform in the gap, Maxwellian velocities.

    Returns ``(xi, u_e, u_i)`` in FP64 cell units; ion ids are 0..n-1.
    """
    n = int(cfg["n_pairs"] if n_pairs is None else n_pairs)
    N = int(cfg["n_cells"])
    rng = np.random.default_rng([int(cfg["seed"] if seed is None else seed), 0x10AD])
    xi = rng.random(n) * N
    xi = np.where(xi > 0.0, xi, 1e-9)  # keep every particle strictly inside (0, N)
    ue = rng.standard_normal(n) * thermal_u(cfg, cfg["m_e"], cfg["T_load_eV"])
    ui = rng.standard_normal(n) * thermal_u(cfg, cfg["m_i"], cfg["T_load_eV"])
    return xi, ue, ui


def as_precision(xi, u, N, precision):
    """Round a particle set to the storage precision, keeping xi inside (0, N)."""
    if precision == FP64:
        return np.asarray(xi, np.float64), np.asarray(u, np.float64)
    x32 = np.asarray(xi, np.float64).astype(np.float32)
    hi = np.nextafter(np.float32(N), np.float32(0))
    x32 = np.minimum(x32, hi)
    x32 = np.maximum(x32, np.float32(np.finfo(np.float32).tiny))
    u32 = np.asarray(u, np.float64).astype(np.float32)
    return x32.astype(np.float64), u32.astype(np.float64)
