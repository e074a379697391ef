"""Pins of the 2D gap oracle (transverse-periodic extension of the 1D cycle).

* The bilinear fixed-point deposit equals an exact-rational brute force and
  carries 2^16 per macroparticle (end nodes in x counted half).
* The transverse-FFT solve equals a dense solve of the whole 2D discrete
  system (five-point Laplacian, equipotential electrodes, Gauss row on the
  transverse mean) on small grids.
* A test charge in the uniform field of a surface charge follows the
  analytic trajectory in x and drifts (periodically) in y.
* Coupled runs conserve the grid's charge and the particle ledger, and the
  beam's transverse profile has the stated centre and width.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W


@pytest.fixture(scope="module")
def g2(orc):
    from oracle import gap2d
    return gap2d


def small2d(seed=0, Nx=16, Ny=8, n_pairs=300, beam=4, circuit=0):
    cfg = W.gap_2d(seed, Nx=Nx, Ny=Ny, n_pairs=n_pairs, steps=50, beam_per_step=beam)
    cfg["circuit"] = circuit
    return cfg


def test_deposit_matches_exact_rationals(g2):
    rng = np.random.default_rng(1)
    Nx, Ny = 7, 5
    xi = np.concatenate([rng.random(200) * Nx, [1e-9, Nx - 1e-9, 3.0, 0.5]])
    eta = np.concatenate([rng.random(200) * Ny, [0.0, Ny - 1e-9, 2.0, 4.999]])
    G = g2.deposit2d(Nx, Ny, xi, eta, +1)
    want = np.zeros((Nx + 1, Ny), dtype=object)
    for x, y in zip(xi, eta):
        fx, fy = Fraction(x), Fraction(y)
        i, j = int(fx // 1), int(fy // 1)
        F = 65536  # 2^16 per axis
        wx1 = int((fx - i) * F // 1)
        wy1 = int((fy - j) * F // 1)
        for ii, jj, w in ((i, j, (F - wx1) * (F - wy1)), (i + 1, j, wx1 * (F - wy1)),
                          (i, (j + 1) % Ny, (F - wx1) * wy1), (i + 1, (j + 1) % Ny, wx1 * wy1)):
            want[ii, jj] += w * (2 if ii in (0, Nx) else 1)
    np.testing.assert_array_equal(G, want.astype(np.int64))
    half = G.copy()
    half[0] //= 2
    half[Nx] //= 2
    assert half.sum() == 2**32 * xi.size


@pytest.mark.parametrize("Nx,Ny", [(6, 4), (9, 8)])
def test_fft_solve_equals_dense_2d_system(g2, Nx, Ny):
    rng = np.random.default_rng(Nx)
    cfg = small2d(Nx=Nx, Ny=Ny, circuit=1)  # open circuit: the electrode row is Gauss's law
    cfg["area"] = cfg["C"] * cfg["d"] / cfg["eps0"]
    G = g2.deposit2d(Nx, Ny, rng.random(60) * Nx, rng.random(60) * Ny, +1)
    G = g2.deposit2d(Nx, Ny, rng.random(40) * Nx, rng.random(40) * Ny, -1, G)
    sigma = 3e-9
    rc, phi, Ex, Ey, out = g2.solve2d(cfg, 0, G, 0, sigma, np.zeros(4), 0.0, 0.0)
    assert rc == 0
    dx, dy = cfg["d"] / Nx, cfg["Ly"] / Ny
    Lz = cfg["area"] / cfg["Ly"]
    rho = G * cfg["e"] * cfg["weight"] / (dx * dy * Lz * 2.0**32)
    eps0 = cfg["eps0"]
    # unknowns: V (electrode) then phi[i, j] for i = 1..Nx-1
    idx = lambda i, j: 1 + (i - 1) * Ny + (j % Ny)  # noqa: E731
    n = 1 + (Nx - 1) * Ny
    M = np.zeros((n, n))
    b = np.zeros(n)
    r2 = (dx / dy) ** 2
    for i in range(1, Nx):
        for j in range(Ny):
            row = idx(i, j)
            M[row, row] += -2.0 - 2.0 * r2
            for (ii, jj, c) in ((i - 1, j, 1.0), (i + 1, j, 1.0), (i, j - 1, r2), (i, j + 1, r2)):
                if ii == 0:
                    M[row, 0] += c
                elif ii < Nx:
                    M[row, idx(ii, jj)] += c
            b[row] = -dx * dx * rho[i, j] / eps0
    # electrode row: Gauss's law on the transverse mean, V - mean(phi_1) = dx sigma/eps0 + dx^2 mean(rho_0)/(2 eps0)
    M[0, 0] = 1.0
    for j in range(Ny):
        M[0, idx(1, j)] -= 1.0 / Ny
    b[0] = dx * sigma / eps0 + dx * dx * rho[0].mean() / (2 * eps0)
    x = np.linalg.solve(M, b)
    want = np.zeros((Nx + 1, Ny))
    want[0, :] = x[0]
    for i in range(1, Nx):
        want[i] = x[idx(i, 0):idx(i, 0) + Ny]
    np.testing.assert_allclose(phi, want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_test_charge_in_uniform_field(g2, orc):
    from oracle import gap2d
    cfg = small2d(Nx=16, Ny=8, n_pairs=1, beam=0, circuit=1)
    cfg["sigma0"] = 2e-9
    cfg["weight"] = 1e-30  # negligible space charge
    o = gap2d.Oracle2D(cfg)
    # one ion and one electron, both with a transverse velocity
    o.set_particles(1, [8.3], [2.5], [0.0], [0.37])
    o.set_particles(0, [7.1], [6.9], [0.0], [-0.21])
    steps = 30
    assert o.step(0, steps) == orc.OK
    dx, dy, dt = cfg["d"] / 16, cfg["Ly"] / 8, cfg["dt"]
    E = cfg["sigma0"] / cfg["eps0"]
    for s, x0, y0, w0, q, m in ((1, 8.3, 2.5, 0.37, 1, cfg["m_i"]), (0, 7.1, 6.9, -0.21, -1, cfg["m_e"])):
        a = q * cfg["e"] * E / m
        T = steps * dt
        x = x0 + 0.5 * a * T * T / dx  # from rest (leapfrog started with a half kick)
        y = (y0 + w0 * steps) % 8
        assert o.p[s]["xi"][0] == pytest.approx(x, rel=1e-12)
        assert o.p[s]["eta"][0] == pytest.approx(y, rel=1e-12)
        assert np.all(o.Ey == pytest.approx(0.0, abs=1e-9 * E))


def test_coupled_run_conserves_charge_and_particles(g2, orc):
    from oracle import gap2d
    cfg = small2d(Nx=16, Ny=8, n_pairs=400, beam=6)
    cfg["d"] = cfg["Ly"] = 5e-4
    cfg["area"] = cfg["C"] * cfg["d"] / cfg["eps0"]
    cfg["weight"] = cfg["n0"] * cfg["d"] * cfg["area"] / cfg["n_pairs"]
    cfg["see_scale"] = 8.0
    cfg["beam_yc"], cfg["beam_sigma"] = 2.5e-4, 5e-5
    xi, eta, ue, we, ui, wi = W.load_pairs_2d(cfg)
    o = gap2d.Oracle2D(cfg)
    o.set_particles(0, xi, eta, ue, we)
    o.set_particles(1, xi, eta, ui, wi)
    assert o.step(0, 400) == orc.OK
    h = o.history()
    assert h["absorbed"][:, 0, 1].sum() > 10 and h["emitted"][:, 0].sum() > 0
    nl = h["n_live"]
    G = o.G.copy()
    G[0] //= 2
    G[-1] //= 2
    assert G.sum() == 2**32 * (nl[-1, 1] - nl[-1, 0] - nl[-1, 2])
    ab = h["absorbed"]
    np.testing.assert_array_equal(np.diff(nl[:, 1]), -ab[1:, :, 1].sum(axis=1) + 6)
    np.testing.assert_array_equal(np.diff(nl[:, 2]), -ab[1:, :, 2].sum(axis=1) + h["emitted"][1:].sum(axis=1))
    # loop charge = surface-charge change - convection (strict)
    qw = cfg["e"] * cfg["weight"]
    assert h["Q_circ"][-1] == pytest.approx(h["Q_surf"][-1] - qw * h["conv_count"].sum(),
                                            rel=1e-9, abs=1e-9 * abs(h["Q_surf"]).max())


def test_beam_profile(g2, orc):
    from oracle import gap2d
    cfg = small2d(Nx=64, Ny=64, n_pairs=1, beam=200)
    o = gap2d.Oracle2D(cfg)
    o.set_particles(1, [32.0], [1.0], [0.0], [0.0])
    assert o.step(1, 10) == orc.OK
    eta = o.p[1]["eta"][1:]
    dy = cfg["Ly"] / 64
    assert eta.size == 2000
    assert eta.mean() * dy == pytest.approx(cfg["beam_yc"], abs=4 * cfg["beam_sigma"] / np.sqrt(2000))
    assert eta.std() * dy == pytest.approx(cfg["beam_sigma"], rel=0.08)
