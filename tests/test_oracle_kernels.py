"""Pins of the oracle's per-particle building blocks: deposit, gather, push,
tridiagonal solve and SEE sampling."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W


# ---------------------------------------------------------------- deposit
def exact_deposit(N, xi, sign):
    """Brute force with exact rational arithmetic: W1 = floor(frac(xi) 2^16)."""
    G = [0] * (N + 1)
    for x in xi:
        fx = Fraction(float(x))
        i = math.floor(fx)
        W1 = math.floor((fx - i) * 2**16)
        W0 = 2**16 - W1
        if i == 0:
            W0 *= 2
        if i + 1 == N:
            W1 *= 2
        G[i] += sign * W0
        G[i + 1] += sign * W1
    return np.array(G, dtype=np.int64)


@pytest.mark.parametrize("N", [2, 7, 256])
def test_deposit_bit_exact_against_rational_brute_force(orc, N):
    rng = np.random.default_rng(N)
    xi = rng.random(300) * N
    xi = np.concatenate([xi, [1e-300, 0.5, 1.0, N - 1.0, N - 1e-9, np.nextafter(N, 0)]])
    xi = xi[(xi > 0) & (xi < N)]
    for sign in (+1, -1):
        np.testing.assert_array_equal(orc.deposit(N, xi, sign), exact_deposit(N, xi, sign))


def test_deposit_conserves_charge_with_half_end_nodes(orc):
    N = 64
    xi = np.random.default_rng(1).random(1000) * N
    G = orc.deposit(N, xi, +1)
    # each particle carries 2^16 with boundary nodes counted half
    assert G[0] % 2 == 0 and G[N] % 2 == 0
    assert G[0] // 2 + G[1:N].sum() + G[N] // 2 == 2**16 * xi.size


# ----------------------------------------------------------------- gather
def test_gather_is_linear_interpolation_between_edges(orc):
    N = 32
    a, b = 0.7, -1.3
    E = a + b * (np.arange(N) + 0.5)  # linear field sampled at half-grid points
    for xi in np.random.default_rng(2).random(200) * (N - 1) + 0.5:
        assert orc.gather(E, N, xi) == pytest.approx(a + b * xi, rel=1e-13, abs=1e-13)
    # clamped to the nearest edge value between a wall and the first edge
    assert orc.gather(E, N, 0.2) == E[0]
    assert orc.gather(E, N, N - 0.1) == E[-1]
    # exact at the edges themselves
    for k in range(N):
        assert orc.gather(E, N, k + 0.5) == E[k]


# ------------------------------------------------------------------ Thomas
def test_thomas_matches_dense_solve(orc):
    rng = np.random.default_rng(3)
    for n in (2, 5, 100):
        a, c = rng.standard_normal(n), rng.standard_normal(n)
        b = 4 + rng.random(n)
        r = rng.standard_normal(n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        np.testing.assert_allclose(orc.thomas(a, b, c, r), np.linalg.solve(A, r), rtol=1e-12,
                                   atol=1e-12)


# ------------------------------------------------------------ trajectory
@pytest.mark.parametrize("species,xi0,u0", [(1, 100.25, 0.01), (0, 30.5, -0.002)])
def test_uniform_field_trajectory_is_exact(orc, species, xi0, u0):
    """A test particle in the uniform field of a floating charged electrode
    follows x0 + v0 t + a t^2 / 2: leapfrog started with a half kick is exact
    for constant acceleration."""
    cfg = W.scaled(W.gap_1d_fp64(), circuit=1, sigma0=1e-9, weight=1e-30, beam_per_step=0)
    N = cfg["n_cells"]
    dx = cfg["d"] / N
    g = orc.OracleGap(cfg)
    g.set_particles(species, np.array([xi0]), np.array([u0]))
    steps = 300
    xs = []
    for _ in range(steps):
        assert g.step(orc.STRICT, 1) == orc.OK
        xs.append(g.particles(species)[0][0])
    E0 = cfg["sigma0"] / cfg["eps0"]
    q = cfg["e"] if species == 1 else -cfg["e"]
    m = cfg["m_i"] if species == 1 else cfg["m_e"]
    a_cells = q * E0 / m * cfg["dt"] ** 2 / dx  # cells per step^2
    n = np.arange(1, steps + 1)
    want = xi0 + u0 * n + 0.5 * a_cells * n**2
    np.testing.assert_allclose(np.array(xs), want, rtol=1e-12)
    # the field itself is uniform: sigma / eps0 on every edge
    np.testing.assert_allclose(g.grid()["E"], E0, rtol=1e-12)
    g.close()


# --------------------------------------------------------------------- SEE
@pytest.mark.parametrize("E_keV", [0.0, 1.0, 5.0, 20.0, 40.0, 80.0, 5000.0])
def test_mean_yield_over_a_million_impacts(orc, E_keV):
    cfg = W.gap_1d_fp64()
    n = 1_000_000
    counts = orc.see_count_batch(cfg, E_keV * 1e3, 7, n, 12)
    gamma = min(0.05 * math.sqrt(E_keV), 3.0)
    lo = math.floor(gamma)
    assert set(np.unique(counts)) <= {lo, lo + 1}
    frac = gamma - lo
    sigma = math.sqrt(max(frac * (1 - frac), 1e-300) / n)
    assert abs(counts.mean() - gamma) <= 5 * sigma + 1e-12
    # the scale factor multiplies the yield (0 = SEE-free)
    assert orc.see_count(W.scaled(cfg, see_scale=0.0), E_keV * 1e3, 3, 5)[0] == 0


def test_emission_energy_moments(orc):
    cfg = W.gap_1d_fp64()
    n = 1_000_000
    v, frac = orc.see_electron_batch(cfg, 11, n, 4)
    assert np.all(v >= 0)
    E_eV = 0.5 * cfg["m_e"] * v**2 / cfg["e"]
    T = cfg["T_emit_eV"]
    # half-Maxwellian of temperature T in 1D: <m v^2 / 2> = T / 2, Var = T^2 / 2
    assert abs(E_eV.mean() - T / 2) < 5 * math.sqrt(T * T / 2 / n)
    assert abs(np.mean(v) - math.sqrt(2 / math.pi) * math.sqrt(cfg["e"] * T / cfg["m_e"])) < \
        5 * math.sqrt(cfg["e"] * T / cfg["m_e"]) / math.sqrt(n)
    assert np.all((frac > 0) & (frac < 1))
    assert abs(frac.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)


def test_see_draws_are_keyed_by_ion_and_step(orc):
    cfg = W.gap_1d_fp64()
    a = orc.see_electron(cfg, 5, 9, 0)
    assert a == orc.see_electron(cfg, 5, 9, 0)
    assert a != orc.see_electron(cfg, 6, 9, 0)
    assert a != orc.see_electron(cfg, 5, 10, 0)
    assert a != orc.see_electron(cfg, 5, 9, 1)
    assert a != orc.see_electron(W.scaled(cfg, seed=1), 5, 9, 0)
