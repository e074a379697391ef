"""Pins of the oracle's initial plasma (co-located electron/ion pairs).

The gap starts filled with a uniform plasma at temperature T (the paper's
runs start from a loaded plasma, Sec. 3.1; density and temperature are the
workload's).  Checked against what the distribution must be, over 2 x 10^5
pairs:

* positions uniform in (0, N): mean, variance and Kolmogorov-Smirnov;
* each species' velocity normal with variance e T / m (in cells per step):
  mean, variance and Kolmogorov-Smirnov, for two temperatures;
* electron and ion velocities of a pair independent (correlation ~ 0);
* co-located pairs: the deposited charge is exactly zero at every node;
* the same seed gives the same load, another seed another.
"""
import math

import numpy as np
import pytest
from scipy.stats import kstest

from paper_2603_24010_gb300 import workloads as W

N_PAIRS = 200_000


def thermal(cfg, m, T):
    dx = cfg["d"] / cfg["n_cells"]
    return math.sqrt(cfg["e"] * T / m) * cfg["dt"] / dx


@pytest.mark.parametrize("T", [1.0, 25.0])
def test_load_moments(orc, T):
    cfg = W.gap_1d_fp32_large(0)
    N = cfg["n_cells"]
    xi, ue, ui = orc.load_pairs(cfg, N_PAIRS, T, 1234)
    n = N_PAIRS
    assert np.all(xi > 0) and np.all(xi < N)
    assert abs(xi.mean() - N / 2) < 5 * N / math.sqrt(12 * n)
    assert abs(xi.var() - N * N / 12) < 5 * 0.0745 * N * N / math.sqrt(n)
    assert kstest(xi / N, "uniform").pvalue > 1e-4
    for u, m in ((ue, cfg["m_e"]), (ui, cfg["m_i"])):
        s = thermal(cfg, m, T)
        assert abs(u.mean()) < 5 * s / math.sqrt(n)
        assert abs(u.var() / (s * s) - 1) < 5 * math.sqrt(2 / n)
        assert kstest(u / s, "norm").pvalue > 1e-4
    corr = np.corrcoef(ue, ui)[0, 1]
    assert abs(corr) < 5 / math.sqrt(n)


def test_load_is_neutral_and_seeded(orc):
    cfg = W.gap_1d_fp64()
    N = cfg["n_cells"]
    xi, ue, ui = orc.load_pairs(cfg, 10_000, 1.0, 7)
    G = orc.deposit(N, xi, -1)
    orc.deposit(N, xi, +1, G)
    assert not G.any()
    x2, ue2, ui2 = orc.load_pairs(cfg, 10_000, 1.0, 7)
    np.testing.assert_array_equal(xi, x2)
    np.testing.assert_array_equal(ue, ue2)
    x3, _, _ = orc.load_pairs(cfg, 10_000, 1.0, 8)
    assert np.mean(x3 == xi) < 1e-3
    # a prefix of a larger load is the smaller load (pair k depends on k alone)
    x4, ue4, _ = orc.load_pairs(cfg, 20_000, 1.0, 7)
    np.testing.assert_array_equal(x4[:10_000], xi)
    np.testing.assert_array_equal(ue4[:10_000], ue)
