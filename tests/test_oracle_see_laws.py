"""Pins of the paper's SEE sampling laws in the oracle (Sec. 2.3, Algorithm
see_sampling_1d): n_SE ~ Poisson(mean yield), E_SE ~ Lognormal(mu, sigma)
with v = sqrt(2 E / m_e).  (The paper's fitted yield polynomial and
lognormal parameters are not published; the workload's yield law and
placeholder mu, sigma stand in -- the sampling is what is pinned.)

* Poisson counts over 10^6 impacts at three mean yields: mean and variance
  within 5 sigma, the zero-count fraction exp(-gamma), and a chi-square test
  of the whole distribution.
* Lognormal energies over 2 x 10^5 electrons: ln(E / 1 eV) has mean mu and
  variance sigma^2 (5 sigma) and passes a Kolmogorov-Smirnov test against
  the normal distribution; emission is normal to the wall.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2603_24010_gb300 import workloads as W


def gap_with_laws(count_law, energy_law, scale=1.0):
    return W.scaled(W.gap_1d_fp64(), see_count_law=count_law, see_energy_law=energy_law,
                    see_scale=scale, gamma_max=14.0)


@pytest.mark.parametrize("E_keV", [20.0, 80.0, 600.0])
def test_poisson_counts(orc, E_keV):
    cfg = gap_with_laws(1, 0, scale=3.0)
    n = 1_000_000
    counts = orc.see_count_batch(cfg, E_keV * 1e3, 1000, n, 17)
    gam = min(cfg["see_scale"] * cfg["gamma_coef"] * math.sqrt(E_keV), cfg["gamma_max"])
    assert abs(counts.mean() - gam) < 5 * math.sqrt(gam / n)
    # variance of a Poisson variable is its mean; the sample variance's sd is
    # sqrt((mu4 - sigma^4) / n) = sqrt((gam + 2 gam^2) / n)
    assert abs(counts.var() - gam) < 5 * math.sqrt((gam + 2 * gam * gam) / n)
    p0 = math.exp(-gam)
    assert abs((counts == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / n)
    kmax = int(gam + 8 * math.sqrt(gam) + 5)
    obs = np.bincount(np.minimum(counts, kmax), minlength=kmax + 1)
    pmf = stats.poisson.pmf(np.arange(kmax + 1), gam)
    pmf[kmax] = stats.poisson.sf(kmax - 1, gam)
    keep = pmf * n > 20
    exp_ = pmf[keep] * n
    chi2 = ((obs[keep] - exp_) ** 2 / exp_).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_bernoulli_law_unchanged(orc):
    """The workload's law: floor(gamma) + Bernoulli, counts in {2, 3}."""
    cfg = gap_with_laws(0, 0, scale=3.0)
    counts = orc.see_count_batch(cfg, 80e3, 0, 200_000, 3)
    gam = 3.0 * 0.05 * math.sqrt(80.0)
    assert set(np.unique(counts)) <= {math.floor(gam), math.floor(gam) + 1}


def test_lognormal_energies(orc):
    cfg = gap_with_laws(0, 1)
    n = 200_000
    v, frac = orc.see_electron_batch(cfg, 7, n, 11)
    E_eV = 0.5 * cfg["m_e"] * v * v / cfg["e"]
    y = np.log(E_eV)
    mu, sg = cfg["see_ln_mu"], cfg["see_ln_sigma"]
    assert abs(y.mean() - mu) < 5 * sg / math.sqrt(n)
    assert abs(y.var() / (sg * sg) - 1) < 5 * math.sqrt(2 / n)
    assert stats.kstest((y - mu) / sg, "norm").pvalue > 1e-4
    assert np.all(v > 0) and np.all((frac > 0) & (frac < 1))
