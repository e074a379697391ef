"""The paper's SEE sampling laws (Sec. 2.3, Algorithm see_sampling_1d:
Poisson counts, lognormal energies) on the GPU against the oracle.

Ions placed just inside the driven electrode hit it in their first push; a
vanishing field keeps the impact velocities those of the stored values, so
the Poisson counts, the convection count and the emitted electrons must be
the oracle's: counts exactly, electrons to the last bits of the two
platforms' exp/log/cos (FP64 1e-12, FP32 one float ulp).  An ensemble
instance with the same laws equals its single-context run bit for bit.
"""
import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24010_gb300 import native
    native.lib()
    return native


def impacts(cfg, n, seed):
    rng = np.random.default_rng(seed)
    N = cfg["n_cells"]
    dx = cfg["d"] / N
    E_keV = rng.random(n) * 80 + 1
    u = -np.sqrt(2 * E_keV * 1e3 * cfg["e"] / cfg["m_i"]) * cfg["dt"] / dx
    xi = (rng.random(n) * 0.9 + 0.01) * np.abs(u)
    xi, u = W.as_precision(xi, u, N, cfg["precision"])
    return xi, u, rng.permutation(10 * n)[:n].astype(np.uint32)


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
@pytest.mark.parametrize("count_law,energy_law", [(1, 0), (0, 1), (1, 1)])
def test_see_laws_match_oracle(nat, orc, precision, count_law, energy_law):
    cfg = W.scaled(W.gap_1d_fp64(), beam_per_step=0, see_scale=12.0, gamma_max=14.0,
                   precision=precision, weight=1e-30, circuit=orc.OPEN,
                   see_count_law=count_law, see_energy_law=energy_law)
    N = cfg["n_cells"]
    xi, u, ids = impacts(cfg, 3000, 21 + count_law + 2 * energy_law)
    g = nat.Gap(cfg, max_steps=4)
    g.set_particles(nat.IONS, xi, u, ids)
    r = orc.OracleGap(cfg)
    r.set_particles(orc.IONS, xi, u, ids)
    g.step(0, 1)
    assert r.step(orc.STRICT, 1) == orc.OK
    hg, hr = g.history(), r.history()
    np.testing.assert_array_equal(hg["emitted"], hr["emitted"])
    np.testing.assert_array_equal(hg["conv_count"], hr["conv_count"])
    assert hr["emitted"][1, 0] > 3000
    xg, ug, _ = g.particles(nat.SECONDARIES)
    xr, ur, _ = r.particles(orc.SECONDARIES)
    xr, ur = W.as_precision(xr, ur, N, precision)
    og, orr = np.lexsort((ug, xg)), np.lexsort((ur, xr))
    tol = 1e-12 if precision == W.FP64 else 2**-23
    np.testing.assert_allclose(xg[og], xr[orr], rtol=tol, atol=0)
    np.testing.assert_allclose(ug[og], ur[orr], rtol=tol, atol=0)
    g.close()
    r.close()


def test_ensemble_instance_with_the_paper_laws(nat):
    cfgs = W.ensemble(3, seed=5, steps=200, thin=400, n_cells_max=512)
    for c in cfgs:
        c["d"] = 5e-4
        c["area"] = c["C"] * c["d"] / c["eps0"]
        c["weight"] = c["n0"] * c["d"] * c["area"] / c["n_pairs"]
        c["see_scale"] = 6.0
        c["see_count_law"], c["see_energy_law"] = 1, 1
    steps = 200
    b = nat.Batch(cfgs, max_steps=steps)
    loads = [W.load_pairs(c) for c in cfgs]
    for i, (xi, ue, ui) in enumerate(loads):
        b.set_particles(i, nat.ELECTRONS, xi, ue)
        b.set_particles(i, nat.IONS, xi, ui, np.arange(xi.size, dtype=np.uint32))
    assert b.step(0, steps) == 0
    emitted = 0
    for i, c in enumerate(cfgs):
        g = nat.Gap(c, max_steps=steps)
        xi, ue, ui = loads[i]
        g.set_particles(nat.ELECTRONS, xi, ue)
        g.set_particles(nat.IONS, xi, ui, np.arange(xi.size, dtype=np.uint32))
        g.step(0, steps)
        h, hb = g.history(), b.history(i)
        for k in ("V_gap", "Q_surf", "emitted", "n_live", "conv_count"):
            np.testing.assert_array_equal(hb[k], h[k], err_msg=k)
        emitted += int(h["emitted"].sum())
        g.close()
    b.close()
    assert emitted > 10
