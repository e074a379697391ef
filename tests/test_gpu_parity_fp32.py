"""FP32 particles (the benchmarked push) through ion impacts, against the
FP64 oracle.

* Secondary emission (Sec. 2.3, Algorithm see_sampling_1d) from ions that
  hit the driven electrode in their first push, with a vanishing field so
  that both sides see the same impact velocities: emitted counts and the
  convection count (Sec. 2.4.1) are equal, the emitted electrons equal the
  oracle's to FP32 rounding, and the absorbed-ion energy tally is equal.
* A 4096-cell gap of the large workload's physics, thinned 250 times
  (2e4 pairs, 20 beam ions per step), for 6000 steps: the beam crosses the
  gap (about 5100 steps at 20 keV) and SEE starts.  FP32 positions differ
  from FP64 ones by about ulp(N) = 2^-12 cells, so an absorption can happen
  one step earlier or later than in the oracle; cumulative absorbed,
  emitted and convection counts are compared at every step within that
  event-shift allowance, and V_gap, I_circ and Q_surf within 0.5 % over the
  whole run (strict and weak coupling, mono-energetic and uniform beams).
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


def rel(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / s if s > 0 else np.max(np.abs(a - b))


def test_fp32_see_matches_oracle(nat, orc):
    cfg = W.scaled(W.gap_1d_fp64(), beam_per_step=0, see_scale=20.0, gamma_max=3.0,
                   precision=W.FP32, weight=1e-30, circuit=orc.OPEN)
    N = cfg["n_cells"]
    rng = np.random.default_rng(15)
    n = 4000
    E_keV = rng.random(n) * 80 + 1
    dx = cfg["d"] / N
    u = -np.sqrt(2 * E_keV * 1e3 * cfg["e"] / cfg["m_i"]) * cfg["dt"] / dx
    xi = (rng.random(n) * 0.9 + 0.01) * np.abs(u)  # every ion reaches x = 0 in one push
    xi, u = W.as_precision(xi, u, N, W.FP32)
    ids = rng.permutation(10 * n)[:n].astype(np.uint32)
    g = nat.Gap(cfg, max_steps=4)
    g.set_particles(nat.IONS, xi, u, ids)
    r = orc.OracleGap(cfg)
    r.set_particles(orc.IONS, xi, u, ids)
    g.step(0, 1)
    assert r.step(orc.STRICT, 1) == orc.OK
    hg, hr = g.history(), r.history()
    np.testing.assert_array_equal(hg["absorbed"], hr["absorbed"])
    np.testing.assert_array_equal(hg["emitted"], hr["emitted"])
    np.testing.assert_array_equal(hg["conv_count"], hr["conv_count"])
    assert hr["emitted"][1, 0] > n
    assert hg["ion_energy_eV"][1] == hr["ion_energy_eV"][1]
    xg, ug, _ = g.particles(nat.SECONDARIES)
    xr, ur, _ = r.particles(orc.SECONDARIES)
    xr32, ur32 = W.as_precision(xr, ur, N, W.FP32)
    og, orr = np.lexsort((ug, xg)), np.lexsort((ur32, xr32))
    # the oracle's FP64 electron, rounded to FP32: equal up to the last bit of
    # the two libraries' log/cos
    np.testing.assert_allclose(xg[og], xr32[orr], rtol=2**-23, atol=0)
    np.testing.assert_allclose(ug[og], ur32[orr], rtol=2**-23, atol=0)
    g.close()
    r.close()


def thinned(seed, steps):
    cfg = W.gap_1d_fp32_thinned(seed, factor=250, steps=steps)
    return cfg


# (coupling, seed): strict with the mono-energetic 20 keV beam (seed 1), weak
# with the uniform 5-50 keV beam (seed 0)
@pytest.mark.parametrize("mode,seed", [(0, 1), (1, 0)])
def test_fp32_run_through_impacts(nat, orc, mode, seed):
    steps = 6000
    cfg = thinned(seed, steps)
    assert cfg["beam_mode"] == (0 if seed == 1 else 1)
    xi, ue, ui = W.load_pairs(cfg)
    N = cfg["n_cells"]
    xe, ue = W.as_precision(xi, ue, N, W.FP32)
    xo, ui = W.as_precision(xi, ui, N, W.FP32)
    g = nat.Gap(cfg, max_steps=steps)
    g.set_particles(nat.ELECTRONS, xe, ue)
    g.set_particles(nat.IONS, xo, ui)
    g.step(mode, steps)
    hg = g.history()
    g.close()
    r = orc.OracleGap(cfg)
    r.set_particles(orc.ELECTRONS, xe, ue)
    r.set_particles(orc.IONS, xo, ui)
    assert r.step(mode, steps) == orc.OK
    hr = r.history()
    r.close()
    # the run reaches the regime of interest: ion impacts and emission at x = 0
    assert hr["absorbed"][:, 0, 1].sum() > 2000
    assert hr["emitted"][:, 0].sum() > 100
    # cumulative event counts: an event may move by a step, a few may differ
    for name, a, b in (("ions absorbed at x = 0", hg["absorbed"][:, 0, 1], hr["absorbed"][:, 0, 1]),
                       ("electrons absorbed at x = 0", hg["absorbed"][:, 0, 0], hr["absorbed"][:, 0, 0]),
                       ("electrons absorbed at x = d", hg["absorbed"][:, 1, 0], hr["absorbed"][:, 1, 0]),
                       ("emitted at x = 0", hg["emitted"][:, 0], hr["emitted"][:, 0]),
                       ("convection count", hg["conv_count"], hr["conv_count"])):
        ca, cb = np.cumsum(a), np.cumsum(b)
        allow = 3 * cfg["beam_per_step"] + 0.01 * np.abs(cb)
        bad = np.abs(ca - cb) > allow
        assert not bad.any(), (name, int(np.argmax(bad)), ca[bad][:3], cb[bad][:3])
    np.testing.assert_array_equal(hg["injected"], hr["injected"])
    for k in ("V_gap", "I_circ", "Q_surf"):
        e = rel(hg[k], hr[k])
        assert e < 5e-3, (k, e)


@pytest.mark.parametrize("seed", [1, 0])
def test_pushed_grid_is_the_deposit_of_the_pushed_particles(nat, orc, seed):
    """After pushes with a beam in flight (ions of one step fly together, so
    a warp's deposits fall on a few nodes and are summed per node before the
    atomics), the charge grid of every level equals the oracle's deposit of
    the GPU's own particles, bit for bit."""
    cfg = thinned(seed, 400)
    cfg = W.scaled(cfg, beam_per_step=600)  # clusters of beam ions in every tile
    xi, ue, ui = W.load_pairs(cfg)
    N = cfg["n_cells"]
    xe, ue = W.as_precision(xi, ue, N, W.FP32)
    xo, ui = W.as_precision(xi, ui, N, W.FP32)
    g = nat.Gap(cfg, max_steps=400, compact_every=64)
    g.set_particles(nat.ELECTRONS, xe, ue)
    g.set_particles(nat.IONS, xo, ui)
    for n in (1, 37, 130, 300):
        g.step(0, n - g.level)
        G = g.grid()["G"]
        want = np.zeros(N + 1, dtype=np.int64)
        for sp, sign in ((nat.ELECTRONS, -1), (nat.IONS, 1), (nat.SECONDARIES, -1)):
            x = g.particles(sp)[0]
            if x.size:
                orc.deposit(N, x, sign, want)
        np.testing.assert_array_equal(G, want)
    g.close()


@pytest.mark.parametrize("beam_mode", [0, 1])
def test_beam_ions_take_their_computed_slots(nat, orc, beam_mode):
    """Beam ions of a push are stored at slots n_proc + k in the order of
    their index k (no shared counter), with ids base + step B + k, and their
    entry positions and speeds equal the oracle's rounded to FP32 (Sec. 3.2;
    mono-energetic and uniform beams).  Every CTA takes ceil(B / 304) of them,
    so B = 1000 spreads them over all CTAs unevenly."""
    cfg = W.scaled(W.gap_1d_fp64(seed=5), precision=W.FP32, beam_per_step=1000,
                   weight=1e-30, circuit=orc.OPEN)
    cfg["beam_mode"] = beam_mode
    N = cfg["n_cells"]
    rng = np.random.default_rng(3)
    n0 = 4001  # not a multiple of 4: the first slot after the padding is n_proc
    xi = rng.uniform(0.3, N - 0.3, n0)
    ui = np.zeros(n0)
    xi, ui = W.as_precision(xi, ui, N, W.FP32)
    g = nat.Gap(cfg, max_steps=4)
    g.set_particles(nat.IONS, xi, ui)
    r = orc.OracleGap(cfg)
    r.set_particles(orc.IONS, xi, ui)
    for n in (1, 2):
        g.step(0, 1)
        assert r.step(orc.STRICT, 1) == orc.OK
        gx, gu, gid = g.particles(nat.IONS)
        rx, ru, rid = r.particles(orc.IONS)
        B = cfg["beam_per_step"]
        # the newest B ions of both stores, in index order
        np.testing.assert_array_equal(gid[-B:], rid[-B:].astype(np.uint32))
        np.testing.assert_array_equal(np.diff(gid[-B:].astype(np.int64)), np.ones(B - 1))
        rx32, ru32 = W.as_precision(rx[-B:], ru[-B:], N, W.FP32)
        np.testing.assert_allclose(gx[-B:], rx32, rtol=2**-23, atol=0)
        np.testing.assert_allclose(gu[-B:], ru32, rtol=2**-23, atol=0)
    g.close()
    r.close()

