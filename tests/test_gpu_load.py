"""The initial plasma drawn on the device (cp_load_species) against the oracle.

* Positions equal the oracle's bit for bit (one Philox draw and one
  correctly rounded product, then the store's rounding); velocities agree
  to the last bits of the platforms' log/cos/sin (FP64: 1e-14 relative;
  FP32: within one float ulp); ion ids are 0..n-1.
* The level-0 charge grid is exactly zero (co-located pairs).
* A coupled run from the device load tracks the oracle run from its own
  load of the same seed.
* At the large gap's full size (5e6 pairs, FP32) every position matches.
"""
import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24010_gb300 import native
    from oracle import oracle as orc
    native.lib()
    orc.lib()
    return torch, native, orc


def oracle_load(orc, cfg, n, T, seed):
    xi, ue, ui = orc.load_pairs(cfg, n, T, seed)
    xe, ue = W.as_precision(xi, ue, cfg["n_cells"], cfg["precision"])
    xo, ui = W.as_precision(xi, ui, cfg["n_cells"], cfg["precision"])
    return xe, ue, xo, ui


def close_velocities(a, b, precision):
    if precision == W.FP64:
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)
    else:
        a32, b32 = a.astype(np.float32), b.astype(np.float32)
        ulps = np.abs(a32.view(np.int32).astype(np.int64) - b32.view(np.int32).astype(np.int64))
        assert ulps.max() <= 1, ulps.max()


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_load_matches_the_oracle(env, precision):
    torch, native, orc = env
    cfg = W.scaled(W.gap_1d_fp64(seed=3), precision=precision)
    n, T, seed = 50_000, 1.0, 77
    g = native.Gap(cfg, max_steps=4)
    g.load_species(n, T, seed)
    g.step(native.STRICT, 0)
    xe, ue, xo, ui = oracle_load(orc, cfg, n, T, seed)
    gx, gu = g.particles(native.ELECTRONS)[:2]
    ix, iu, ids = g.particles(native.IONS)
    assert not g.grid()["G"].any()
    g.close()
    # particles come back in store order (slot k = pair k)
    np.testing.assert_array_equal(gx, xe)
    np.testing.assert_array_equal(ix, xo)
    np.testing.assert_array_equal(ids, np.arange(n, dtype=np.uint32))
    close_velocities(gu, ue, precision)
    close_velocities(iu, ui, precision)


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_run_from_the_device_load_tracks_the_oracle(env, precision):
    torch, native, orc = env
    cfg = W.scaled(W.gap_1d_fp64(seed=4), precision=precision, n_pairs=8000)
    cfg["weight"] = cfg["n0"] * cfg["d"] * cfg["area"] / cfg["n_pairs"]
    steps = 60
    g = native.Gap(cfg, max_steps=steps)
    g.load_species(cfg["n_pairs"], cfg["T_load_eV"], 11, n0=cfg["n0"])
    g.step(native.STRICT, steps)
    hg, Eg = g.history(), g.grid()["E"]
    g.close()
    r = orc.OracleGap(cfg)
    xe, ue, xo, ui = oracle_load(orc, cfg, cfg["n_pairs"], cfg["T_load_eV"], 11)
    r.set_particles(orc.ELECTRONS, xe, ue)
    r.set_particles(orc.IONS, xo, ui)
    assert r.step(orc.STRICT, steps) == orc.OK
    hr, Er = r.history(), r.grid()["E"]
    r.close()
    tol = 1e-9 if precision == W.FP64 else 8e-5
    assert np.abs(Eg - Er).max() <= tol * np.abs(Er).max()
    scale = np.abs(hr["V_gap"]).max()
    assert np.abs(hg["V_gap"] - hr["V_gap"]).max() <= tol * scale
    if precision == W.FP64:
        np.testing.assert_array_equal(hg["n_live"], hr["n_live"])
    else:  # an FP32 position may cross a wall one step earlier or later
        assert np.abs(hg["n_live"] - hr["n_live"]).max() <= 3


def test_full_size_load(env):
    torch, native, orc = env
    cfg = W.gap_1d_fp32_large(0)
    n = cfg["n_pairs"]
    g = native.Gap(cfg, max_steps=2)
    g.load_species(n, cfg["T_load_eV"], 0)
    g.step(native.STRICT, 0)
    gx = g.particles(native.ELECTRONS)[0]
    ix, iu, ids = g.particles(native.IONS)
    assert not g.grid()["G"].any()
    g.close()
    xe, _, _, ui = oracle_load(orc, cfg, n, cfg["T_load_eV"], 0)
    np.testing.assert_array_equal(gx, xe)
    np.testing.assert_array_equal(ix, xe)
    np.testing.assert_array_equal(ids, np.arange(n, dtype=np.uint32))
    close_velocities(iu, ui, W.FP32)


def test_load_arguments(env):
    torch, native, orc = env
    cfg = W.scaled(W.gap_1d_fp64(), precision=W.FP32)
    g = native.Gap(cfg, max_steps=2)
    assert native.cp_load_species(g.ctx, -1, 1.0, 0) == native.ERR_ARG
    assert native.cp_load_species(g.ctx, 10, float("nan"), 0) == native.ERR_ARG
    assert native.cp_load_species(g.ctx, 10, -1.0, 0) == native.ERR_ARG
    assert native.cp_load_species(g.ctx, 100, 1.0, 0) == native.OK
    # electrons and ions now come from the load; secondaries may still be set
    assert native.cp_set_particles(g.ctx, native.IONS, np.array([1.5]), np.zeros(1)) == native.ERR_ARG
    assert native.cp_set_particles(g.ctx, native.SECONDARIES, np.array([1.5]), np.zeros(1)) == native.OK
    g.step(native.STRICT, 1)
    assert native.cp_load_species(g.ctx, 100, 1.0, 0) == native.ERR_ARG  # after the first step
    g.close()
