"""The 2D planar gap on the GPU against the 2D oracle.

* The bilinear fixed-point deposit is bit-exact on identical particle sets
  (window path with several work items per tile, and the global path on a
  grid too narrow for windows).
* The level-0 fields equal the oracle's transverse-FFT solve (FP32 modes
  around the FP64 mean).
* One push from identical states agrees to FP32 rounding; a coupled run with
  beam and SEE tracks the oracle's V_gap and circuit charge.
* Results do not depend on how often the store is re-sorted (window and
  global paths share their arithmetic).  At full size (1024 x 1024 cells,
  2e7 pairs) the charge and particle ledgers are exact, the grid is the
  oracle's deposit of the GPU's particles and the fields are the oracle's
  solve of that grid.
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
    from oracle import gap2d
    native.lib()
    return torch, native, gap2d


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def loaded(cfg):
    xi, eta, ue, we, ui, wi = W.load_pairs_2d(cfg)
    xi = np.minimum(f32(xi), np.nextafter(np.float32(cfg["n_cells"]), np.float32(0)))
    eta = f32(eta)
    eta = np.where(eta >= cfg["Ny"], 0.0, eta)
    return xi, eta, f32(ue), f32(we), f32(ui), f32(wi)


def gpu_gap(native, cfg, steps, mode=0, sort_every=0, parts=None):
    g = native.Gap2D(cfg, max_steps=max(steps, 1), sort_every=sort_every)
    xi, eta, ue, we, ui, wi = parts if parts is not None else loaded(cfg)
    g.set_particles(native.ELECTRONS, xi, eta, ue, we)
    g.set_particles(native.IONS, xi, eta, ui, wi, np.arange(xi.size, dtype=np.uint32))
    g.step(mode, steps)
    return g


def oracle_gap(gap2d, cfg, steps, mode=0, parts=None):
    o = gap2d.Oracle2D(cfg)
    xi, eta, ue, we, ui, wi = parts if parts is not None else loaded(cfg)
    o.set_particles(0, xi, eta, ue, we)
    o.set_particles(1, xi, eta, ui, wi)
    assert o.step(mode, steps) == 0
    return o


def cfg2d(Nx, Ny, n_pairs, beam=0, gap=5e-3, see=1.0):
    cfg = W.gap_2d(0, Nx=Nx, Ny=Ny, n_pairs=n_pairs, steps=10, beam_per_step=beam)
    cfg["d"] = cfg["Ly"] = gap
    cfg["area"] = cfg["C"] * cfg["d"] / cfg["eps0"]
    cfg["weight"] = cfg["n0"] * cfg["d"] * cfg["area"] / cfg["n_pairs"]
    cfg["beam_yc"], cfg["beam_sigma"] = gap / 2, gap / 10
    cfg["see_scale"] = see
    return cfg


@pytest.mark.parametrize("Nx,Ny,n_pairs", [(64, 64, 150000), (96, 128, 40000), (40, 8, 20000)])
def test_level0_deposit_and_fields(env, Nx, Ny, n_pairs):
    torch, native, gap2d = env
    cfg = cfg2d(Nx, Ny, n_pairs)
    parts = loaded(cfg)
    g = gpu_gap(native, cfg, 0, parts=parts)
    f = g.fields()
    g.close()
    o = oracle_gap(gap2d, cfg, 0, parts=parts)
    np.testing.assert_array_equal(f["G"], o.G)
    scale = np.abs(o.phi).max()
    np.testing.assert_allclose(f["phi"], o.phi, rtol=0, atol=2e-5 * scale)
    ex_s = np.abs(o.Ex).max()
    np.testing.assert_allclose(f["Ex"], o.Ex, rtol=0, atol=2e-4 * ex_s)
    np.testing.assert_allclose(f["Ey"], o.Ey, rtol=0, atol=2e-4 * ex_s)


def test_one_push_matches_the_oracle(env):
    torch, native, gap2d = env
    cfg = cfg2d(64, 64, 30000)
    parts = loaded(cfg)
    g = gpu_gap(native, cfg, 1, parts=parts)
    o = oracle_gap(gap2d, cfg, 1, parts=parts)
    # ions are matched by id
    xg, yg, ug, wg, ids = g.particles(native.IONS)
    q = o.p[native.IONS]
    og, oo = np.argsort(ids), np.argsort(o.ids)
    np.testing.assert_array_equal(ids[og], o.ids[oo].astype(np.uint32))
    for a_, b_, tol in ((xg, q["xi"], 2e-5), (yg, q["eta"], 2e-5), (ug, q["u"], 1e-6),
                        (wg, q["w"], 1e-6)):
        np.testing.assert_allclose(a_[og], b_[oo], rtol=0, atol=tol * max(1.0, np.abs(b_).max()))
    # electrons (no ids): each coordinate's sorted values
    xg, yg, ug, wg, _ = g.particles(native.ELECTRONS)
    q = o.p[native.ELECTRONS]
    assert xg.size == q["xi"].size
    for a_, b_ in ((xg, q["xi"]), (yg, q["eta"]), (ug, q["u"]), (wg, q["w"])):
        np.testing.assert_allclose(np.sort(a_), np.sort(b_), rtol=0,
                                   atol=2e-5 * max(1.0, np.abs(b_).max()))
    # the level-1 grid is the oracle's deposit of the GPU's own positions, bit
    # for bit (the deposit is exact on identical particle sets) ...
    G = g.fields()["G"]
    Gd = np.zeros_like(o.G)
    for sp, sign in ((native.ELECTRONS, -1), (native.IONS, 1), (native.SECONDARIES, -1)):
        xs, ys, _, _, _ = g.particles(sp)
        if xs.size:
            gap2d.deposit2d(cfg["n_cells"], cfg["Ny"], xs, ys, sign, Gd)
    np.testing.assert_array_equal(G, Gd)
    # ... and differs from the oracle's (FP64 positions) only by the FP32
    # rounding of the positions: a particle within ulp(N) of its FP64 position
    # moves at most 2 ulp(N) 2^32 between its nodes, summed over a node's
    # particles; same total charge
    half = lambda a: np.concatenate([a[:1] // 2, a[1:-1], a[-1:] // 2])  # noqa: E731
    assert half(G).sum() == half(o.G).sum()  # 2^32 per macroparticle on both sides
    ulp = float(np.spacing(np.float32(cfg["n_cells"])))
    per_node = 2 * 2 * 30000 * 4 / G.size  # mean contributions to a node (both species)
    assert np.abs(G - o.G).max() <= 4 * ulp * 2.0**32 * 8 * per_node
    g.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_coupled_run_tracks_the_oracle(env, mode):
    torch, native, gap2d = env
    cfg = cfg2d(64, 64, 8000, beam=24, gap=5e-4, see=8.0)
    steps = 300
    g = gpu_gap(native, cfg, steps, mode=mode)
    hg = g.history()
    g.close()
    o = oracle_gap(gap2d, cfg, steps, mode=mode)
    ho = o.history()
    assert ho["absorbed"][:, 0, 1].sum() > 20 and ho["emitted"][:, 0].sum() > 5
    for k in ("V_gap", "Q_surf", "Q_circ"):
        scale = np.abs(ho[k]).max()
        np.testing.assert_allclose(hg[k], ho[k], rtol=0, atol=5e-3 * scale, err_msg=k)


def test_learned_weak_coupling_of_the_mean(env):
    """Learned weak coupling in 2D with the hand-built persistence network
    (J_hat^{n+1} = J^n of the transverse mean): the network's prediction for
    each level is the realised J of the level before (from the run's own
    history), and with it the weak run tracks the strict one more closely
    than the plain weak run."""
    torch, native, gap2d = env
    import predictor_nets as PN
    cfg = cfg2d(64, 64, 8000, beam=24, gap=5e-4, see=8.0)
    steps = 300
    parts = loaded(cfg)
    runs = {}
    for mode in (0, 1):
        g = gpu_gap(native, cfg, steps, mode=mode, parts=parts)
        runs[mode] = g.history()
        g.close()
    hw = runs[1]
    C = cfg["C"]
    Jw = C * np.diff(hw["V_gap"]) - np.diff(hw["Q_circ"])  # J^n, n = 1..steps
    S = float(np.abs(Jw).max()) / 10.0  # keeps the network in its linear range
    p, si, so = PN.persistence_net(C, S)
    nm = native.cp_predictor()
    for f in range(5):
        nm.in_scale[f] = float(si[f])
    for o in range(2):
        nm.out_scale[o] = float(so[o])
    nm.bound = 0.5
    g = native.Gap2D(cfg, max_steps=steps)
    xi, eta, ue, we, ui, wi = parts
    g.set_particles(native.ELECTRONS, xi, eta, ue, we)
    g.set_particles(native.IONS, xi, eta, ui, wi, np.arange(xi.size, dtype=np.uint32))
    g.set_predictor(p, nm)
    g.step(native.WEAK_LEARNED, steps)
    hl = g.history()
    g.close()
    used = hl["J_hat"] != 0
    assert used.sum() > 200, used.sum()
    J = C * np.diff(hl["V_gap"]) - np.diff(hl["Q_circ"])  # J[k] = J^{k+1}
    n = np.nonzero(used[2:])[0] + 2  # levels n with a prediction, n >= 2
    np.testing.assert_allclose(hl["J_hat"][n], J[n - 2], rtol=0, atol=1e-3 * np.abs(J).max())
    hs = runs[0]
    err = lambda h: np.abs(h["V_gap"] - hs["V_gap"]).max() / np.abs(hs["V_gap"]).max()
    assert err(hl) < err(hw), (err(hl), err(hw))


def test_results_do_not_depend_on_the_sort_interval(env):
    torch, native, gap2d = env
    cfg = cfg2d(64, 64, 60000, beam=40, gap=5e-4, see=4.0)
    steps = 40
    parts = loaded(cfg)
    hs = []
    for every in (1, 3, 8):
        g = gpu_gap(native, cfg, steps, sort_every=every, parts=parts)
        hs.append((g.history(), g.fields()["G"]))
        g.close()
    for h, G in hs[1:]:
        np.testing.assert_array_equal(h["V_gap"], hs[0][0]["V_gap"])
        np.testing.assert_array_equal(h["n_live"], hs[0][0]["n_live"])
        np.testing.assert_array_equal(G, hs[0][1])


def test_full_size_ledgers_and_fields(env):
    """1024 x 1024 cells, 2e7 pairs, 2e4 beam ions per step, 12 steps: the
    charge and particle ledgers are exact, the charge grid equals the
    oracle's deposit of the GPU's own particles bit for bit, and the fields
    equal the oracle's solve of that grid with the GPU's circuit state (the
    level-0 test's tolerances)."""
    torch, native, gap2d = env
    cfg = W.gap_2d(0, n_pairs=20_000_000)
    cfg["beam_per_step"] = 20000
    parts = loaded(cfg)
    steps = 12
    g = gpu_gap(native, cfg, steps, parts=parts)
    h = g.history()
    f = g.fields()
    G = f["G"].copy()
    Nx, Ny = int(cfg["n_cells"]), int(cfg["Ny"])
    Go = np.zeros((Nx + 1, Ny), dtype=np.int64)
    for sp, sign in ((native.ELECTRONS, -1), (native.IONS, 1), (native.SECONDARIES, -1)):
        xi, eta = g.particles(sp)[:2]
        if xi.size:
            gap2d.deposit2d(Nx, Ny, xi, eta, sign, Go)
    g.close()
    nl = h["n_live"]
    assert nl[0, 0] == 20_000_000
    np.testing.assert_array_equal(np.diff(nl[:, 1]), -h["absorbed"][1:, :, 1].sum(axis=1) + 20000)
    np.testing.assert_array_equal(G, Go)
    Gh = G.copy()
    Gh[0] //= 2
    Gh[-1] //= 2
    assert Gh.sum() == 2**32 * (nl[-1, 1] - nl[-1, 0] - nl[-1, 2])
    assert np.all(h["residual"] <= 1e-12)
    # the oracle's solve of the last level from the GPU's grid and circuit state
    n = steps
    Qc = h["Q_circ"]
    Qhist = np.array([Qc[n - 1 - k] if n - 1 - k >= 0 else 0.0 for k in range(4)])
    rc, phi, Ex, Ey, out = gap2d.solve2d(cfg, 0, G, int(h["conv_count"][n]),
                                         h["Q_surf"][n - 1] / cfg["area"], Qhist,
                                         n * cfg["dt"], h["V_gap"][n - 1])
    assert rc == 0
    scale = np.abs(phi).max()
    ex_s = np.abs(Ex).max()
    np.testing.assert_allclose(f["phi"], phi, rtol=0, atol=2e-5 * scale)
    np.testing.assert_allclose(f["Ex"], Ex, rtol=0, atol=2e-4 * ex_s)
    np.testing.assert_allclose(f["Ey"], Ey, rtol=0, atol=2e-4 * ex_s)
    assert h["V_gap"][n] == pytest.approx(phi[0, 0], rel=1e-9)
