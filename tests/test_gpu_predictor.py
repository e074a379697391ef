"""The predictor network's CUDA kernels and the learned weak scheme.

* Batch forward, loss + gradient and Adam against the FP64 oracle network
  (same BF16-rounded weights), on several tiles with a ragged tail.
* Initialisation, scales, normalisation and training samples against their
  definitions.
* The in-solve inference against the batch forward on the same windows.
* The learned weak scheme against the oracle's with the same hand-built
  persistence network.
* Training on strict runs gains over the plain weak scheme on held-out seeds.
"""
import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W
from test_oracle_invariants import small_gap
import predictor_nets as PN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24010_gb300 import native
    native.lib()
    return torch, native


def dev(torch, a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(PN.NP, dtype=np.float32)
    for name, (o, i) in (("W1", (64, 40)), ("W2", (64, 64)), ("W3", (64, 64)), ("W4", (2, 64))):
        p[PN.OFF[name]:PN.OFF[name] + o * i] = rng.uniform(-1, 1, o * i) * np.sqrt(6.0 / i)
    for name, n in (("b1", 64), ("b2", 64), ("b3", 64), ("b4", 2)):
        p[PN.OFF[name]:PN.OFF[name] + n] = rng.normal(0, 0.1, n)
    return p


@pytest.mark.parametrize("n", [1, 33, 3000])
def test_forward_matches_oracle(env, orc, n):
    torch, native = env
    p = random_params(n)
    X = np.random.default_rng(n + 7).normal(0, 1, (n, 40)).astype(np.float32)
    Yh = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    assert native.cp_mlp_forward(dev(torch, p).data_ptr(), dev(torch, X).data_ptr(), n,
                                 Yh.data_ptr()) == native.OK
    want = orc.mlp_forward(p, X.astype(np.float64))
    got = Yh.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5 * np.abs(want).max())


@pytest.mark.parametrize("n", [1, 33, 3000])
def test_loss_gradient_matches_oracle(env, orc, n):
    torch, native = env
    p = random_params(100 + n)
    rng = np.random.default_rng(n)
    X = rng.normal(0, 1, (n, 40)).astype(np.float32)
    Y = rng.normal(0, 1, (n, 2)).astype(np.float32)
    g = torch.empty(PN.NP, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(native.cp_mlp_work_floats(), dtype=torch.float32, device="cuda")
    pd, Xd, Yd = dev(torch, p), dev(torch, X), dev(torch, Y)
    assert native.cp_mlp_loss_grad(pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), n, g.data_ptr(),
                                   loss.data_ptr(), work.data_ptr()) == native.OK
    want_loss, want = orc.mlp_loss_grad(p, X.astype(np.float64), Y.astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(want_loss, rel=2e-5)
    for name, size in (("W1", 2560), ("b1", 64), ("W2", 4096), ("b2", 64), ("W3", 4096),
                       ("b3", 64), ("W4", 128), ("b4", 2)):
        sl = slice(PN.OFF[name], PN.OFF[name] + size)
        np.testing.assert_allclose(got[sl], want[sl], rtol=0,
                                   atol=1e-4 * np.abs(want[sl]).max(), err_msg=name)
    # deterministic: a second call gives the same bits
    g2 = torch.empty_like(g)
    assert native.cp_mlp_loss_grad(pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), n, g2.data_ptr(),
                                   loss.data_ptr(), work.data_ptr()) == native.OK
    assert torch.equal(g, g2)


def test_adam_matches_oracle(env, orc):
    torch, native = env
    rng = np.random.default_rng(9)
    p0 = rng.normal(0, 1, PN.NP).astype(np.float32)
    pd, md, vd = dev(torch, p0), torch.zeros(PN.NP, device="cuda"), torch.zeros(PN.NP, device="cuda")
    p, m, v = p0.astype(np.float64), np.zeros(PN.NP), np.zeros(PN.NP)
    for t in range(1, 4):
        gr = rng.normal(0, 1, PN.NP).astype(np.float32)
        assert native.cp_mlp_adam(pd.data_ptr(), dev(torch, gr).data_ptr(), md.data_ptr(),
                                  vd.data_ptr(), t, 1e-2) == native.OK
        orc.adam(p, gr.astype(np.float64), m, v, t, 1e-2)
    np.testing.assert_allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)


def test_init_scales_and_normalize(env):
    torch, native = env
    a = torch.empty(PN.NP, device="cuda")
    b = torch.empty(PN.NP, device="cuda")
    native.cp_mlp_init(a.data_ptr(), 5)
    native.cp_mlp_init(b.data_ptr(), 5)
    pa = a.cpu().numpy()
    assert torch.equal(a, b)
    for name, (o, i) in (("W1", (64, 40)), ("W2", (64, 64)), ("W4", (2, 64))):
        w = pa[PN.OFF[name]:PN.OFF[name] + o * i]
        assert np.abs(w).max() <= np.sqrt(6.0 / i) and np.abs(w).max() > 0.9 * np.sqrt(6.0 / i)
    for name, n in (("b1", 64), ("b3", 64), ("b4", 2)):
        assert np.all(pa[PN.OFF[name]:PN.OFF[name] + n] == 0)
    rng = np.random.default_rng(3)
    n = 777
    X = (rng.normal(0, 1, (n, 40)) * np.tile([1e-13, 3.0, 2e-13, 10.0, 5e4], 8)).astype(np.float32)
    Y = (rng.normal(0, 1, (n, 2)) * [1e-13, 4e-14]).astype(np.float32)
    norm = native.cp_predictor()
    assert native.cp_mlp_scales(dev(torch, X).data_ptr(), dev(torch, Y).data_ptr(), n,
                                norm) == native.OK
    Xd = X.astype(np.float64).reshape(n, 8, 5)
    for f in range(5):
        assert norm.in_scale[f] == pytest.approx(np.sqrt(np.mean(Xd[:, :, f] ** 2)), rel=1e-6)
    for o in range(2):
        assert norm.out_scale[o] == pytest.approx(np.sqrt(np.mean(Y[:, o].astype(np.float64) ** 2)),
                                                  rel=1e-6)
    Xn = torch.empty((n, 40), device="cuda")
    Yn = torch.empty((n, 2), device="cuda")
    assert native.cp_mlp_normalize(dev(torch, X).data_ptr(), dev(torch, Y).data_ptr(), n, norm,
                                   Xn.data_ptr(), Yn.data_ptr()) == native.OK
    si = np.tile(np.array(norm.in_scale[:], dtype=np.float32), 8)
    np.testing.assert_array_equal(Xn.cpu().numpy(), X / si)
    np.testing.assert_array_equal(Yn.cpu().numpy(),
                                  Y / np.array(norm.out_scale[:], dtype=np.float32))


def gpu_gap(native, cfg, steps, mode=0, net=None):
    g = native.Gap(cfg, max_steps=steps)
    xi, ue, ui = W.load_pairs(cfg)
    g.set_particles(native.ELECTRONS, xi, ue)
    g.set_particles(native.IONS, xi, ui, np.arange(xi.size, dtype=np.uint32))
    if net is not None:
        g.set_predictor(*net)
    g.step(mode, steps)
    return g


def norm_of(native, in_scale, out_scale, bound):
    nm = native.cp_predictor()
    for f in range(5):
        nm.in_scale[f] = float(in_scale[f])
    for o in range(2):
        nm.out_scale[o] = float(out_scale[o])
    nm.bound = float(bound)
    return nm


def test_samples_follow_their_definition(env):
    torch, native = env
    cfg = small_gap()
    steps = 80
    g = gpu_gap(native, cfg, steps)
    h = g.history()
    n = steps - 8
    X = torch.empty((n, 40), device="cuda")
    Y = torch.empty((n, 2), device="cuda")
    assert native.cp_predictor_samples(g.ctx, 8, n, X.data_ptr(), Y.data_ptr()) == native.OK
    assert native.cp_predictor_samples(g.ctx, 8, n + 1, X.data_ptr(), Y.data_ptr()) == native.ERR_ARG
    assert native.cp_predictor_samples(g.ctx, 7, 1, X.data_ptr(), Y.data_ptr()) == native.ERR_ARG
    torch.cuda.synchronize()
    g.close()
    Xg, Yg = X.cpu().numpy(), Y.cpu().numpy()
    for k in (0, 1, 37, n - 1):
        L = 8 + k
        for j in range(8):
            m = L - 7 + j
            row = [h["Q_conv"][m], h["V_gap"][m] - h["V_gap"][m - 1],
                   h["Q_surf"][m] - h["Q_surf"][m - 1], float(h["emitted"][m, 0]),
                   h["ion_energy_eV"][m]]
            np.testing.assert_array_equal(Xg[k, 5 * j:5 * j + 5], np.array(row).astype(np.float32))
        J = cfg["C"] * (h["V_gap"][L + 1] - h["V_gap"][L]) - (h["Q_circ"][L + 1] - h["Q_circ"][L])
        assert Yg[k, 0] == np.float32(h["Q_conv"][L + 1])
        assert Yg[k, 1] == pytest.approx(J, rel=1e-6, abs=1e-30)


def test_in_solve_inference_matches_batch_forward(env):
    torch, native = env
    cfg = small_gap()
    steps = 120
    p = random_params(21) * np.float32(0.3)
    S = 1e-13
    nm = norm_of(native, [S, S / cfg["C"], S, 1.0, 100.0], [S, S], 1e30)  # always trusted
    g = gpu_gap(native, cfg, steps, mode=native.WEAK_LEARNED, net=(p, nm))
    h = g.history()
    n = steps - 8
    X = torch.empty((n, 40), device="cuda")
    Y = torch.empty((n, 2), device="cuda")
    assert native.cp_predictor_samples(g.ctx, 8, n, X.data_ptr(), Y.data_ptr()) == native.OK
    Xn = torch.empty_like(X)
    assert native.cp_mlp_normalize(X.data_ptr(), None, n, nm, Xn.data_ptr(), None) == native.OK
    Yh = torch.empty((n, 2), device="cuda")
    assert native.cp_mlp_forward(dev(torch, p).data_ptr(), Xn.data_ptr(), n,
                                 Yh.data_ptr()) == native.OK
    torch.cuda.synchronize()
    g.close()
    yh = Yh.cpu().numpy().astype(np.float64)
    J_batch = S * yh[:, 1]  # prediction for level 8 + k + 1
    used = h["J_hat"] != 0
    assert not used[:25].any() and used[25:].all()
    lv = np.arange(25, steps + 1)
    np.testing.assert_allclose(h["J_hat"][lv], J_batch[lv - 9], rtol=1e-4,
                               atol=1e-5 * np.abs(J_batch).max())


def test_learned_weak_matches_oracle(env, orc):
    torch, native = env
    cfg = small_gap()
    steps = 300
    p, si, so = PN.persistence_net(cfg["C"], 1e-13)
    g = gpu_gap(native, cfg, steps, mode=native.WEAK_LEARNED, net=(p, norm_of(native, si, so, 0.5)))
    hg = g.history()
    g.close()
    o = orc.OracleGap(cfg)
    xi, ue, ui = W.load_pairs(cfg)
    o.set_particles(orc.ELECTRONS, xi, ue)
    o.set_particles(orc.IONS, xi, ui)
    o.set_predictor(p, si.astype(np.float64), so.astype(np.float64), 0.5)
    assert o.step(orc.WEAK_LEARNED, steps) == orc.OK
    ho = o.history()
    o.close()
    np.testing.assert_array_equal(hg["J_hat"] != 0, ho["J_hat"] != 0)
    assert (ho["J_hat"] != 0).sum() > 250
    np.testing.assert_allclose(hg["J_hat"], ho["J_hat"], rtol=1e-4,
                               atol=1e-4 * np.abs(ho["J_hat"]).max())
    np.testing.assert_allclose(hg["V_gap"], ho["V_gap"], rtol=0,
                               atol=1e-6 * np.abs(ho["V_gap"]).max())


def test_trained_predictor_beats_plain_weak(env):
    """Train on strict runs of one workload family, then on held-out seeds the
    learned weak scheme is closer to strict than the plain weak scheme."""
    torch, native = env
    from paper_2603_24010_gb300 import predictor as PR
    steps = 6000
    fam = [W.gap_1d_fp32_thinned(seed, factor=250, steps=steps) for seed in range(10)]
    Xs, Ys = zip(*(PR.strict_samples(cfg) for cfg in fam[:8]))
    X, Y = torch.cat(Xs), torch.cat(Ys)
    params, norm, losses = PR.train(X, Y, iters=1500, batch=4096, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    for cfg in fam[8:]:
        res = PR.evaluate(cfg, params, norm)
        err = PR.vgap_errors(res)
        used = (res[native.WEAK_LEARNED]["J_hat"] != 0).mean()
        assert used > 0.5
        assert err[native.WEAK_LEARNED] < 0.7 * err[native.WEAK], (err, used)
