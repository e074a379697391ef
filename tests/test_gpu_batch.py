"""The ensemble path (cp_batch_*) against single-instance contexts.

Every instance of an ensemble must give bit for bit what it gives as a
context of its own: the per-particle arithmetic is the same, the charge is
integer, the draws are counter-based and the solve is an exact integer scan.
Checked on instances of uneven size and physics (the ensemble workload,
thinned), over enough steps for graph replays and removals, in strict,
weak and learned weak coupling, for every launch shape of the autotuner, and with one
instance stopping on a capacity error while the others go on.
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
    native.lib()
    return torch, native


def instances(n=6, seed=0, thin=400, n_cells_max=1024):
    cfgs = W.ensemble(n, seed=seed, steps=300, thin=thin, n_cells_max=n_cells_max)
    for c in cfgs:  # short runs: a thinner, faster-crossing gap so impacts happen
        c["d"] = 5e-4
        c["area"] = c["C"] * c["d"] / c["eps0"]
        c["weight"] = c["n0"] * c["d"] * c["area"] / c["n_pairs"]
        c["see_scale"] *= 4.0
    return cfgs


def load(cfg):
    xi, ue, ui = W.load_pairs(cfg)
    return xi, ue, ui, np.arange(xi.size, dtype=np.uint32)


def single_run(native, cfg, mode, steps):
    g = native.Gap(cfg, max_steps=steps)
    xi, ue, ui, ids = load(cfg)
    g.set_particles(native.ELECTRONS, xi, ue)
    g.set_particles(native.IONS, xi, ui, ids)
    rc = native.cp_step_strict(g.ctx, steps, 1e-12) if mode == 0 else native.cp_step_weak(g.ctx, steps)
    out = dict(rc=rc, h=g.history(), grid=g.grid(),
               parts=[g.particles(s) for s in range(3)])
    g.close()
    return out


def batch_of(native, cfgs, steps, capacity=None):
    b = native.Batch(cfgs, max_steps=steps)
    for i, cfg in enumerate(cfgs):
        xi, ue, ui, ids = load(cfg)
        b.set_particles(i, native.ELECTRONS, xi, ue)
        b.set_particles(i, native.IONS, xi, ui, ids)
    return b


def same_particles(a, b):
    for s in range(3):
        xa, ua = a[s][0], a[s][1]
        xb, ub = b[s][0], b[s][1]
        assert xa.size == xb.size, s
        oa, ob = np.lexsort((ua, xa)), np.lexsort((ub, xb))
        np.testing.assert_array_equal(xa[oa], xb[ob])
        np.testing.assert_array_equal(ua[oa], ub[ob])


def check_same(native, b, i, ref):
    h = b.history(i)
    for k in ("V_gap", "I_circ", "Q_surf", "Q_circ", "Q_conv", "residual"):
        np.testing.assert_array_equal(h[k], ref["h"][k], err_msg=k)
    for k in ("absorbed", "emitted", "injected", "n_live", "conv_count"):
        np.testing.assert_array_equal(h[k], ref["h"][k], err_msg=k)
    gr = b.grid(i)
    np.testing.assert_array_equal(gr["G"], ref["grid"]["G"])
    np.testing.assert_array_equal(gr["phi"], ref["grid"]["phi"])
    same_particles([b.particles(i, s) for s in range(3)], ref["parts"])


def predictor_of(native, cfg):
    """The hand-built persistence network (J^{n+1} = J^n) for an instance."""
    import predictor_nets as PN
    p, si, so = PN.persistence_net(cfg["C"], 1e-13)
    nm = native.cp_predictor()
    for f in range(5):
        nm.in_scale[f] = float(si[f])
    for o in range(2):
        nm.out_scale[o] = float(so[o])
    nm.bound = 0.5
    return p, nm


def test_learned_weak_ensemble_equals_single_instances(env):
    """Learned weak coupling: each instance with its own network gives bit
    for bit its single-context learned run (history including J_hat, grid,
    particles); an instance left without a network runs plain weak."""
    torch, native = env
    cfgs = instances()
    steps = 200
    with_net = [i % 3 != 2 for i in range(len(cfgs))]
    refs = []
    for i, c in enumerate(cfgs):
        g = native.Gap(c, max_steps=steps)
        xi, ue, ui, ids = load(c)
        g.set_particles(native.ELECTRONS, xi, ue)
        g.set_particles(native.IONS, xi, ui, ids)
        if with_net[i]:
            g.set_predictor(*predictor_of(native, c))
            rc = native.cp_step_weak_learned(g.ctx, steps)
        else:
            rc = native.cp_step_weak(g.ctx, steps)
        refs.append(dict(rc=rc, h=g.history(), grid=g.grid(), parts=[g.particles(s) for s in range(3)]))
        g.close()
    b = batch_of(native, cfgs, steps)
    for i, c in enumerate(cfgs):
        if with_net[i]:
            b.set_predictor(i, *predictor_of(native, c))
    assert b.step(native.WEAK_LEARNED, steps) == native.OK
    for i in range(len(cfgs)):
        check_same(native, b, i, refs[i])
        np.testing.assert_array_equal(b.history(i)["J_hat"], refs[i]["h"]["J_hat"])
    b.close()
    used = [int((r["h"]["J_hat"] != 0).sum()) for r in refs]
    assert all(u == 0 for u, w in zip(used, with_net) if not w)
    assert sum(used) > 100, used  # the learned path was exercised


def test_ensemble_training_samples_equal_single_runs(env):
    """The predictor's training samples read from an ensemble of strict runs
    are those of the same runs as contexts of their own, bit for bit."""
    torch, native = env
    cfgs = instances(n=3)
    steps = 120
    n = steps - native.PRED_WINDOW
    b = batch_of(native, cfgs, steps)
    assert b.step(native.STRICT, steps) == native.OK
    for i, cfg in enumerate(cfgs):
        Xb = torch.empty((n, native.MLP_IN), dtype=torch.float32, device="cuda")
        Yb = torch.empty((n, native.MLP_OUT), dtype=torch.float32, device="cuda")
        b.predictor_samples(i, native.PRED_WINDOW, n, Xb.data_ptr(), Yb.data_ptr())
        g = native.Gap(cfg, max_steps=steps)
        xi, ue, ui, ids = load(cfg)
        g.set_particles(native.ELECTRONS, xi, ue)
        g.set_particles(native.IONS, xi, ui, ids)
        assert native.cp_step_strict(g.ctx, steps, 1e-12) == native.OK
        Xs = torch.empty_like(Xb)
        Ys = torch.empty_like(Yb)
        assert native.cp_predictor_samples(g.ctx, native.PRED_WINDOW, n, Xs.data_ptr(),
                                           Ys.data_ptr()) == native.OK
        torch.cuda.synchronize()
        g.close()
        assert torch.equal(Xb, Xs) and torch.equal(Yb, Ys)
    b.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_equals_single_instances(env, mode):
    torch, native = env
    cfgs = instances()
    steps = 200  # three removals; graph replays of 64 steps
    refs = [single_run(native, c, mode, steps) for c in cfgs]
    b = batch_of(native, cfgs, steps)
    assert b.step(mode, steps) == native.OK
    assert b.last_launch_count() > 0
    for i in range(len(cfgs)):
        check_same(native, b, i, refs[i])
    b.close()
    # the runs exercised impacts, emission and the beam
    assert sum(r["h"]["emitted"][:, 0].sum() for r in refs) > 30
    assert sum(r["h"]["absorbed"][:, 0, 1].sum() for r in refs) > 50


def test_every_launch_shape_gives_the_same_bits(env):
    torch, native = env
    cfgs = instances(n=5, seed=3)
    steps = 90
    ref = None
    shapes = [(512, 2), (512, 1), (256, 2), (256, 1), (1024, 1)]
    ran = 0
    for threads, per_sm in shapes:
        b = batch_of(native, cfgs, steps)
        assert b.step(0, 1) == native.OK  # first step: set-up with the default shape
        if b.set_launch(threads, per_sm) != native.OK:
            b.close()
            continue
        assert b.launch()[0] == threads
        assert b.step(0, steps - 1) == native.OK
        hs = [b.history(i) for i in range(len(cfgs))]
        b.close()
        ran += 1
        if ref is None:
            ref = hs
            continue
        for i in range(len(cfgs)):
            np.testing.assert_array_equal(hs[i]["V_gap"], ref[i]["V_gap"])
            np.testing.assert_array_equal(hs[i]["n_live"], ref[i]["n_live"])
    assert ran >= 3


def test_autotune_keeps_the_run(env):
    torch, native = env
    cfgs = instances(n=4, seed=5)
    steps = 120
    refs = [single_run(native, c, 0, steps) for c in cfgs]
    b = batch_of(native, cfgs, steps)
    rc, threads, per_sm, ms = b.autotune(4)
    assert rc == native.OK and threads in (256, 512, 1024) and per_sm >= 1 and ms > 0
    assert b.launch()[0] == threads
    lv = b.level
    assert lv >= 4 * 3  # the tuner's trial steps are steps of the run
    assert b.step(0, steps - lv) == native.OK
    for i in range(len(cfgs)):
        check_same(native, b, i, refs[i])
    b.close()


def test_a_failing_instance_stops_alone(env):
    torch, native = env
    cfgs = instances(n=4, seed=7)
    steps = 100
    # instance 2: room for its loaded ions and a few beam steps only
    cfgs[2] = dict(cfgs[2])
    cap_ions = cfgs[2]["n_pairs"] + 4 * cfgs[2]["beam_per_step"]
    # the batch takes the capacities of its runs: instance 2 gets a small ion store
    n = len(cfgs)
    G, Cc, S, R = ((native.cp_gap * n)(), (native.cp_circuit * n)(), (native.cp_see_beam * n)(),
                   (native.cp_run * n)())
    for i, cfg in enumerate(cfgs):
        cap = (0, (cap_ions + 64 + 3) // 4 * 4, 0) if i == 2 else (0, 0, 0)
        g_, c_, s_, r_ = native.structs_from_config(cfg, capacity=cap, max_steps=steps)
        G[i], Cc[i], S[i], R[i] = g_, c_, s_, r_
    import ctypes as C
    h = C.c_void_p()
    assert native.lib().cp_batch_create(n, G, Cc, S, R, C.c_void_p(native.current_stream()),
                                        C.byref(h)) == native.OK
    bb = native.Batch.__new__(native.Batch)
    bb.h, bb.n, bb.cfgs = h, n, cfgs
    for i, cfg in enumerate(cfgs):
        xi, ue, ui, ids = load(cfg)
        bb.set_particles(i, native.ELECTRONS, xi, ue)
        bb.set_particles(i, native.IONS, xi, ui, ids)
    rc = bb.step(0, steps)
    assert rc == native.ERR_CAPACITY
    st = bb.status()
    assert st[2] == native.ERR_CAPACITY and np.all(st[[0, 1, 3]] == 0)
    for i in (0, 1, 3):
        ref = single_run(native, cfgs[i], 0, steps)
        np.testing.assert_array_equal(bb.history(i)["V_gap"], ref["h"]["V_gap"])
    assert bb.history(2)["V_gap"].size < steps + 1  # stopped early
    bb.close()


def test_ensemble_instances_match_the_oracle(env, orc):
    """Four uneven instances of one ensemble against the FP64 oracle run of
    each: the level-0 charge grid bit for bit, then 300 strict steps with
    impacts and emission, V_gap, I_circ and Q_surf within 0.5 % and the
    cumulative event counts within the FP32 event-shift allowance."""
    torch, native = env
    cfgs = instances(4, seed=3, thin=400)
    steps = 300
    b = batch_of(native, cfgs, steps)
    b.step(0, 0)
    G0 = [b.grid(i)["G"].copy() for i in range(len(cfgs))]
    b.step(0, steps)
    assert (b.status() == 0).all()
    emitted = 0
    for i, cfg in enumerate(cfgs):
        xi, ue, ui, ids = load(cfg)
        N = cfg["n_cells"]
        xe, ue32 = W.as_precision(xi, ue, N, W.FP32)
        xo, ui32 = W.as_precision(xi, ui, N, W.FP32)
        r = orc.OracleGap(cfg)
        r.set_particles(orc.ELECTRONS, xe, ue32)
        r.set_particles(orc.IONS, xo, ui32, ids)
        assert r.step(orc.STRICT, 0) == orc.OK
        np.testing.assert_array_equal(G0[i], r.grid()["G"])
        assert r.step(orc.STRICT, steps) == orc.OK
        hr = r.history()
        r.close()
        hg = b.history(i)
        assert len(hg["V_gap"]) == len(hr["V_gap"])
        for k in ("V_gap", "I_circ", "Q_surf"):
            s = np.abs(hr[k]).max()
            assert np.abs(hg[k] - hr[k]).max() <= 5e-3 * s, (i, k)
        for a, c in ((hg["absorbed"][:, 0, 1], hr["absorbed"][:, 0, 1]),
                     (hg["emitted"][:, 0], hr["emitted"][:, 0]),
                     (hg["conv_count"], hr["conv_count"])):
            ca, cb = np.cumsum(a), np.cumsum(c)
            assert np.all(np.abs(ca - cb) <= 3 * cfg["beam_per_step"] + 0.01 * np.abs(cb)), i
        emitted += int(hr["emitted"][:, 0].sum())
    b.close()
    assert emitted > 20  # the run reaches secondary emission
