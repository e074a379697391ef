"""The allocation-free ion push against the context path.

``cp_push_ions_noalloc`` serves callers that cannot call cudaMalloc (a step
run inside a real-time loop, or a process that must not grow device memory
after start-up): it takes every buffer from the caller and keeps its
absorbed-ion list in a static device array.  Here the caller's buffers come
from torch; the same ions pushed by a context (cp_set_particles +
cp_step_strict) must give the same charge grid, survivors, emitted electrons
and tallies -- on two calls in a row, since the static array keeps the
previous call's contents.
"""
import ctypes as C

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


def ion_set(cfg, seed, n):
    """Ions near x = 0 heading into it (most are absorbed) and ions in the bulk."""
    rng = np.random.default_rng(seed)
    N = cfg["n_cells"]
    dx = cfg["d"] / N
    E_keV = rng.random(n) * 60 + 2
    u = -np.sqrt(2 * E_keV * 1e3 * cfg["e"] / cfg["m_i"]) * cfg["dt"] / dx
    xi = np.where(rng.random(n) < 0.7, (rng.random(n) * 0.9 + 0.01) * np.abs(u),
                  rng.random(n) * (N - 2) + 1)
    xi, u = W.as_precision(xi, u, N, W.FP32)
    ids = rng.permutation(20 * n)[:n].astype(np.uint32)
    return xi, u, ids


def context_step(native, cfg, xi, u, ids):
    g = native.Gap(cfg, max_steps=4)
    g.set_particles(native.IONS, xi, u, ids)
    g.step(0, 0)
    E0 = g.grid()["E"].copy()
    g.step(0, 1)
    out = dict(E0=E0, G=g.grid()["G"], ions=g.particles(native.IONS)[:2],
               se=g.particles(native.SECONDARIES)[:2], h=g.history(1, 1))
    g.close()
    return out


def noalloc_step(torch, native, cfg, xi, u, ids, E0):
    dev = torch.device("cuda")
    N = cfg["n_cells"]
    gap, _, see, run = native.structs_from_config(cfg)
    n = xi.size
    x_t = torch.tensor(xi, dtype=torch.float32, device=dev)
    u_t = torch.tensor(u, dtype=torch.float32, device=dev)
    id_t = torch.tensor(ids.view(np.int32), dtype=torch.int32, device=dev)
    E_t = torch.tensor(E0, dtype=torch.float64, device=dev)
    G_t = torch.full((N + 1,), -7, dtype=torch.int64, device=dev)  # overwritten by the call
    cap = 4 * n + 16
    sx = torch.zeros(cap, dtype=torch.float32, device=dev)
    su = torch.zeros(cap, dtype=torch.float32, device=dev)
    counts = torch.zeros(6, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    rc = native.cp_push_ions_noalloc(gap, see, cfg["dt"], cfg["seed"], 0, 1, E_t.data_ptr(),
                                     x_t.data_ptr(), u_t.data_ptr(), id_t.data_ptr(), n,
                                     G_t.data_ptr(), sx.data_ptr(), su.data_ptr(), cap,
                                     counts.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == native.OK, native.cp_status_str(rc)
    c = counts.cpu().numpy()
    xs, us = x_t.cpu().numpy().astype(np.float64), u_t.cpu().numpy().astype(np.float64)
    live = xs > 0
    m = int(c[4])
    return dict(G=G_t.cpu().numpy(), ions=(xs[live], us[live]),
                se=(sx.cpu().numpy()[:m].astype(np.float64), su.cpu().numpy()[:m].astype(np.float64)),
                counts=c)


def same_multiset(a, b):
    oa, ob = np.lexsort((a[1], a[0])), np.lexsort((b[1], b[0]))
    np.testing.assert_array_equal(a[0][oa], b[0][ob])
    np.testing.assert_array_equal(a[1][oa], b[1][ob])


@pytest.mark.parametrize("call", [0, 1])
def test_noalloc_push_matches_context_path(env, call):
    """Run as two calls in a row (the parametrisation) with different ion sets
    and SEE strength; each is compared with a fresh context doing its first step."""
    torch, native = env
    cfg = W.scaled(W.gap_1d_fp64(seed=3 + call), beam_per_step=0, see_scale=[20.0, 8.0][call],
                   precision=W.FP32)
    xi, u, ids = ion_set(cfg, 11 + call, [3000, 5000][call])
    ref = context_step(native, cfg, xi, u, ids)
    got = noalloc_step(torch, native, cfg, xi, u, ids, ref["E0"])
    h = ref["h"]
    c = got["counts"]
    assert c[0] == h["absorbed"][0, 0, 1] and c[1] == h["absorbed"][0, 1, 1]
    assert c[2] == h["emitted"][0, 0] and c[3] == h["emitted"][0, 1]
    assert c[4] == h["n_live"][0, 2] and c[5] == h["conv_count"][0]
    assert c[0] > 1000 and c[2] > 1000  # the impacts and emission really happened
    np.testing.assert_array_equal(got["G"], ref["G"])
    same_multiset(got["ions"], ref["ions"])
    same_multiset(got["se"], ref["se"])


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, native = env
    cfg = W.scaled(W.gap_1d_fp64(), precision=W.FP32)
    gap, _, see, _ = native.structs_from_config(cfg)
    dev = torch.device("cuda")
    dummy = torch.zeros(8, dtype=torch.float64, device=dev).data_ptr()
    rc = native.cp_push_ions_noalloc(gap, see, cfg["dt"], 0, 0, 1, dummy, dummy, dummy, dummy,
                                     (1 << 19) + 1, dummy, dummy, dummy, 8, dummy, None)
    assert rc == native.ERR_CAPACITY
    big = native.cp_gap(**{k: getattr(gap, k) for k, _ in native.cp_gap._fields_})
    big.n_cells = 8192
    rc = native.cp_push_ions_noalloc(big, see, cfg["dt"], 0, 0, 1, dummy, dummy, dummy, dummy, 0,
                                     dummy, dummy, dummy, 8, dummy, None)
    assert rc == native.ERR_ARG
    # SEE laws that cp_create refuses are refused before any GPU work
    for field, bad in (("gamma_max", 15.0), ("gamma_max", float("nan")), ("scale", -1.0),
                       ("scale", float("inf")), ("T_emit_eV", -2.0), ("T_emit_eV", float("nan")),
                       ("gamma_coef", float("nan"))):
        s2 = native.cp_see_beam(**{k: getattr(see, k) for k, _ in native.cp_see_beam._fields_})
        setattr(s2, field, bad)
        rc = native.cp_push_ions_noalloc(gap, s2, cfg["dt"], 0, 0, 1, dummy, dummy, dummy, dummy,
                                         4, dummy, dummy, dummy, 8, dummy, None)
        assert rc == native.ERR_ARG, (field, bad)


def test_noalloc_reports_only_the_electrons_it_wrote(env):
    """With too small an output array the call fails with CP_ERR_CAPACITY and
    counts[4] gives the electrons actually written (se_cap), not the number
    the impacts asked for (counts[2] + counts[3])."""
    torch, native = env
    cfg = W.scaled(W.gap_1d_fp64(seed=5), beam_per_step=0, see_scale=20.0, precision=W.FP32)
    xi, u, ids = ion_set(cfg, 17, 2000)
    ref = context_step(native, cfg, xi, u, ids)
    dev = torch.device("cuda")
    N = cfg["n_cells"]
    gap, _, see, _ = native.structs_from_config(cfg)
    x_t = torch.tensor(xi, dtype=torch.float32, device=dev)
    u_t = torch.tensor(u, dtype=torch.float32, device=dev)
    id_t = torch.tensor(ids.view(np.int32), dtype=torch.int32, device=dev)
    E_t = torch.tensor(ref["E0"], dtype=torch.float64, device=dev)
    G_t = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    cap = 64
    sx = torch.zeros(cap, dtype=torch.float32, device=dev)
    su = torch.zeros(cap, dtype=torch.float32, device=dev)
    counts = torch.zeros(6, dtype=torch.int64, device=dev)
    rc = native.cp_push_ions_noalloc(gap, see, cfg["dt"], cfg["seed"], 0, 1, E_t.data_ptr(),
                                     x_t.data_ptr(), u_t.data_ptr(), id_t.data_ptr(), xi.size,
                                     G_t.data_ptr(), sx.data_ptr(), su.data_ptr(), cap,
                                     counts.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == native.ERR_CAPACITY
    c = counts.cpu().numpy()
    assert c[2] + c[3] > cap
    assert c[4] == cap
    assert c[2] == ref["h"]["emitted"][0, 0] and c[3] == ref["h"]["emitted"][0, 1]
