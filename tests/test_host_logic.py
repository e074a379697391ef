"""Host-side logic that needs no GPU: the workload families the benchmark
and the predictor study draw from, the predictor driver's error summary,
and the benchmark's clock sampling, peak and host-name helpers.  (The
kernels are covered by the -m gpu tests.)"""
import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W


def test_thinned_gap_keeps_the_charge_of_the_full_gap():
    """factor x fewer macroparticles of factor x the weight: the same plasma
    density and beam current as the large gap, for every seed."""
    for seed in range(4):
        full = W.gap_1d_fp32_large(seed)
        for f in (25, 100):
            t = W.gap_1d_fp32_thinned(seed, factor=f)
            assert t["n_pairs"] * t["weight"] == pytest.approx(full["n_pairs"] * full["weight"], rel=1e-12)
            assert t["beam_per_step"] * f == full["beam_per_step"]
            assert t["beam_mode"] == full["beam_mode"]  # same seed-drawn physics
            for k in ("n_cells", "d", "dt", "C", "V0", "area"):
                assert t[k] == full[k], k


def test_ensemble_instances_are_seeded_and_uneven():
    a = W.ensemble(64, seed=3, steps=10, thin=100)
    b = W.ensemble(64, seed=3, steps=10, thin=100)
    assert [x["n_cells"] for x in a] == [x["n_cells"] for x in b]
    assert len({x["n_cells"] for x in a}) > 10  # uneven grids
    assert all(256 <= x["n_cells"] <= 4096 for x in a)
    assert all(x["see_scale"] == 0.0 for i, x in enumerate(a) if i % 8 == 7)
    # each instance is a capacitor C = eps0 A / d when particle-free
    for x in a:
        assert x["C"] == pytest.approx(x["eps0"] * x["area"] / x["d"], rel=1e-12)


def test_ensemble_vgap_errors_summary():
    """Per run: max_t |V - V_strict| / max_t |V_strict| of each weak scheme."""
    from paper_2603_24010_gb300 import native, predictor as PR
    t = np.linspace(0.0, 1.0, 50)
    Vs = np.stack([np.sin(3 * t) * (k + 1) for k in range(3)])
    res = {native.STRICT: {"V_gap": Vs},
           native.WEAK: {"V_gap": Vs + 0.01},
           native.WEAK_LEARNED: {"V_gap": Vs * (1 + 1e-4)}}
    err = PR.ensemble_vgap_errors(res)
    scale = np.abs(Vs).max(axis=1)
    np.testing.assert_allclose(err[native.WEAK], 0.01 / scale)
    np.testing.assert_allclose(err[native.WEAK_LEARNED], 1e-4, rtol=1e-9)


def test_bench_predictor_study_glue(monkeypatch):
    """bench.py's predictor study assembles its JSON from the results of
    predictor.py's calls: run here with stand-ins for the GPU calls (shapes
    only)."""
    import json
    import types
    torch = pytest.importorskip("torch")
    import bench
    from paper_2603_24010_gb300 import native, predictor as PR
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a, **k: None)

    def ens_samples(cfgs, steps=None, capacity=(0, 0, 0)):
        n = steps - native.PRED_WINDOW
        return torch.zeros(len(cfgs) * n, native.MLP_IN), torch.zeros(len(cfgs) * n, native.MLP_OUT)

    def samples(cfg, steps=None):
        n = (steps or cfg["steps"]) - native.PRED_WINDOW
        return torch.zeros(n, native.MLP_IN), torch.zeros(n, native.MLP_OUT)

    def train(X, Y, iters=1, batch=1, seed=0, **k):
        return np.zeros(native.MLP_NPARAM, np.float32), native.cp_predictor(), [1.0, 0.1]

    def runs(V, dv):
        return {native.STRICT: dict(V_gap=V, J_hat=0 * V, ms_per_step=1.0),
                native.WEAK: dict(V_gap=V + dv, J_hat=0 * V, ms_per_step=1.0),
                native.WEAK_LEARNED: dict(V_gap=V + dv / 100, J_hat=0 * V + 1, ms_per_step=1.0)}

    def ens_eval(cfgs, params, norm, steps=None, capacity=(0, 0, 0), modes=None):
        return runs(np.ones((len(cfgs), steps + 1)), 0.01)

    def evaluate(cfg, params, norm, steps=None, modes=None):
        return runs(np.ones((steps or cfg["steps"]) + 1), 0.01)

    monkeypatch.setattr(PR, "ensemble_strict_samples", ens_samples)
    monkeypatch.setattr(PR, "strict_samples", samples)
    monkeypatch.setattr(PR, "train", train)
    monkeypatch.setattr(PR, "ensemble_evaluate", ens_eval)
    monkeypatch.setattr(PR, "evaluate", evaluate)
    args = types.SimpleNamespace(coupling_steps=100, coupling_factor=100, coupling_train=3,
                                 coupling_train_full=2, coupling_eval=4, coupling_eval_full=2,
                                 coupling_iters=5)
    out = json.loads(json.dumps(bench.run_coupling(args)))
    assert out["samples"] == 5 * (100 - native.PRED_WINDOW)
    assert out["vgap_err_weak"] == pytest.approx(0.01)
    assert out["vgap_err_learned"] == pytest.approx(1e-4)
    assert out["learned_better_frac"] == 1.0
    assert [r["seed"] for r in out["full_size"]] == [bench.EVAL_FULL_SEED0, bench.EVAL_FULL_SEED0 + 1]


def test_predictor_study_holds_out_its_evaluation_seeds(monkeypatch):
    """No held-out seed of the predictor study (thinned or full size) is a
    training seed, at the default sizes and at the largest the ranges allow;
    overlapping ranges are refused."""
    import types
    import bench
    for n_train, n_eval in ((2048, 256), (400_000, 900_000)):
        args = types.SimpleNamespace(coupling_train=n_train, coupling_train_full=16,
                                     coupling_eval=n_eval, coupling_eval_full=16)
        s = bench.coupling_seeds(args)
        assert len(s["train"]) == n_train and len(s["eval"]) == n_eval
        train = set(s["train"]) | set(s["train_full"])
        assert not train & (set(s["eval"]) | set(s["eval_full"]))
    monkeypatch.setattr(bench, "EVAL_SEED0", bench.TRAIN_SEED0 + 10)
    with pytest.raises(ValueError):
        bench.coupling_seeds(types.SimpleNamespace(coupling_train=64, coupling_train_full=1,
                                                   coupling_eval=4, coupling_eval_full=1))


# ---------------------------------------------------------------- bench.py helpers
class _FakeProc:
    """Stands in for the nvidia-smi process of ClockSampler."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler_with_rows(tmp_path, text):
    import bench
    cs = bench.ClockSampler(0)
    f = open(tmp_path / "clocks.csv", "w+")
    f.write(text)
    cs.file, cs.proc = f, _FakeProc()
    return cs


def test_clock_sampler_summarises_rows(tmp_path):
    """Median SM clock, the highest maximum, and the throttle reasons seen
    Active in any row; rows that do not parse are skipped."""
    rows = ("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "0, 1980, 2070, 1401.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "garbage line\n"
            "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    out = _sampler_with_rows(tmp_path, rows).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_why_it_has_no_rows(tmp_path):
    out = _sampler_with_rows(tmp_path, "").stop()
    assert out["samples"] == 0 and "no rows" in out["why"]


def test_measured_peak_or_fallback(tmp_path, monkeypatch):
    """The HBM peak comes from MEASURED_PEAKS.json at the repository root
    when it exists, else the stated 6800 GB/s fallback."""
    import json
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6778.3, "bf16_tflops": 1900.0}))
    assert bench.measured_peaks() == (6778.3, "measured")


def test_cpu_model_names_the_host():
    import bench
    name = bench.cpu_model()
    assert isinstance(name, str) and name


def test_push_traffic_only_from_a_capture_of_the_current_sources(tmp_path, monkeypatch):
    """The bench reports the push's DRAM traffic from the committed ncu
    summary only while the kernel sources hash to the value recorded there;
    otherwise traffic is null and the line says why."""
    import bench
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [str(src)])
    prof = tmp_path / "push.md"
    monkeypatch.setattr(bench, "PUSH_PROFILE", str(prof))
    assert bench.profiled_push_traffic()[0] is None  # no summary
    h = bench.kernel_source_hash()
    prof.write_text("dram_bytes_per_particle_step: 13.99\nsource_sha256: `%s`\n" % h)
    assert bench.profiled_push_traffic() == (13.99, None)
    src.write_text("__global__ void k() { /* changed */ }\n")
    v, why = bench.profiled_push_traffic()
    assert v is None and "changed" in why and h in why
