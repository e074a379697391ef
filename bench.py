"""Throughput of the circuit-coupled PIC step on one GB300 (or N replicas).

A step is one pass of the whole hot path (gather, push, absorption + SEE,
beam injection, deposit, coupled Poisson/circuit solve) over the large FP32
1D gap workload: 4096 cells, 1e7 macroparticles at start (5e6 e-/H+ pairs
drawn on the device), 5000 beam ions per step, dt = 0.5 ps, strict coupling.
The gap is advanced outside the timed region to a steady-state level
(--start-level, default 12000: the beam fills the gap, about 3e7 live
particles, ion impacts and SEE at the cathode every step), then W warm-up and
K timed steps follow.  The metric is particle-steps/s = sum over timed steps
of the live macroparticles pushed in that step / timed seconds.  Prints one
JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--start-level L]
                    [--impl native|reference]

After the timed run (outside it), the learned weak-coupling predictor is
trained on 2048 strict runs of the same gap distribution (generated as one
ensemble) and the V_gap(t) error of plain and learned weak coupling against
strict is reported on 256 held-out seeds ("coupling"; skip with
--no-coupling).

``--impl reference`` times the FP64 CPU oracle (the plain implementation
written from the paper) on the host cores on a bounded sample of the same
workload.
"""
import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2603_24010_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = {W.FP32: 16, W.FP64: 32}  # read + write of (xi, u)


def workload(name, seed, pairs=None):
    if name == "gap_1d_fp32_large":
        cfg = W.gap_1d_fp32_large(seed)
    elif name == "gap_1d_fp64":
        cfg = W.gap_1d_fp64(seed)
    else:
        raise SystemExit("unknown workload " + name)
    if pairs:  # same density and physics with a different number of macroparticles
        cfg["weight"] = cfg["weight"] * cfg["n_pairs"] / pairs
        cfg["n_pairs"] = int(pairs)
    return cfg


PUSH_PROFILE = os.path.join(ROOT, "profiles", "k_push_async_gap_1d_fp32_large.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2603_24010_gb300", "csrc", f)
                  for f in ("cp_push_async.cu", "cp_push.cu", "cp_common.cuh", "cp_device.cuh")]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_push_traffic():
    """(DRAM bytes per particle-step of the push kernel from the committed
    ncu summary, None) -- or (None, why) when there is no summary or the
    kernel sources changed since it was taken."""
    try:
        text = open(PUSH_PROFILE).read()
    except OSError:
        return None, "no committed ncu summary of the push"
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith(("dram_bytes_per_particle_step", "source_sha256")):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    now = kernel_source_hash()
    if vals.get("source_sha256") != now:
        return None, ("the push's sources changed since the committed ncu capture (source hash %s, "
                      "capture %s); traffic not re-measured" % (now, vals.get("source_sha256")))
    try:
        return float(vals["dram_bytes_per_particle_step"]), None
    except (KeyError, ValueError):
        return None, "the ncu summary gives no DRAM bytes per particle-step"



def workload_desc(cfg, K, W_, L0):
    where = ("advanced to level %d outside the timed region (steady state: the beam across the "
             "gap, ion impacts and SEE at the cathode), then %d warm-up + %d timed steps"
             % (L0, W_, K)) if L0 else ("%d warm-up + %d timed steps from t = 0" % (W_, K))
    return ("%s: %d cells, %d e-/H+ pairs loaded on the device (1 eV Maxwellian), %d beam "
            "ions/step (%s), dt %.3g s, %s particles, strict coupling; %s"
            % (cfg["name"], cfg["n_cells"], cfg["n_pairs"], cfg["beam_per_step"],
               "mono 20 keV" if cfg["beam_mode"] == 0 else "uniform 5-50 keV", cfg["dt"],
               "FP32" if cfg["precision"] == W.FP32 else "FP64", where))


def cpu_model():
    """The host CPU's model name (x86 'model name', else Arm implementer/part)."""
    info = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in info:
        return info["model name"]
    if "CPU implementer" in info:
        return "Arm implementer %s part %s" % (info["CPU implementer"], info.get("CPU part", "?"))
    import platform
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.file = None
        self.why = None
        try:  # the physical GPU by UUID (a logical index can differ under CUDA_VISIBLE_DEVICES)
            import torch
            uuid = getattr(torch.cuda.get_device_properties(gpu_index), "uuid", None)
            if uuid:
                u = str(uuid)
                self.gpu = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception as e:
            self.proc = None
            self.why = "nvidia-smi did not start: %s" % e

    def stop(self):
        if not self.proc:
            return {"samples": 0, "why": self.why} if self.why else None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.split(",") for l in self.file.read().strip().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"samples": 0, "gpu": self.gpu,
                    "why": "nvidia-smi returned no rows for this GPU during the region"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm), "gpu": self.gpu}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- native arm
def load_particles(cfg, seed):
    xi, ue, ui = W.load_pairs(cfg, seed=seed)
    N = cfg["n_cells"]
    xe, ue = W.as_precision(xi, ue, N, cfg["precision"])
    xI, ui = W.as_precision(xi, ui, N, cfg["precision"])
    return xe, ue, xI, ui


def reduce_over_ranks(ms, e2e_ms, psteps, e2e_psteps, device):
    """Whole-job figures of independent replicas: the slowest rank's times
    and the sum of the particle-steps of all ranks."""
    import torch
    t = torch.tensor([ms, e2e_ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    c = torch.tensor([psteps, e2e_psteps], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(c, op=torch.distributed.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(c[0]), int(c[1])


def run_native(args, rank, world):
    """The large gap through the C ABI: the initial plasma drawn on the device
    (cp_load_species), advanced outside the timed region to the start level,
    then W warm-up and K timed steps (CUDA-graph replays); K more steps with
    per-launch CUDA events give each kernel's device time; the t = 0 window
    and the end-to-end job are measured beside them."""
    import torch
    from paper_2603_24010_gb300 import native

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = workload(args.workload, seed=args.seed + rank, pairs=args.pairs)
    K, Wm, L0 = args.steps, args.warmup, args.start_level
    stream = torch.cuda.current_stream()
    bpp = BYTES_PER_PARTICLE_STEP[cfg["precision"]]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def make(max_steps):
        g = native.Gap(cfg, max_steps=max_steps, stream=stream.cuda_stream)
        g.load_species(cfg["n_pairs"], cfg["T_load_eV"], cfg["seed"])
        return g

    # ---- device-resident timed region (graph replays, the user's path) ------
    g = make(L0 + Wm + 2 * K + 1)
    clocks = ClockSampler(dev)
    clocks.start()  # sampled over the advance (seconds of load) and the timed steps
    g.step(0, L0 + Wm)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_window:  # a profiler started with profiling off captures the timed steps only
        torch.cuda.profiler.start()
    e0.record(stream)
    g.step(0, K)
    e1.record(stream)
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = native.cp_last_launch_count(g.ctx)
    hist = g.history(L0 + Wm, K)  # rows of the timed levels: particles pushed by the timed steps
    live = hist["n_live"].sum(axis=1)
    psteps = int(live.sum())
    impacts = int(hist["absorbed"][:, 0, 1].sum())
    emitted = int(hist["emitted"].sum())
    if args.single:  # one graph pass only (used under ncu)
        clk = clocks.stop()
        g.close()
        return dict(cfg=cfg, ms=ms, psteps=psteps, launches=launches, clocks=clk)

    # ---- K more steps of the same gap with per-launch CUDA events -----------
    native.cp_enable_timing(g.ctx, True)
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    g.step(0, K)
    t1e.record(stream)
    torch.cuda.synchronize()
    ms_timed = t0e.elapsed_time(t1e)
    kms, kn = native.cp_read_timing(g.ctx)
    per_launch_ms = np.asarray(native.cp_read_launch_times(g.ctx))
    native.cp_enable_timing(g.ctx, False)
    live_t = g.history(L0 + Wm + K, K)["n_live"].sum(axis=1)
    clk = clocks.stop()
    g.close()

    # ---- the first K steps from t = 0 (a second figure) ---------------------
    g0 = make(Wm + K + 1)
    g0.step(0, Wm)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    g0.step(0, K)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_t0 = a0.elapsed_time(a1)
    psteps_t0 = int(g0.history(Wm, K)["n_live"].sum())
    g0.close()

    # ---- end to end through the C ABI: the whole job a user runs ------------
    # cp_create + cp_load_species (parameters from host structs), every step up
    # to the end of the timed window, and the read-back of every level's
    # diagnostics row into host memory
    n_all = L0 + Wm + K
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    g2 = make(n_all + 1)
    g2.step(0, n_all)
    h2 = native.cp_read_history(g2.ctx, 0, n_all + 1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_psteps = int(sum(sum(h2[k].n_live) for k in range(n_all)))
    g2.close()
    h2d = sum(ctypes.sizeof(c) for c in (native.cp_gap, native.cp_circuit, native.cp_see_beam,
                                          native.cp_run, native.cp_species))
    d2h = (n_all + 1) * ctypes.sizeof(native.cp_diag)

    if world > 1:
        ms, e2e_ms, psteps, e2e_psteps = reduce_over_ranks(ms, e2e_s * 1e3, psteps, e2e_psteps, "cuda")
    else:
        e2e_ms = e2e_s * 1e3
    peak, peak_kind = measured_peaks()
    # Roofline of the push: algorithmic bytes per launch / launch time, over the
    # launches whose particle state (xi, u) exceeds 1.5 x the 129 MB L2
    state = live_t * bpp / 2
    sel = state > 1.5 * 129e6
    all_above = bool(sel.all())
    if not sel.any():
        sel = np.ones_like(sel)
    n_sel = int(sel.sum())
    sel_ms = float(per_launch_ms[:len(sel)][sel[:len(per_launch_ms)]].sum())
    avg_launch_ms = sel_ms / n_sel
    achieved = bpp * float(live_t[sel].sum()) / (sel_ms * 1e-3) / 1e9
    dbpp, traffic_why = (profiled_push_traffic() if cfg["precision"] == W.FP32
                         else (None, "no ncu summary of the FP64 push"))
    traffic = dbpp * float(live_t[sel].sum()) / n_sel if dbpp else None
    smin, smax = float((live * bpp / 2).min()) / 1e6, float((live * bpp / 2).max()) / 1e6
    l2 = ("particle state (x, u) %.0f-%.0f MB over the timed steps, %s the 129 MB L2; no flush"
          % (smin, smax, "above" if smin > 129 else ("partly above" if smax > 129 else "within")))
    if not all_above:
        l2 += ("; roofline over %s launches (state above 1.5 x L2 in %d of %d)"
               % ("all" if n_sel == len(state) else "those", int((state > 1.5 * 129e6).sum()),
                  len(state)))
    return dict(cfg=cfg, ms=ms, ms_timed=ms_timed, psteps=psteps, e2e_ms=e2e_ms,
                e2e_psteps=e2e_psteps, h2d=h2d, d2h=d2h, launches=launches,
                kernel_ms=kms.tolist(), kernel_n=kn.tolist(), avg_launch_ms=avg_launch_ms,
                achieved=achieved, peak=peak, peak_kind=peak_kind, clocks=clk, bpp=bpp,
                n_sel=n_sel, traffic=traffic, traffic_why=traffic_why, l2=l2, impacts=impacts,
                emitted=emitted,
                live_mean=float(live.mean()), ms_t0=ms_t0, psteps_t0=psteps_t0, n_all=n_all)


# ---------------------------------------------------------------- ensemble
def run_ensemble(args, K, Wm):
    """The ensemble workload: 512 independent gaps of uneven size advanced by
    one persistent push and one solve launch per step (CUDA graph).  Strict
    coupling is timed (the line's value); weak coupling is run on the same
    instances and reported beside it."""
    import torch
    from paper_2603_24010_gb300 import native
    n_inst = args.ensemble_instances
    total = Wm + K + 1 + 5 * args.tune_steps + args.ensemble_timed_steps
    cfgs = W.ensemble(n_inst, seed=args.seed, steps=total)
    stream = torch.cuda.current_stream()
    loads = []
    for cfg in cfgs:
        xi, ue, ui = W.load_pairs(cfg)
        xe, ue = W.as_precision(xi, ue, cfg["n_cells"], W.FP32)
        xo, ui = W.as_precision(xi, ui, cfg["n_cells"], W.FP32)
        loads.append((xe, ue, xo, ui))
    out = {}
    for mode, name in ((native.STRICT, "strict"), (native.WEAK, "weak")):
        b = native.Batch(cfgs, max_steps=total, stream=stream.cuda_stream)
        for i, (xe, ue, xo, ui) in enumerate(loads):
            b.set_particles(i, native.ELECTRONS, xe, ue)
            b.set_particles(i, native.IONS, xo, ui, np.arange(xo.size, dtype=np.uint32))
        rc = b.step(mode, Wm)
        tune = b.autotune(args.tune_steps, mode)
        lv0 = b.level
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clocks.start()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc2 = b.step(mode, K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
        launches = b.last_launch_count()
        psteps = 0
        for i in range(n_inst):
            h = b.history(i, lv0, K)
            psteps += int(h["n_live"].sum())
        entry = dict(ms=ms, psteps=psteps, launches=launches, rc=[rc, tune[0], rc2],
                     shape={"threads": tune[1], "ctas_per_sm": tune[2], "push_ms": tune[3]},
                     clocks=clk)
        if mode == native.STRICT:  # a short per-kernel timed pass for the roofline
            b.enable_timing(True)
            lv1 = b.level
            Kt = min(args.ensemble_timed_steps, total - lv1)
            b.step(mode, Kt)
            kms, kn = b.timing()
            b.enable_timing(False)
            live_t = sum(int(b.history(i, lv1, Kt)["n_live"].sum()) for i in range(n_inst))
            entry.update(kernel_ms=kms.tolist(), kernel_n=kn.tolist(), timed_psteps=live_t)
        b.close()
        out[name] = entry
    tot_init = sum(2 * c["n_pairs"] for c in cfgs)
    cells = [c["n_cells"] for c in cfgs]
    out["desc"] = ("ensemble: %d gaps, cells %d-%d (log-uniform 256-4096), %.3g initial "
                   "macroparticles (log-uniform 1e4-2e6 each), V0 50-200 kV, C 20-500 pF, SEE "
                   "scale 0-2 (every 8th 0), mono beam 5-50 keV at max(50, N/2000) ions/step, "
                   "dt 1 ps, FP32; %d warm-up + %d tuner + %d timed steps"
                   % (n_inst, min(cells), max(cells), tot_init, Wm, 5 * args.tune_steps, K))
    return out


def ensemble_main(args, config, emit=True):
    import torch  # noqa: F401
    from paper_2603_24010_gb300 import native  # noqa: F401
    K = args.steps if args.steps is not None else 10000
    Wm = args.warmup
    r = run_ensemble(args, K, Wm)
    st = r["strict"]
    value = st["psteps"] / (st["ms"] * 1e-3)
    peak, peak_kind = measured_peaks()
    kms, kn = st["kernel_ms"], st["kernel_n"]
    achieved = 16.0 * st["timed_psteps"] / (kms[0] * 1e-3) / 1e9
    config = dict(config)
    config["workload"] = r["desc"]
    config["l2"] = "inputs larger than L2 (about 3 GB of particle state), no flush"
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": 1, "steps": K,
        "warmup": Wm, "ms_per_step": st["ms"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "gpu_launches": st["launches"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_push_ens",
                     "peak_source": peak_kind, "bytes_per_particle_step": 16,
                     "push_avg_ms": kms[0] / max(kn[0], 1), "solve_avg_ms": kms[1] / max(kn[1], 1),
                     "removal_avg_ms": kms[2] / max(kn[2], 1),
                     "source": "per-launch CUDA events over %d steps after the timed region"
                               % kn[0], "timed_steps": int(kn[0])},
        "clocks": st["clocks"],
        "autotuned_shape": st["shape"],
        "weak": {"value": r["weak"]["psteps"] / (r["weak"]["ms"] * 1e-3),
                 "ms_per_step": r["weak"]["ms"] / K, "shape": r["weak"]["shape"]},
        "status": {"strict": st["rc"], "weak": r["weak"]["rc"]},
        "particle_steps": st["psteps"],
    }
    if emit:
        print(json.dumps(line))
    return line


# ---------------------------------------------------------------- 2D gap
def gap2d_main(args, config, emit=True):
    """The 2D planar gap: 1024 x 1024 cells (y periodic), 1e8 macroparticles,
    Gaussian beam; strict coupling; one CUDA-event pass times the steps and a
    second, shorter pass times each kernel group for the roofline."""
    import torch
    from paper_2603_24010_gb300 import native
    K = args.steps if args.steps is not None else 2000
    Wm = args.warmup
    Kt = args.gap2d_timed_steps
    cfg = W.gap_2d(args.seed, n_pairs=args.pairs or 50_000_000)
    xi, eta, ue, we, ui, wi = W.load_pairs_2d(cfg)
    stream = torch.cuda.current_stream()
    g = native.Gap2D(cfg, max_steps=Wm + K + Kt + 1, stream=stream.cuda_stream)
    g.set_particles(native.ELECTRONS, xi, eta, ue, we)
    g.set_particles(native.IONS, xi, eta, ui, wi, np.arange(xi.size, dtype=np.uint32))
    del xi, eta, ue, we, ui, wi
    g.step(native.STRICT, Wm)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(native.STRICT, K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = g.last_launch_count()
    h = g.history(Wm, K)
    psteps = int(h["n_live"].sum())
    g.enable_timing(True)
    lv = g.level
    g.step(native.STRICT, Kt)
    kms, kn = g.timing()
    ht = g.history(lv, Kt)
    live_t = float(ht["n_live"].sum())
    g.close()
    peak, peak_kind = measured_peaks()
    achieved = 32.0 * live_t / (kms[0] * 1e-3) / 1e9
    config = dict(config)
    config["workload"] = ("gap_2d: %d x %d cells (y periodic), %d e-/H+ pairs loaded, %d beam "
                          "ions/step (20 keV, Gaussian sigma 0.5 mm), dt %.3g s, FP32 particles, "
                          "strict coupling; %d warm-up + %d timed steps"
                          % (cfg["n_cells"], cfg["Ny"], cfg["n_pairs"], cfg["beam_per_step"],
                             cfg["dt"], Wm, K))
    config["l2"] = "inputs larger than L2 (1.6 GB of particle state at start), no flush"
    line = {
        "metric": METRIC, "value": psteps / (ms * 1e-3), "unit": "particle-steps/s", "n_gpus": 1,
        "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config, "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k2_push",
                     "peak_source": peak_kind, "bytes_per_particle_step": 32,
                     "push_avg_ms": kms[0] / max(kn[0], 1), "solve_avg_ms": kms[1] / max(kn[1], 1),
                     "sort_avg_ms": kms[2] / max(kn[2], 1), "timed_steps": int(kn[0]),
                     "source": "per-kernel-group CUDA events over %d steps after the timed region"
                               % kn[0]},
        "clocks": clk, "particle_steps": psteps,
    }
    if emit:
        print(json.dumps(line))
    return line


# ---------------------------------------------------------------- coupling
# Seed ranges of the predictor study.  Training and held-out seeds come from
# disjoint ranges (a held-out run must be a run the network never saw); the
# thinned and full-size runs of one seed share the seed-drawn physics (beam
# mode) but not their particle draws.
TRAIN_SEED0, TRAIN_FULL_SEED0 = 1000, 500_000
EVAL_SEED0, EVAL_FULL_SEED0 = 1_000_000, 2_000_000


def coupling_seeds(args):
    """Seeds of the thinned training runs, full-size training runs, thinned
    held-out runs and full-size held-out runs; raises if any held-out seed is
    also a training seed."""
    s = {"train": [TRAIN_SEED0 + k for k in range(args.coupling_train)],
         "train_full": [TRAIN_FULL_SEED0 + k for k in range(args.coupling_train_full)],
         "eval": [EVAL_SEED0 + k for k in range(args.coupling_eval)],
         "eval_full": [EVAL_FULL_SEED0 + k for k in range(args.coupling_eval_full)]}
    train = set(s["train"]) | set(s["train_full"])
    held = set(s["eval"]) | set(s["eval_full"])
    if train & held:
        raise ValueError("predictor study: held-out seeds overlap the training seeds")
    return s


def run_coupling(args):
    """The learned weak-coupling predictor on the large gap's distribution:
    an ensemble of thinned strict runs plus a few full-size strict runs
    generate the training set, the network is trained, and on held-out seeds
    (thinned: one ensemble per scheme; full-size: one run per scheme) the
    V_gap(t) error of plain and learned weak coupling against strict and the
    wall time of the three schemes are compared."""
    import torch
    from paper_2603_24010_gb300 import native
    from paper_2603_24010_gb300 import predictor as PR
    S, f = args.coupling_steps, args.coupling_factor
    fam = lambda seed: W.gap_1d_fp32_thinned(seed, factor=f, steps=S)  # noqa: E731
    big = lambda seed: dict(W.gap_1d_fp32_large(seed), steps=S)  # noqa: E731
    seeds = coupling_seeds(args)
    t0 = time.perf_counter()
    X, Y = PR.ensemble_strict_samples([fam(s) for s in seeds["train"]], S)
    Xf, Yf = [X], [Y]
    for s in seeds["train_full"]:
        xk, yk = PR.strict_samples(big(s), S)
        Xf.append(xk)
        Yf.append(yk)
    X, Y = torch.cat(Xf), torch.cat(Yf)
    del Xf, Yf
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, norm, losses = PR.train(X, Y, iters=args.coupling_iters, batch=8192, seed=1)
    t_train = time.perf_counter() - t0
    n_samples = int(X.shape[0])
    del X, Y
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    res = PR.ensemble_evaluate([fam(s) for s in seeds["eval"]], params, norm, S)
    errs = PR.ensemble_vgap_errors(res)
    used = (res[native.WEAK_LEARNED]["J_hat"] != 0).mean(axis=1)
    full = []
    for s in seeds["eval_full"]:
        rk = PR.evaluate(big(s), params, norm, S)
        ek = PR.vgap_errors(rk)
        full.append({"seed": s, "vgap_err_weak": ek[native.WEAK],
                     "vgap_err_learned": ek[native.WEAK_LEARNED],
                     "predictor_used_frac": float((rk[native.WEAK_LEARNED]["J_hat"] != 0).mean()),
                     "ms_per_step": {"strict": rk[native.STRICT]["ms_per_step"],
                                     "weak": rk[native.WEAK]["ms_per_step"],
                                     "weak_learned": rk[native.WEAK_LEARNED]["ms_per_step"]}})
    t_eval = time.perf_counter() - t0
    cfg = fam(seeds["eval"][0] if seeds["eval"] else 0)
    return {
        "workload": ("gap_1d_fp32_thinned: the large gap's distribution (4096 cells, seed-drawn "
                     "beam mode) with %d x fewer, heavier macroparticles: %d pairs, %d beam "
                     "ions/step, dt %.3g s, %d steps; plus full-size runs of the large gap"
                     % (f, cfg["n_pairs"], cfg["beam_per_step"], cfg["dt"], S)),
        "seeds": {k: ([v[0], v[-1]] if v else []) for k, v in seeds.items()},
        "train_runs": args.coupling_train, "train_runs_full_size": args.coupling_train_full,
        "eval_runs": args.coupling_eval, "eval_runs_full_size": args.coupling_eval_full,
        "data": "thinned training runs generated as one strict ensemble, full-size ones one by "
                "one; thinned held-out seeds evaluated as one ensemble per scheme",
        "samples": n_samples, "train_iters": args.coupling_iters,
        "loss_first_last": [losses[0], losses[-1]],
        "metric": "max_t |V_gap - V_gap(strict)| / max_t |V_gap(strict)|, mean over eval seeds",
        "vgap_err_weak": float(np.mean(errs[native.WEAK])),
        "vgap_err_learned": float(np.mean(errs[native.WEAK_LEARNED])),
        "vgap_err_weak_max": float(np.max(errs[native.WEAK])),
        "vgap_err_learned_max": float(np.max(errs[native.WEAK_LEARNED])),
        "learned_better_frac": float(np.mean(errs[native.WEAK_LEARNED] < errs[native.WEAK])),
        "predictor_used_frac": float(np.mean(used)),
        "ms_per_step_ensemble": {"strict": res[native.STRICT]["ms_per_step"],
                                 "weak": res[native.WEAK]["ms_per_step"],
                                 "weak_learned": res[native.WEAK_LEARNED]["ms_per_step"]},
        "full_size": full,
        "seconds": {"data": t_data, "train": t_train, "eval": t_eval},
    }


# ---------------------------------------------------------------- oracle arm
def oracle_sample(cfg, K, Wm, budget_s, rate_guess=4e7):
    """Run the FP64 oracle on a sub-sampled copy of the workload (fewer
    macroparticles and beam ions, same physics) for Wm + K steps, sized to
    about budget_s seconds; returns (particle-steps/s, description)."""
    from oracle import oracle as orc
    # average live particles of the full workload over its first steps
    beam_fill = min(Wm + K, int(cfg["d"] / (math.sqrt(2 * 20e3 * cfg["e"] / cfg["m_i"]) * cfg["dt"])))
    avg_live = 2 * cfg["n_pairs"] + cfg["beam_per_step"] * beam_fill / 2.0
    frac = min(1.0, budget_s * rate_guess / max(1.0, (Wm + K) * avg_live))
    n_pairs = max(64, int(cfg["n_pairs"] * frac))
    beam = max(1, int(round(cfg["beam_per_step"] * frac))) if cfg["beam_per_step"] else 0
    sub = W.scaled(cfg, n_pairs=n_pairs, beam_per_step=beam)
    sub["weight"] = cfg["weight"] * cfg["n_pairs"] / n_pairs
    xi, ue, ui = W.load_pairs(sub)
    r = orc.OracleGap(sub)
    r.set_particles(orc.ELECTRONS, xi, ue)
    r.set_particles(orc.IONS, xi, ui)
    if Wm:
        r.step(orc.STRICT, Wm)
    t0 = time.perf_counter()
    rc = r.step(orc.STRICT, K)
    dt = time.perf_counter() - t0
    h = r.history()
    psteps = int(h["n_live"][Wm:Wm + K].sum())
    r.close()
    oracle_sample.ms_per_step = 1e3 * dt / max(K, 1)
    desc = ("oracle (plain FP64 C, 1 thread) on the same workload sub-sampled to %d pairs and "
            "%d beam ions/step (fraction %.4g of the macroparticles, weights scaled), %d "
            "warm-up + %d timed steps, %.1f s, status %d" % (n_pairs, beam, frac, Wm, K, dt, rc))
    return psteps / dt, desc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 2000; 10000 for the ensemble)")
    ap.add_argument("--start-level", type=int, default=12000,
                    help="level the large gap is advanced to before the timed window "
                         "(outside the timed region; 0 times from t = 0)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--workload", default="gap_1d_fp32_large")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairs", type=int, default=None,
                    help="override the workload's loaded pairs (weight scaled to keep the density)")
    ap.add_argument("--single", action="store_true",
                    help="only the device-resident graph pass (for profiler captures)")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for a profiler "
                         "run with --profile-from-start off)")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the ensemble and 2D gap figures added to the main line")
    ap.add_argument("--no-coupling", action="store_true",
                    help="skip the learned-vs-plain weak coupling comparison")
    ap.add_argument("--coupling-train", type=int, default=2048)
    ap.add_argument("--coupling-eval", type=int, default=256)
    ap.add_argument("--coupling-train-full", type=int, default=16,
                    help="full-size strict training runs added to the thinned ones")
    ap.add_argument("--coupling-eval-full", type=int, default=16,
                    help="full-size held-out seeds evaluated one run per scheme")
    ap.add_argument("--coupling-steps", type=int, default=20000)
    ap.add_argument("--coupling-factor", type=int, default=100)
    ap.add_argument("--coupling-iters", type=int, default=6000)
    ap.add_argument("--ensemble-instances", type=int, default=512)
    ap.add_argument("--ensemble-timed-steps", type=int, default=200)
    ap.add_argument("--tune-steps", type=int, default=3)
    ap.add_argument("--gap2d-timed-steps", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload == "ensemble":
        ensemble_main(args, {"parallelism": "1 GPU"})
        return
    if args.workload == "gap_2d":
        gap2d_main(args, {"parallelism": "1 GPU"})
        return
    if args.steps is None:
        args.steps = 2000
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    cfg = workload(args.workload, args.seed, pairs=args.pairs)
    config = {"workload": workload_desc(cfg, args.steps, args.warmup, args.start_level),
              "parallelism": ("replicas x%d (independent seeds)" % world) if world > 1 else "1 GPU"}

    if args.impl == "reference":
        if rank != 0:
            return
        value, desc = oracle_sample(cfg, args.steps, args.warmup, budget_s=120.0)
        config["l2"] = "not applicable (host cores)"
        line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": getattr(oracle_sample, "ms_per_step", None),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config, "impl": "reference",
                "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1,
                                 "cpu_model": cpu_model(), "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_native(args, rank, world)
    if args.single:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": r["psteps"] / (r["ms"] * 1e-3),
                              "unit": "particle-steps/s", "steps": args.steps,
                              "config": config, "note": "single graph pass (profiling run)"}))
        return
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:  # the oracle is timed beside one GPU only
        v, desc = oracle_sample(cfg, 200, 3, budget_s=20.0)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": 1, "cpu_model": cpu_model(),
               "kind": "oracle", "sample": desc}
    # the predictor study is a single-GPU experiment: replica runs skip it
    coupling = None if (args.no_coupling or world > 1) else run_coupling(args)
    K = args.steps
    value = r["psteps"] / (r["ms"] * 1e-3)
    config["l2"] = r["l2"]
    clk = r["clocks"] or {}
    cycles = (r["avg_launch_ms"] * 1e-3 * clk["sm_mhz"] * 1e6) if clk.get("sm_mhz") else None
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": r["ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if r["cfg"]["precision"] == W.FP32 else "f64", "data": "synthetic",
        "config": config,
        "e2e": {"value": r["e2e_psteps"] / (r["e2e_ms"] * 1e-3), "unit": "particle-steps/s",
                "h2d_bytes_per_step": r["h2d"] / r["n_all"], "d2h_bytes_per_step": r["d2h"] / r["n_all"],
                "job": "cp_create + cp_load_species (initial plasma drawn on the device from host "
                       "parameter structs) + %d strict steps + read-back of every level's "
                       "diagnostics row into host memory; particle-steps of all %d steps"
                       % (r["n_all"], r["n_all"])},
        "gpu_launches": r["launches"],
        "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["peak"],
                     "unit": "GB/s", "frac": r["achieved"] / r["peak"], "traffic": r["traffic"],
                     "traffic_note": r["traffic_why"],
                     "kernel": "k_push_async" if r["cfg"]["precision"] == W.FP32 else "k_push",
                     "peak_source": r["peak_kind"],
                     "avg_launch_ms": r["avg_launch_ms"], "launches_used": r["n_sel"],
                     "bytes_per_particle_step": r["bpp"],
                     "solve_avg_ms": r["kernel_ms"][1] / max(r["kernel_n"][1], 1),
                     "removal_avg_ms": r["kernel_ms"][2] / max(r["kernel_n"][2], 1),
                     "timed_pass_ms_per_step": r["ms_timed"] / K,
                     "push_sm_cycles_per_launch": cycles,
                     "source": "per-launch CUDA events over the %d steps after the timed window "
                               "(same gap, direct launches)" % K},
        "clocks": r["clocks"],
        "cpu_baseline": cpu,
        "coupling": coupling,
        "particle_steps": r["psteps"],
        "window": {"start_level": args.start_level, "live_mean": r["live_mean"],
                   "ion_impacts_per_step": r["impacts"] / K, "secondaries_per_step": r["emitted"] / K},
        "t0_window": {"value": r["psteps_t0"] / (r["ms_t0"] * 1e-3), "ms_per_step": r["ms_t0"] / K,
                      "note": "the same K steps timed from t = 0 (1e7 particles, no impacts yet)"},
    }
    if world == 1 and not args.no_other_workloads:
        line["other_workloads"] = other_workloads(args)
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def other_workloads(args):
    """The ensemble and 2D gap benchmarks at their own default sizes, run
    after the main line's measurements (their figures ride on the same JSON
    line; `--workload ensemble` / `--workload gap_2d` print their full lines)."""
    out = {}
    for name, fn in (("ensemble", ensemble_main), ("gap_2d", gap2d_main)):
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.pairs = None, None
        ln = fn(sub, {"parallelism": "1 GPU"}, emit=False)
        rf = ln["roofline"]
        out[name] = {"value": ln["value"], "unit": ln["unit"], "steps": ln["steps"],
                     "ms_per_step": ln["ms_per_step"], "workload": ln["config"]["workload"],
                     "l2": ln["config"]["l2"], "gpu_launches": ln.get("gpu_launches"),
                     "roofline": {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                     "kernel", "peak_source",
                                                     "bytes_per_particle_step")},
                     "clocks": ln.get("clocks")}
    return out


if __name__ == "__main__":
    main()
