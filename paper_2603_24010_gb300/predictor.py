"""Training and evaluation driver of the learned weak-coupling predictor.

Orchestration only: every sample, forward and backward pass, optimiser step
and time step runs in the library's kernels through the C ABI
(``cp_predictor_samples``, ``cp_mlp_*``, ``cp_step_*``); PyTorch supplies the
device buffers and the stream.

Data: strict-coupling runs of a workload family, one Gap per seed
(``strict_samples``) or one ensemble of all seeds advanced together
(``ensemble_strict_samples``).  Each run of S steps gives S - 8 samples: the
8-level feature window ending at level L and the targets of level L+1.
"""
import time

import numpy as np

from . import native
from . import workloads as W


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the predictor needs a CUDA device")
    return torch


def load_gap(cfg, max_steps=None):
    """A Gap with the workload's pairs loaded (plasma electrons and ions)."""
    g = native.Gap(cfg, max_steps=max_steps or cfg["steps"])
    xi, ue, ui = W.load_pairs(cfg)
    prec = cfg.get("precision", W.FP64)
    xe, ue = W.as_precision(xi, ue, cfg["n_cells"], prec)
    xo, ui = W.as_precision(xi, ui, cfg["n_cells"], prec)
    g.set_particles(native.ELECTRONS, xe, ue)
    g.set_particles(native.IONS, xo, ui, np.arange(xi.size, dtype=np.uint32))
    return g


def strict_samples(cfg, steps=None):
    """Run one strict-coupling instance; return its samples (X, Y) on the device."""
    torch = _torch()
    steps = int(steps or cfg["steps"])
    g = load_gap(cfg, steps)
    g.step(native.STRICT, steps)
    n = steps - native.PRED_WINDOW  # windows ending at levels 8..steps-1
    X = torch.empty((n, native.MLP_IN), dtype=torch.float32, device="cuda")
    Y = torch.empty((n, native.MLP_OUT), dtype=torch.float32, device="cuda")
    native._check("cp_predictor_samples",
                  native.cp_predictor_samples(g.ctx, native.PRED_WINDOW, n, X.data_ptr(),
                                              Y.data_ptr()))
    torch.cuda.synchronize()
    g.close()
    return X, Y


def load_batch(cfgs, steps, capacity=(0, 0, 0)):
    """An ensemble of the workloads with their pairs loaded."""
    b = native.Batch(cfgs, max_steps=steps, capacity=capacity)
    for i, cfg in enumerate(cfgs):
        xi, ue, ui = W.load_pairs(cfg)
        prec = cfg.get("precision", W.FP64)
        xe, ue = W.as_precision(xi, ue, cfg["n_cells"], prec)
        xo, ui = W.as_precision(xi, ui, cfg["n_cells"], prec)
        b.set_particles(i, native.ELECTRONS, xe, ue)
        b.set_particles(i, native.IONS, xo, ui, np.arange(xi.size, dtype=np.uint32))
    return b


def _step_batch(b, mode, n):
    rc = b.step(mode, n)
    if rc != native.OK:
        raise native.CpError("cp_batch_step", rc)


def ensemble_strict_samples(cfgs, steps=None, capacity=(0, 0, 0)):
    """Advance all runs together as one strict-coupling ensemble; return the
    samples of every run, concatenated, on the device."""
    torch = _torch()
    steps = int(steps or cfgs[0]["steps"])
    b = load_batch(cfgs, steps, capacity)
    _step_batch(b, native.STRICT, steps)
    n = steps - native.PRED_WINDOW  # windows ending at levels 8..steps-1
    X = torch.empty((len(cfgs) * n, native.MLP_IN), dtype=torch.float32, device="cuda")
    Y = torch.empty((len(cfgs) * n, native.MLP_OUT), dtype=torch.float32, device="cuda")
    for i in range(len(cfgs)):
        b.predictor_samples(i, native.PRED_WINDOW, n, X[i * n:].data_ptr(), Y[i * n:].data_ptr())
    torch.cuda.synchronize()
    b.close()
    return X, Y


def ensemble_evaluate(cfgs, params, norm, steps=None, capacity=(0, 0, 0),
                      modes=(native.STRICT, native.WEAK, native.WEAK_LEARNED)):
    """Every run under each scheme, as one ensemble per scheme (the network
    installed on every instance of the learned scheme only, so that the
    other schemes run without it); V_gap(t) and J_hat histories (runs x
    levels) and the ensemble's wall time per step."""
    torch = _torch()
    steps = int(steps or cfgs[0]["steps"])
    out = {}
    for mode in modes:
        b = load_batch(cfgs, steps, capacity)
        if params is not None and mode == native.WEAK_LEARNED:
            for i in range(len(cfgs)):
                b.set_predictor(i, params, norm)
        _step_batch(b, mode, 1)  # level 0 solve and first push outside the timing
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _step_batch(b, mode, steps - 1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        hs = [b.history(i) for i in range(len(cfgs))]
        b.close()
        out[mode] = dict(V_gap=np.stack([h["V_gap"] for h in hs]),
                         J_hat=np.stack([h["J_hat"] for h in hs]),
                         ms_per_step=1e3 * wall / (steps - 1))
    return out


def ensemble_vgap_errors(res):
    """Per run: max_t |V_gap - V_gap(strict)| / max_t |V_gap(strict)| of the
    weak schemes."""
    Vs = res[native.STRICT]["V_gap"]
    scale = np.abs(Vs).max(axis=1)
    return {mode: np.abs(res[mode]["V_gap"] - Vs).max(axis=1) / scale
            for mode in (native.WEAK, native.WEAK_LEARNED) if mode in res}


def train(X, Y, iters=3000, batch=8192, lr=2e-3, lr_final=1e-4, seed=0, bound=0.5):
    """Adam on the MSE of the normalised targets; returns (params host array,
    cp_predictor, loss history).  Mini-batches are drawn on the device."""
    torch = _torch()
    st = torch.cuda.current_stream().cuda_stream
    n = X.shape[0]
    norm = native.cp_predictor()
    norm.bound = float(bound)
    native._check("cp_mlp_scales", native.cp_mlp_scales(X.data_ptr(), Y.data_ptr(), n, norm, st))
    Xn = torch.empty_like(X)
    Yn = torch.empty_like(Y)
    native._check("cp_mlp_normalize", native.cp_mlp_normalize(X.data_ptr(), Y.data_ptr(), n, norm,
                                                              Xn.data_ptr(), Yn.data_ptr(), st))
    P = native.MLP_NPARAM
    params = torch.empty(P, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(native.cp_mlp_work_floats(), dtype=torch.float32, device="cuda")
    native._check("cp_mlp_init", native.cp_mlp_init(params.data_ptr(), seed, st))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(int(seed) + 1)
    b = min(int(batch), n)
    Xb = torch.empty((b, native.MLP_IN), dtype=torch.float32, device="cuda")
    Yb = torch.empty((b, native.MLP_OUT), dtype=torch.float32, device="cuda")
    losses = []
    for it in range(1, int(iters) + 1):
        idx = torch.randint(0, n, (b,), device="cuda", generator=gen)
        torch.index_select(Xn, 0, idx, out=Xb)
        torch.index_select(Yn, 0, idx, out=Yb)
        native._check("cp_mlp_loss_grad",
                      native.cp_mlp_loss_grad(params.data_ptr(), Xb.data_ptr(), Yb.data_ptr(), b,
                                              grad.data_ptr(), loss.data_ptr(), work.data_ptr(),
                                              st))
        # cosine decay from lr to lr_final
        rate = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * (it - 1) / max(iters - 1, 1)))
        native._check("cp_mlp_adam", native.cp_mlp_adam(params.data_ptr(), grad.data_ptr(),
                                                        m.data_ptr(), v.data_ptr(), it, rate,
                                                        stream=st))
        if it == 1 or it % 100 == 0 or it == iters:
            losses.append(float(loss.item()))
    torch.cuda.synchronize()
    return params.cpu().numpy(), norm, losses


def evaluate(cfg, params, norm, steps=None, modes=(native.STRICT, native.WEAK,
                                                    native.WEAK_LEARNED)):
    """Run the same instance under each scheme (the network installed for the
    learned scheme only); V_gap(t) histories and timings."""
    torch = _torch()
    steps = int(steps or cfg["steps"])
    out = {}
    for mode in modes:
        g = load_gap(cfg, steps)
        if params is not None and mode == native.WEAK_LEARNED:
            g.set_predictor(params, norm)
        g.step(mode, 1)  # level 0 solve and first push outside the timing
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(mode, steps - 1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        h = g.history()
        g.close()
        out[mode] = dict(V_gap=h["V_gap"], J_hat=h["J_hat"], I_circ=h["I_circ"],
                         ms_per_step=1e3 * wall / (steps - 1))
    return out


def vgap_errors(res):
    """Max |V_gap - V_gap(strict)| / max |V_gap(strict)| of the weak schemes."""
    Vs = res[native.STRICT]["V_gap"]
    scale = np.abs(Vs).max()
    err = {}
    for mode in (native.WEAK, native.WEAK_LEARNED):
        if mode in res:
            err[mode] = float(np.abs(res[mode]["V_gap"] - Vs).max() / scale)
    return err
