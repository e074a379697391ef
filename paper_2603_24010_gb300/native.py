"""Thin ctypes binding of the C ABI in ``include/cp.h`` (argument marshalling only).

Every function named ``cp_*`` here calls the function of the same name in
``libcp.so``; the class :class:`Gap` bundles them for one gap instance.  All
arithmetic of the PIC step runs in the library's CUDA kernels.  There is no
CPU fallback: if the library cannot be built or loaded, or no GPU is
present, the calls raise.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_RESIDUAL, ERR_NONFINITE, ERR_TIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
ELECTRONS, IONS, SECONDARIES = 0, 1, 2
FP64, FP32 = 0, 1
SERIES_RLC, OPEN, TESLA = 0, 1, 2
UNITS_CELL, UNITS_SI = 0, 1

#: every symbol ``include/cp.h`` declares
EXPORTS = ("cp_create", "cp_set_particles", "cp_load_species", "cp_step_strict", "cp_step_weak", "cp_read_scalars",
           "cp_read_history", "cp_read_grid", "cp_get_particles", "cp_get_level",
           "cp_save_state", "cp_load_state", "cp_last_launch_count", "cp_enable_timing",
           "cp_read_timing", "cp_read_launch_times", "cp_push_ions_noalloc", "cp_set_predictor",
           "cp_step_weak_learned", "cp_predictor_samples", "cp_mlp_init", "cp_mlp_scales",
           "cp_mlp_normalize", "cp_mlp_forward", "cp_mlp_work_floats", "cp_mlp_loss_grad",
           "cp_mlp_adam", "cp_batch_create", "cp_batch_set_particles", "cp_batch_step_strict",
           "cp_batch_step_weak", "cp_batch_set_predictor", "cp_batch_step_weak_learned",
           "cp_batch_predictor_samples",
           "cp_batch_read_history", "cp_batch_read_grid",
           "cp_batch_get_particles", "cp_batch_status", "cp_batch_get_level",
           "cp_batch_last_launch_count", "cp_batch_set_launch", "cp_batch_get_launch",
           "cp_batch_autotune", "cp_batch_enable_timing", "cp_batch_read_timing",
           "cp_batch_destroy", "cp2d_create", "cp2d_set_particles", "cp2d_step_strict",
           "cp2d_step_weak", "cp2d_set_predictor", "cp2d_step_weak_learned", "cp2d_read_history",
           "cp2d_get_level", "cp2d_read_fields",
           "cp2d_get_particles", "cp2d_enable_timing", "cp2d_read_timing", "cp2d_last_launch_count",
           "cp2d_destroy", "cp_destroy", "cp_status_str")
STRICT, WEAK, WEAK_LEARNED = 0, 1, 2
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM = 40, 64, 2, 11074
PRED_WINDOW, PRED_FEATURES = 8, 5


class CpError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__("%s failed: %d (%s)" % (fn, status, cp_status_str(status)))


class cp_gap(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("d", "area", "eps0", "e", "m_e", "m_i", "weight",
                                          "sigma0")] + [("n_cells", C.c_int32), ("pad0", C.c_int32)]


class cp_tesla(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("R1", "R2", "R3", "C1", "C2", "C3", "L1", "L2", "M",
                                          "V1")]


class cp_circuit(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("R", "L", "C", "V0", "f", "tau", "polarity")] + [
        ("kind", C.c_int32), ("pad0", C.c_int32), ("tesla", cp_tesla)]


class cp_see_beam(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("gamma_coef", "gamma_max", "E_ref_eV", "scale",
                                          "T_emit_eV", "beam_E_eV", "beam_Emin_eV",
                                          "beam_Emax_eV")] + [
        ("beam_per_step", C.c_int32), ("beam_mode", C.c_int32), ("count_law", C.c_int32),
        ("energy_law", C.c_int32), ("ln_mu", C.c_double), ("ln_sigma", C.c_double)]


class cp_species(C.Structure):
    _fields_ = [("n0", C.c_double), ("T_load_eV", C.c_double), ("n_pairs", C.c_int64),
                ("weight", C.c_double)]


class cp_run(C.Structure):
    _fields_ = [("dt", C.c_double), ("seed", C.c_uint64), ("capacity", C.c_int64 * 3),
                ("max_steps", C.c_int64), ("precision", C.c_int32), ("compact_every", C.c_int32)]


class cp_diag(C.Structure):
    _fields_ = [("step", C.c_int64)] + [(n, C.c_double) for n in (
        "t", "V_gap", "I_circ", "Q_surf", "Q_conv", "Q_circ", "V_source", "residual",
        "ion_energy_eV", "max_cfl", "J_hat")] + [
        ("absorbed", (C.c_int64 * 3) * 2), ("emitted", C.c_int64 * 2), ("injected", C.c_int64),
        ("n_live", C.c_int64 * 3), ("conv_count", C.c_int64)]


class cp_transverse(C.Structure):
    _fields_ = [("n_cells_y", C.c_int32), ("sort_every", C.c_int32), ("length_y", C.c_double),
                ("beam_sigma", C.c_double), ("beam_y0", C.c_double)]


class cp_predictor(C.Structure):
    _fields_ = [("in_scale", C.c_float * 5), ("out_scale", C.c_float * 2), ("pad0", C.c_float),
                ("bound", C.c_double)]


_lib = None


def lib():
    """Load (building if needed) ``libcp.so``; raises if that is impossible."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
        u32p = C.POINTER(C.c_uint32)
        L.cp_create.argtypes = [C.POINTER(cp_gap), C.POINTER(cp_circuit), C.POINTER(cp_see_beam),
                                C.POINTER(cp_run), vp, C.POINTER(vp)]
        L.cp_set_particles.argtypes = [vp, C.c_int32, dp, dp, u32p, C.c_int64, C.c_int32]
        L.cp_load_species.argtypes = [vp, C.POINTER(cp_species), C.c_uint64]
        L.cp_step_strict.argtypes = [vp, C.c_int32, C.c_double]
        L.cp_step_weak.argtypes = [vp, C.c_int32]
        L.cp_read_scalars.argtypes = [vp, C.POINTER(cp_diag)]
        L.cp_read_history.argtypes = [vp, C.c_int64, C.c_int64, C.POINTER(cp_diag)]
        L.cp_read_grid.argtypes = [vp, dp, dp, dp, i64p, C.c_int32]
        L.cp_get_particles.argtypes = [vp, C.c_int32, dp, dp, u32p, C.c_int64, i64p]
        L.cp_get_level.argtypes = [vp, i64p]
        L.cp_save_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.cp_load_state.argtypes = [vp, vp, C.c_size_t]
        L.cp_last_launch_count.argtypes = [vp, i64p]
        L.cp_enable_timing.argtypes = [vp, C.c_int32]
        L.cp_read_timing.argtypes = [vp, dp, i64p]
        L.cp_read_launch_times.argtypes = [vp, dp, C.c_int64, i64p]
        L.cp_push_ions_noalloc.argtypes = [C.POINTER(cp_gap), C.POINTER(cp_see_beam), C.c_double,
                                           C.c_uint64, C.c_int64, C.c_int32, vp, vp, vp, vp,
                                           C.c_int64, vp, vp, vp, C.c_int64, vp, vp]
        fp = C.c_void_p  # device float arrays are passed as addresses
        L.cp_set_predictor.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(cp_predictor)]
        L.cp_step_weak_learned.argtypes = [vp, C.c_int32]
        L.cp_predictor_samples.argtypes = [vp, C.c_int64, C.c_int64, fp, fp]
        L.cp_mlp_init.argtypes = [fp, C.c_uint64, vp]
        L.cp_mlp_scales.argtypes = [fp, fp, C.c_int64, C.POINTER(cp_predictor), vp]
        L.cp_mlp_normalize.argtypes = [fp, fp, C.c_int64, C.POINTER(cp_predictor), fp, fp, vp]
        L.cp_mlp_forward.argtypes = [fp, fp, C.c_int64, fp, vp]
        L.cp_mlp_work_floats.argtypes = []
        L.cp_mlp_work_floats.restype = C.c_int64
        L.cp_mlp_loss_grad.argtypes = [fp, fp, fp, C.c_int64, fp, fp, fp, vp]
        L.cp_mlp_adam.argtypes = [fp, fp, fp, fp, C.c_int64, C.c_float, C.c_float, C.c_float,
                                  C.c_float, vp]
        L.cp_batch_create.argtypes = [C.c_int32, C.POINTER(cp_gap), C.POINTER(cp_circuit),
                                      C.POINTER(cp_see_beam), C.POINTER(cp_run), vp, C.POINTER(vp)]
        L.cp_batch_set_particles.argtypes = [vp, C.c_int32, C.c_int32, dp, dp, u32p, C.c_int64,
                                             C.c_int32]
        L.cp_batch_step_strict.argtypes = [vp, C.c_int32, C.c_double]
        L.cp_batch_step_weak.argtypes = [vp, C.c_int32]
        L.cp_batch_set_predictor.argtypes = [vp, C.c_int32, C.POINTER(C.c_float),
                                             C.POINTER(cp_predictor)]
        L.cp_batch_step_weak_learned.argtypes = [vp, C.c_int32]
        L.cp_batch_predictor_samples.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, C.c_void_p,
                                                 C.c_void_p]
        L.cp_batch_read_history.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, C.POINTER(cp_diag)]
        L.cp_batch_read_grid.argtypes = [vp, C.c_int32, dp, dp, dp, i64p, C.c_int32]
        L.cp_batch_get_particles.argtypes = [vp, C.c_int32, C.c_int32, dp, dp, u32p, C.c_int64, i64p]
        L.cp_batch_status.argtypes = [vp, C.POINTER(C.c_int32)]
        L.cp_batch_get_level.argtypes = [vp, C.c_int32, i64p]
        L.cp_batch_last_launch_count.argtypes = [vp, i64p]
        L.cp_batch_set_launch.argtypes = [vp, C.c_int32, C.c_int32]
        L.cp_batch_get_launch.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.cp_batch_autotune.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32), dp]
        L.cp_batch_enable_timing.argtypes = [vp, C.c_int32]
        L.cp_batch_read_timing.argtypes = [vp, dp, i64p]
        L.cp_batch_destroy.argtypes = [vp]
        L.cp_batch_destroy.restype = None
        L.cp2d_create.argtypes = [C.POINTER(cp_gap), C.POINTER(cp_transverse), C.POINTER(cp_circuit),
                                  C.POINTER(cp_see_beam), C.POINTER(cp_run), vp, C.POINTER(vp)]
        L.cp2d_set_particles.argtypes = [vp, C.c_int32, dp, dp, dp, dp, u32p, C.c_int64, C.c_int32]
        L.cp2d_step_strict.argtypes = [vp, C.c_int32, C.c_double]
        L.cp2d_step_weak.argtypes = [vp, C.c_int32]
        L.cp2d_set_predictor.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(cp_predictor)]
        L.cp2d_step_weak_learned.argtypes = [vp, C.c_int32]
        L.cp2d_read_history.argtypes = [vp, C.c_int64, C.c_int64, C.POINTER(cp_diag)]
        L.cp2d_get_level.argtypes = [vp, i64p]
        L.cp2d_read_fields.argtypes = [vp, dp, C.POINTER(C.c_float), C.POINTER(C.c_float), i64p]
        L.cp2d_get_particles.argtypes = [vp, C.c_int32, dp, dp, dp, dp, u32p, C.c_int64, i64p]
        L.cp2d_enable_timing.argtypes = [vp, C.c_int32]
        L.cp2d_read_timing.argtypes = [vp, dp, i64p]
        L.cp2d_last_launch_count.argtypes = [vp, i64p]
        L.cp2d_destroy.argtypes = [vp]
        L.cp2d_destroy.restype = None
        L.cp_destroy.argtypes = [vp]
        L.cp_destroy.restype = None
        L.cp_status_str.argtypes = [C.c_int]
        L.cp_status_str.restype = C.c_char_p
        _lib = L
    return _lib


def library_path():
    return _build.LIB


def _check(fn, rc):
    if rc != OK:
        raise CpError(fn, rc)
    return rc


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _i64p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int64))


def _u32p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_uint32))


# ---- one wrapper per C entry point -------------------------------------------
def cp_status_str(status):
    return lib().cp_status_str(int(status)).decode()


def cp_create(gap, circuit, see, run, stream=None):
    h = C.c_void_p()
    _check("cp_create", lib().cp_create(C.byref(gap), C.byref(circuit), C.byref(see),
                                        C.byref(run), C.c_void_p(stream or 0), C.byref(h)))
    return h


def cp_set_particles(ctx, species, x, v, ids=None, units=UNITS_CELL):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
    return lib().cp_set_particles(ctx, int(species), _dp(x), _dp(v), _u32p(ids), x.size, int(units))


def cp_load_species(ctx, n_pairs, T_load_eV, seed, n0=0.0, weight=0.0):
    sp = cp_species(n0=float(n0), T_load_eV=float(T_load_eV), n_pairs=int(n_pairs),
                    weight=float(weight))
    return lib().cp_load_species(ctx, C.byref(sp), int(seed) & (2**64 - 1))


def cp_step_strict(ctx, n_steps, residual_tol=1e-12):
    return lib().cp_step_strict(ctx, int(n_steps), float(residual_tol))


def cp_step_weak(ctx, n_steps):
    return lib().cp_step_weak(ctx, int(n_steps))


def cp_read_scalars(ctx):
    d = cp_diag()
    _check("cp_read_scalars", lib().cp_read_scalars(ctx, C.byref(d)))
    return d


def cp_read_history(ctx, first, n):
    arr = (cp_diag * int(n))()
    _check("cp_read_history", lib().cp_read_history(ctx, int(first), int(n), arr))
    return arr


def cp_read_grid(ctx, n_nodes):
    phi, rho = np.zeros(n_nodes), np.zeros(n_nodes)
    E = np.zeros(n_nodes - 1)
    G = np.zeros(n_nodes, dtype=np.int64)
    _check("cp_read_grid", lib().cp_read_grid(ctx, _dp(phi), _dp(rho), _dp(E), _i64p(G),
                                              int(n_nodes)))
    return dict(phi=phi, rho=rho, E=E, G=G)


def cp_get_particles(ctx, species, cap=None):
    """Live particles of one species (cell units); sized by a first query if cap is None."""
    n = C.c_int64()
    if cap is None:
        rc = lib().cp_get_particles(ctx, int(species), None, None, None, 0, C.byref(n))
        if rc not in (OK, ERR_CAPACITY):
            _check("cp_get_particles", rc)
        cap = n.value
    xi, u = np.zeros(max(int(cap), 1)), np.zeros(max(int(cap), 1))
    ids = np.zeros(max(int(cap), 1), dtype=np.uint32)
    _check("cp_get_particles", lib().cp_get_particles(ctx, int(species), _dp(xi), _dp(u),
                                                      _u32p(ids), int(cap), C.byref(n)))
    m = n.value
    return xi[:m], u[:m], (ids[:m] if species == IONS else None)


def cp_get_level(ctx):
    lv = C.c_int64()
    _check("cp_get_level", lib().cp_get_level(ctx, C.byref(lv)))
    return lv.value


def cp_save_state(ctx):
    n = C.c_size_t()
    _check("cp_save_state", lib().cp_save_state(ctx, None, C.byref(n)))
    buf = (C.c_ubyte * n.value)()
    _check("cp_save_state", lib().cp_save_state(ctx, buf, C.byref(n)))
    return bytes(buf)


def cp_load_state(ctx, blob):
    buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
    return lib().cp_load_state(ctx, buf, len(blob))


def cp_last_launch_count(ctx):
    n = C.c_int64()
    _check("cp_last_launch_count", lib().cp_last_launch_count(ctx, C.byref(n)))
    return n.value


def cp_enable_timing(ctx, on):
    _check("cp_enable_timing", lib().cp_enable_timing(ctx, int(bool(on))))


def cp_read_timing(ctx):
    ms = np.zeros(3)
    n = np.zeros(3, dtype=np.int64)
    _check("cp_read_timing", lib().cp_read_timing(ctx, _dp(ms), _i64p(n)))
    return ms, n


def cp_read_launch_times(ctx):
    n = C.c_int64()
    rc = lib().cp_read_launch_times(ctx, None, 0, C.byref(n))
    if rc not in (OK, ERR_CAPACITY):
        _check("cp_read_launch_times", rc)
    ms = np.zeros(max(n.value, 1))
    _check("cp_read_launch_times", lib().cp_read_launch_times(ctx, _dp(ms), n.value, C.byref(n)))
    return ms[:n.value]


def cp_push_ions_noalloc(gap, see, dt, seed, step, half_kick, E, xi, u, ids, n, G, se_xi, se_u,
                         se_cap, counts, stream=None):
    """Allocation-free ion push; every buffer argument is a device address (int)."""
    return lib().cp_push_ions_noalloc(C.byref(gap), C.byref(see), float(dt), int(seed), int(step),
                                      int(half_kick), E, xi, u, ids, int(n), G, se_xi, se_u,
                                      int(se_cap), counts, C.c_void_p(stream or 0))


def cp_set_predictor(ctx, params, norm):
    """params: host FP32 array of MLP_NPARAM values; norm: cp_predictor."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != MLP_NPARAM:
        raise ValueError("expected %d parameters" % MLP_NPARAM)
    return lib().cp_set_predictor(ctx, p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(norm))


def cp_step_weak_learned(ctx, n_steps):
    return lib().cp_step_weak_learned(ctx, int(n_steps))


def cp_predictor_samples(ctx, first_level, n, X, Y):
    """X, Y: device addresses (int) of n x 40 and n x 2 FP32 arrays."""
    return lib().cp_predictor_samples(ctx, int(first_level), int(n), X, Y)


def cp_mlp_init(params, seed, stream=None):
    return lib().cp_mlp_init(params, int(seed), C.c_void_p(stream or 0))


def cp_mlp_scales(X, Y, n, norm, stream=None):
    return lib().cp_mlp_scales(X, Y, int(n), C.byref(norm), C.c_void_p(stream or 0))


def cp_mlp_normalize(X, Y, n, norm, Xn, Yn, stream=None):
    return lib().cp_mlp_normalize(X, Y, int(n), C.byref(norm), Xn, Yn, C.c_void_p(stream or 0))


def cp_mlp_forward(params, Xn, n, Yhat, stream=None):
    return lib().cp_mlp_forward(params, Xn, int(n), Yhat, C.c_void_p(stream or 0))


def cp_mlp_work_floats():
    return int(lib().cp_mlp_work_floats())


def cp_mlp_loss_grad(params, Xn, Yn, n, grad, loss, work, stream=None):
    return lib().cp_mlp_loss_grad(params, Xn, Yn, int(n), grad, loss, work, C.c_void_p(stream or 0))


def cp_mlp_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return lib().cp_mlp_adam(params, grad, m, v, int(t), float(lr), float(beta1), float(beta2),
                             float(eps), C.c_void_p(stream or 0))


def cp_destroy(ctx):
    lib().cp_destroy(ctx)


# ---- convenience ---------------------------------------------------------------
def structs_from_config(cfg, capacity=(0, 0, 0), max_steps=None, compact_every=0):
    """Fill the four parameter structs from a workload dictionary."""
    gap = cp_gap(d=cfg["d"], area=cfg.get("area", 0.0), eps0=cfg["eps0"], e=cfg["e"],
                 m_e=cfg["m_e"], m_i=cfg["m_i"], weight=cfg["weight"],
                 sigma0=cfg.get("sigma0", 0.0), n_cells=int(cfg["n_cells"]))
    circ = cp_circuit(R=cfg["R"], L=cfg["L"], C=cfg["C"], V0=cfg["V0"], f=cfg["f"],
                      tau=cfg["tau"], polarity=cfg["polarity"], kind=int(cfg.get("circuit", 0)))
    if circ.kind == TESLA:
        circ.tesla = cp_tesla(**{k: cfg["t" + k] for k, _ in cp_tesla._fields_})
    see = cp_see_beam(gamma_coef=cfg["gamma_coef"], gamma_max=cfg["gamma_max"],
                      E_ref_eV=cfg["E_ref_eV"], scale=cfg["see_scale"], T_emit_eV=cfg["T_emit_eV"],
                      beam_E_eV=cfg["beam_E_eV"], beam_Emin_eV=cfg["beam_Emin_eV"],
                      beam_Emax_eV=cfg["beam_Emax_eV"], beam_per_step=int(cfg["beam_per_step"]),
                      beam_mode=int(cfg["beam_mode"]), count_law=int(cfg.get("see_count_law", 0)),
                      energy_law=int(cfg.get("see_energy_law", 0)),
                      ln_mu=float(cfg.get("see_ln_mu", 0.0)), ln_sigma=float(cfg.get("see_ln_sigma", 0.0)))
    run = cp_run(dt=cfg["dt"], seed=int(cfg["seed"]), max_steps=int(max_steps or cfg["steps"]),
                 precision=int(cfg.get("precision", FP64)), compact_every=int(compact_every))
    for s in range(3):
        run.capacity[s] = int(capacity[s])
    return gap, circ, see, run


def current_stream():
    """The caller's CUDA stream: torch's current stream on the current device."""
    import torch
    return torch.cuda.current_stream().cuda_stream


class Gap:
    """One gap instance driven through the C ABI."""

    def __init__(self, cfg, capacity=(0, 0, 0), max_steps=None, compact_every=0, stream=None):
        self.cfg = dict(cfg)
        self.N = int(cfg["n_cells"])
        structs = structs_from_config(cfg, capacity, max_steps, compact_every)
        self.ctx = cp_create(*structs, stream=current_stream() if stream is None else stream)

    def close(self):
        if getattr(self, "ctx", None):
            cp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, species, xi, u, ids=None, units=UNITS_CELL):
        _check("cp_set_particles", cp_set_particles(self.ctx, species, xi, u, ids, units))

    def load_species(self, n_pairs, T_load_eV, seed, n0=0.0, weight=0.0):
        """Draw the initial co-located electron/ion pairs on the device."""
        _check("cp_load_species", cp_load_species(self.ctx, n_pairs, T_load_eV, seed, n0, weight))

    def step(self, mode, n_steps, tol=1e-12):
        if mode == STRICT:
            _check("cp_step_strict", cp_step_strict(self.ctx, n_steps, tol))
        elif mode == WEAK:
            _check("cp_step_weak", cp_step_weak(self.ctx, n_steps))
        elif mode == WEAK_LEARNED:
            _check("cp_step_weak_learned", cp_step_weak_learned(self.ctx, n_steps))
        else:
            raise ValueError("unknown coupling mode %r" % (mode,))

    def set_predictor(self, params, norm):
        _check("cp_set_predictor", cp_set_predictor(self.ctx, params, norm))

    @property
    def level(self):
        return cp_get_level(self.ctx)

    def scalars(self):
        return cp_read_scalars(self.ctx)

    def history(self, first=0, n=None):
        if n is None:
            n = self.level + 1 - first
        arr = cp_read_history(self.ctx, first, n)
        return diag_to_dict(arr)

    def grid(self):
        return cp_read_grid(self.ctx, self.N + 1)

    def particles(self, species):
        return cp_get_particles(self.ctx, species)


def _diag_dtype():
    names, formats, offsets = [], [], []
    for name, typ in cp_diag._fields_:
        names.append(name)
        offsets.append(getattr(cp_diag, name).offset)
        if name == "absorbed":
            formats.append(("<i8", (2, 3)))
        elif name == "emitted":
            formats.append(("<i8", (2,)))
        elif name == "n_live":
            formats.append(("<i8", (3,)))
        else:
            formats.append("<i8" if typ is C.c_int64 else "<f8")
    return np.dtype(dict(names=names, formats=formats, offsets=offsets,
                         itemsize=C.sizeof(cp_diag)))


_DIAG_DTYPE = None


def diag_to_dict(arr):
    """Column view (copies) of a ctypes array of cp_diag rows."""
    global _DIAG_DTYPE
    if _DIAG_DTYPE is None:
        _DIAG_DTYPE = _diag_dtype()
    rows = np.frombuffer(arr, dtype=_DIAG_DTYPE, count=len(arr))
    return {name: np.array(rows[name]) for name, _ in cp_diag._fields_}


class Batch:
    """An ensemble of independent gap instances driven through the cp_batch_* calls."""

    def __init__(self, cfgs, max_steps, compact_every=0, stream=None, capacity=(0, 0, 0)):
        n = len(cfgs)
        self.cfgs = [dict(c) for c in cfgs]
        self.n = n
        gaps, circs, sees, runs = (cp_gap * n)(), (cp_circuit * n)(), (cp_see_beam * n)(), (cp_run * n)()
        for i, cfg in enumerate(cfgs):
            g, c, s, r = structs_from_config(cfg, capacity=capacity, max_steps=max_steps,
                                             compact_every=compact_every)
            gaps[i], circs[i], sees[i], runs[i] = g, c, s, r
        h = C.c_void_p()
        _check("cp_batch_create", lib().cp_batch_create(
            n, gaps, circs, sees, runs, C.c_void_p(current_stream() if stream is None else stream),
            C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().cp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, i, species, xi, u, ids=None, units=UNITS_CELL):
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
        _check("cp_batch_set_particles", lib().cp_batch_set_particles(
            self.h, int(i), int(species), _dp(xi), _dp(u), _u32p(ids), xi.size, int(units)))

    def step(self, mode, n_steps, tol=1e-12):
        """Returns the first non-zero instance status (0 if none)."""
        if mode == STRICT:
            return lib().cp_batch_step_strict(self.h, int(n_steps), float(tol))
        if mode == WEAK:
            return lib().cp_batch_step_weak(self.h, int(n_steps))
        if mode == WEAK_LEARNED:
            return lib().cp_batch_step_weak_learned(self.h, int(n_steps))
        raise ValueError("unknown coupling mode %r" % (mode,))

    def predictor_samples(self, i, first_level, n, X, Y):
        """Instance i's training samples into device arrays X (n x 40), Y (n x 2)."""
        _check("cp_batch_predictor_samples", lib().cp_batch_predictor_samples(
            self.h, int(i), int(first_level), int(n), C.c_void_p(X), C.c_void_p(Y)))

    def set_predictor(self, i, params, norm):
        """Install a network on instance i (as Gap.set_predictor)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_NPARAM:
            raise ValueError("expected %d parameters" % MLP_NPARAM)
        _check("cp_batch_set_predictor", lib().cp_batch_set_predictor(
            self.h, int(i), p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(norm)))

    def level_of(self, i):
        lv = C.c_int64()
        _check("cp_batch_get_level", lib().cp_batch_get_level(self.h, int(i), C.byref(lv)))
        return lv.value

    @property
    def level(self):
        return self.level_of(0)

    def history(self, i, first=0, n=None):
        if n is None:
            n = self.level_of(i) + 1 - first
        arr = (cp_diag * int(n))()
        _check("cp_batch_read_history", lib().cp_batch_read_history(self.h, int(i), int(first),
                                                                    int(n), arr))
        return diag_to_dict(arr)

    def grid(self, i):
        N = int(self.cfgs[i]["n_cells"])
        phi, rho, E = np.zeros(N + 1), np.zeros(N + 1), np.zeros(N)
        G = np.zeros(N + 1, dtype=np.int64)
        _check("cp_batch_read_grid", lib().cp_batch_read_grid(self.h, int(i), _dp(phi), _dp(rho),
                                                              _dp(E), _i64p(G), N + 1))
        return dict(phi=phi, rho=rho, E=E, G=G)

    def particles(self, i, species):
        n = C.c_int64()
        rc = lib().cp_batch_get_particles(self.h, int(i), int(species), None, None, None, 0,
                                          C.byref(n))
        if rc not in (OK, ERR_CAPACITY):
            _check("cp_batch_get_particles", rc)
        cap = max(n.value, 1)
        xi, u = np.zeros(cap), np.zeros(cap)
        ids = np.zeros(cap, dtype=np.uint32)
        _check("cp_batch_get_particles", lib().cp_batch_get_particles(
            self.h, int(i), int(species), _dp(xi), _dp(u), _u32p(ids), cap, C.byref(n)))
        m = n.value
        return xi[:m], u[:m], (ids[:m] if species == IONS else None)

    def status(self):
        st = (C.c_int32 * self.n)()
        _check("cp_batch_status", lib().cp_batch_status(self.h, st))
        return np.array(st[:], dtype=np.int32)

    def set_launch(self, threads, ctas_per_sm=0):
        return lib().cp_batch_set_launch(self.h, int(threads), int(ctas_per_sm))

    def launch(self):
        t, g = C.c_int32(), C.c_int32()
        _check("cp_batch_get_launch", lib().cp_batch_get_launch(self.h, C.byref(t), C.byref(g)))
        return t.value, g.value

    def autotune(self, steps_per_shape, mode=STRICT, tol=1e-12):
        t, p = C.c_int32(), C.c_int32()
        ms = C.c_double()
        rc = lib().cp_batch_autotune(self.h, int(steps_per_shape), int(mode), float(tol),
                                     C.byref(t), C.byref(p), C.byref(ms))
        return rc, t.value, p.value, ms.value

    def enable_timing(self, on):
        _check("cp_batch_enable_timing", lib().cp_batch_enable_timing(self.h, int(bool(on))))

    def timing(self):
        ms = np.zeros(3)
        n = np.zeros(3, dtype=np.int64)
        _check("cp_batch_read_timing", lib().cp_batch_read_timing(self.h, _dp(ms), _i64p(n)))
        return ms, n

    def last_launch_count(self):
        n = C.c_int64()
        _check("cp_batch_last_launch_count", lib().cp_batch_last_launch_count(self.h, C.byref(n)))
        return n.value


class Gap2D:
    """The 2D planar gap (x normal, y periodic) driven through the cp2d_* calls."""

    def __init__(self, cfg, max_steps=None, sort_every=0, capacity=(0, 0, 0), stream=None):
        self.cfg = dict(cfg)
        self.Nx, self.Ny = int(cfg["n_cells"]), int(cfg["Ny"])
        gap, circ, see, run = structs_from_config(cfg, capacity=capacity, max_steps=max_steps)
        tr = cp_transverse(n_cells_y=self.Ny, sort_every=int(sort_every), length_y=cfg["Ly"],
                           beam_sigma=cfg["beam_sigma"], beam_y0=cfg["beam_yc"])
        h = C.c_void_p()
        _check("cp2d_create", lib().cp2d_create(C.byref(gap), C.byref(tr), C.byref(circ),
                                                C.byref(see), C.byref(run),
                                                C.c_void_p(current_stream() if stream is None else stream),
                                                C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().cp2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, species, xi, eta, u, w, ids=None, units=UNITS_CELL):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (xi, eta, u, w)]
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
        _check("cp2d_set_particles", lib().cp2d_set_particles(
            self.h, int(species), _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(a[3]), _u32p(ids),
            a[0].size, int(units)))

    def step(self, mode, n_steps, tol=1e-12):
        if mode == STRICT:
            rc = lib().cp2d_step_strict(self.h, int(n_steps), float(tol))
        elif mode == WEAK:
            rc = lib().cp2d_step_weak(self.h, int(n_steps))
        elif mode == WEAK_LEARNED:
            rc = lib().cp2d_step_weak_learned(self.h, int(n_steps))
        else:
            raise ValueError("unknown coupling mode %r" % (mode,))
        _check("cp2d_step", rc)

    def set_predictor(self, params, norm):
        """Install a network on the transverse mean (as Gap.set_predictor)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_NPARAM:
            raise ValueError("expected %d parameters" % MLP_NPARAM)
        _check("cp2d_set_predictor", lib().cp2d_set_predictor(
            self.h, p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(norm)))

    @property
    def level(self):
        lv = C.c_int64()
        _check("cp2d_get_level", lib().cp2d_get_level(self.h, C.byref(lv)))
        return lv.value

    def history(self, first=0, n=None):
        if n is None:
            n = self.level + 1 - first
        arr = (cp_diag * int(n))()
        _check("cp2d_read_history", lib().cp2d_read_history(self.h, int(first), int(n), arr))
        return diag_to_dict(arr)

    def fields(self):
        Nx, Ny = self.Nx, self.Ny
        phi = np.zeros((Nx + 1) * Ny)
        Ex = np.zeros(Nx * Ny, dtype=np.float32)
        Ey = np.zeros((Nx + 1) * Ny, dtype=np.float32)
        G = np.zeros((Nx + 1) * Ny, dtype=np.int64)
        fp = C.POINTER(C.c_float)
        _check("cp2d_read_fields", lib().cp2d_read_fields(
            self.h, _dp(phi), Ex.ctypes.data_as(fp), Ey.ctypes.data_as(fp), _i64p(G)))
        return dict(phi=phi.reshape(Nx + 1, Ny), Ex=Ex.reshape(Nx, Ny), Ey=Ey.reshape(Nx + 1, Ny),
                    G=G.reshape(Nx + 1, Ny))

    def particles(self, species):
        n = C.c_int64()
        rc = lib().cp2d_get_particles(self.h, int(species), None, None, None, None, None, 0,
                                      C.byref(n))
        if rc not in (OK, ERR_CAPACITY):
            _check("cp2d_get_particles", rc)
        cap = max(n.value, 1)
        a = [np.zeros(cap) for _ in range(4)]
        ids = np.zeros(cap, dtype=np.uint32)
        _check("cp2d_get_particles", lib().cp2d_get_particles(
            self.h, int(species), _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(a[3]), _u32p(ids), cap,
            C.byref(n)))
        m = n.value
        return [v[:m] for v in a] + [ids[:m] if species == IONS else None]

    def enable_timing(self, on):
        _check("cp2d_enable_timing", lib().cp2d_enable_timing(self.h, int(bool(on))))

    def timing(self):
        ms = np.zeros(3)
        n = np.zeros(3, dtype=np.int64)
        _check("cp2d_read_timing", lib().cp2d_read_timing(self.h, _dp(ms), _i64p(n)))
        return ms, n

    def last_launch_count(self):
        n = C.c_int64()
        _check("cp2d_last_launch_count", lib().cp2d_last_launch_count(self.h, C.byref(n)))
        return n.value
