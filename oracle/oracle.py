"""ctypes wrapper of the FP64 CPU oracle (``cp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s cpu_baseline leg; the product path never imports it.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

ELECTRONS, IONS, SECONDARIES = 0, 1, 2
STRICT, WEAK, WEAK_LEARNED = 0, 1, 2
MLP_IN, MLP_OUT, MLP_NPARAM = 40, 2, 11074
SERIES_RLC, OPEN, TESLA = 0, 1, 2
OK, ERR_ARG, ERR_RESIDUAL, ERR_NONFINITE = 0, -1, -5, -6
TAG_SEE, TAG_BEAM = 0x5345, 0x4245


class OrParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "d", "area", "eps0", "e", "m_e", "m_i", "R", "L", "C", "V0", "f", "tau",
        "polarity", "gamma_coef", "gamma_max", "E_ref_eV", "see_scale", "T_emit_eV",
        "beam_E_eV", "beam_Emin_eV", "beam_Emax_eV", "dt", "weight", "sigma0", "grid_units",
        "tR1", "tR2", "tR3", "tC1", "tC2", "tC3", "tL1", "tL2", "tM", "tV1",
        "see_ln_mu", "see_ln_sigma")] + [
        ("seed", C.c_uint64), ("n_cells", C.c_int64), ("circuit", C.c_int64),
        ("beam_per_step", C.c_int64), ("beam_mode", C.c_int64), ("see_count_law", C.c_int64),
        ("see_energy_law", C.c_int64)]


class OrDiag(C.Structure):
    _fields_ = [("step", C.c_int64)] + [(n, C.c_double) for n in (
        "t", "V_gap", "I_circ", "Q_surf", "Q_conv", "Q_circ", "V_source", "residual",
        "ion_energy_eV", "max_cfl", "J_hat")] + [
        ("absorbed", (C.c_int64 * 3) * 2), ("emitted", C.c_int64 * 2), ("injected", C.c_int64),
        ("n_live", C.c_int64 * 3), ("conv_count", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int64)
        up = C.POINTER(C.c_uint64)
        u32p = C.POINTER(C.c_uint32)
        L.or_philox4x64_10.argtypes = [up, up, up]
        L.or_u01.argtypes = [C.c_uint64]
        L.or_u01.restype = C.c_double
        L.or_source.argtypes = [C.POINTER(OrParams), C.c_double]
        L.or_source.restype = C.c_double
        L.or_deposit.argtypes = [C.c_int64, C.c_int64, dp, C.c_int64, ip]
        L.or_gather.argtypes = [dp, C.c_int64, C.c_double]
        L.or_gather.restype = C.c_double
        L.or_thomas.argtypes = [C.c_int64, dp, dp, dp, dp, dp]
        L.or_see_count.argtypes = [C.POINTER(OrParams), C.c_double, C.c_uint64, C.c_int64, dp]
        L.or_see_count.restype = C.c_int64
        L.or_see_electron.argtypes = [C.POINTER(OrParams), C.c_uint64, C.c_int64, C.c_int64,
                                      dp, dp]
        L.or_see_count_batch.argtypes = [C.POINTER(OrParams), C.c_double, C.c_uint64, C.c_int64,
                                         C.c_int64, ip]
        L.or_see_electron_batch.argtypes = [C.POINTER(OrParams), C.c_uint64, C.c_int64, C.c_int64,
                                            dp, dp]
        L.or_load_pairs.argtypes = [C.POINTER(OrParams), C.c_int64, C.c_double, C.c_uint64, dp, dp,
                                    dp]
        L.or_tesla_matrix.argtypes = [C.POINTER(OrParams), C.c_int, dp]
        L.or_tesla_rhs.argtypes = [C.POINTER(OrParams), dp, dp]
        L.or_solve5.argtypes = [dp, dp, dp]
        L.or_tesla_step.argtypes = [C.POINTER(OrParams), dp]
        L.or_tesla_state.argtypes = [C.c_void_p, dp]
        L.or_create.argtypes = [C.POINTER(OrParams)]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_particles.argtypes = [C.c_void_p, C.c_int32, dp, dp, u32p, C.c_int64]
        L.or_step.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_double]
        L.or_level.argtypes = [C.c_void_p]
        L.or_level.restype = C.c_int64
        L.or_n_live.argtypes = [C.c_void_p, C.c_int32]
        L.or_n_live.restype = C.c_int64
        L.or_get_particles.argtypes = [C.c_void_p, C.c_int32, dp, dp, u32p, C.c_int64]
        L.or_read_grid.argtypes = [C.c_void_p, dp, dp, dp, ip]
        L.or_history_len.argtypes = [C.c_void_p]
        L.or_history_len.restype = C.c_int64
        L.or_read_history.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(OrDiag)]
        L.or_solve_fields.argtypes = [C.POINTER(OrParams), C.c_int32, ip, C.c_int64, C.c_double,
                                      dp, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp,
                                      dp]
        fp = C.POINTER(C.c_float)
        L.or_bf16.argtypes = [C.c_float]
        L.or_bf16.restype = C.c_double
        L.or_gelu.argtypes = [C.c_double]
        L.or_gelu.restype = C.c_double
        L.or_gelu_grad.argtypes = [C.c_double]
        L.or_gelu_grad.restype = C.c_double
        L.or_mlp_forward.argtypes = [fp, C.c_int64, dp, dp]
        L.or_mlp_loss_grad.argtypes = [fp, C.c_int64, dp, dp, dp, dp]
        L.or_adam.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_int64, C.c_double, C.c_double,
                              C.c_double, C.c_double]
        L.or_set_predictor.argtypes = [C.c_void_p, fp, dp, dp, C.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def make_params(cfg: dict) -> OrParams:
    """Fill the oracle's parameter struct from a workload dictionary."""
    p = OrParams()
    for name, _ in OrParams._fields_:
        if name in cfg:
            setattr(p, name, cfg[name])
    return p


def philox4x64_10(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) & (2**64 - 1) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) & (2**64 - 1) for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def u01(w):
    return lib().or_u01(C.c_uint64(int(w)))


def source(cfg, t):
    p = make_params(cfg)
    return lib().or_source(C.byref(p), float(t))


def deposit(N, xi, sign, G=None):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    if G is None:
        G = np.zeros(N + 1, dtype=np.int64)
    lib().or_deposit(N, xi.size, _dp(xi), int(sign), _ip(G))
    return G


def gather(E, N, xi):
    E = np.ascontiguousarray(E, dtype=np.float64)
    return lib().or_gather(_dp(E), N, float(xi))


def thomas(a, b, c, r):
    a, b, c, r = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, r))
    x = np.zeros_like(r)
    lib().or_thomas(r.size, _dp(a), _dp(b), _dp(c), _dp(r), _dp(x))
    return x


def see_count(cfg, E_eV, ion_id, step):
    p = make_params(cfg)
    g = C.c_double()
    n = lib().or_see_count(C.byref(p), float(E_eV), int(ion_id), int(step), C.byref(g))
    return int(n), g.value


def see_electron(cfg, ion_id, step, j):
    p = make_params(cfg)
    v, fr = C.c_double(), C.c_double()
    lib().or_see_electron(C.byref(p), int(ion_id), int(step), int(j), C.byref(v), C.byref(fr))
    return v.value, fr.value


def see_count_batch(cfg, E_eV, id0, n, step):
    p = make_params(cfg)
    out = np.zeros(int(n), dtype=np.int64)
    lib().or_see_count_batch(C.byref(p), float(E_eV), int(id0), int(n), int(step), _ip(out))
    return out


def see_electron_batch(cfg, id0, n, step):
    p = make_params(cfg)
    v = np.zeros(int(n))
    fr = np.zeros(int(n))
    lib().or_see_electron_batch(C.byref(p), int(id0), int(n), int(step), _dp(v), _dp(fr))
    return v, fr


def load_pairs(cfg, n, T_eV, seed):
    """The initial plasma of n co-located pairs: (xi, u_e, u_i) in cell units."""
    p = make_params(cfg)
    xi, ue, ui = np.zeros(int(n)), np.zeros(int(n)), np.zeros(int(n))
    lib().or_load_pairs(C.byref(p), int(n), float(T_eV), int(seed) & (2**64 - 1), _dp(xi), _dp(ue),
                        _dp(ui))
    return xi, ue, ui


def tesla_matrix(cfg, coupled=False):
    """The BDF2 circuit matrix of the Tesla loops (5 x 5)."""
    p = make_params(cfg)
    T = np.zeros(25)
    lib().or_tesla_matrix(C.byref(p), int(bool(coupled)), _dp(T))
    return T.reshape(5, 5)


def tesla_run(cfg, steps, Q0=None):
    """The Tesla circuit alone for `steps` BDF2 steps from rest in the state
    Q0 (default: only C1 charged, to tV1): loop charges (steps + 1, 5), row 0
    the initial state."""
    p = make_params(cfg)
    Qh = np.zeros((4, 5))
    if Q0 is None:
        Qh[:, 0] = cfg["tC1"] * cfg["tV1"]
    else:
        Qh[:] = np.asarray(Q0, np.float64)[None, :]
    out = [Qh[0].copy()]
    for _ in range(int(steps)):
        if lib().or_tesla_step(C.byref(p), _dp(Qh)) != OK:
            raise ValueError("or_tesla_step failed")
        out.append(Qh[0].copy())
    return np.array(out)


def solve_fields(cfg, mode, G, conv_count, sigma_prev, Qhist, t, tol=1e-12, phi0_prev=0.0,
                 J_hat=0.0):
    p = make_params(cfg)
    N = int(cfg["n_cells"])
    G = np.ascontiguousarray(G, dtype=np.int64)
    Qh = np.ascontiguousarray(Qhist, dtype=np.float64)
    phi = np.zeros(N + 1)
    E = np.zeros(N)
    out = np.zeros(4)
    rc = lib().or_solve_fields(C.byref(p), int(mode), _ip(G), int(conv_count), float(sigma_prev),
                               _dp(Qh), float(phi0_prev), float(J_hat), float(t), float(tol),
                               _dp(phi), _dp(E), _dp(out))
    return rc, phi, E, dict(Q_n=out[0], sigma_n=out[1], I=out[2], residual=out[3])


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def bf16(w):
    """bfloat16 rounding (nearest, ties to even) of FP32 values, as float64."""
    w = np.asarray(w, dtype=np.float32)
    return np.array([lib().or_bf16(float(v)) for v in w.ravel()]).reshape(w.shape)


def gelu(x):
    return lib().or_gelu(float(x))


def gelu_grad(x):
    return lib().or_gelu_grad(float(x))


def mlp_forward(params, Xn):
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(Xn, dtype=np.float64).reshape(-1, MLP_IN)
    Y = np.zeros((X.shape[0], MLP_OUT))
    lib().or_mlp_forward(_fp(p), X.shape[0], _dp(X), _dp(Y))
    return Y


def mlp_loss_grad(params, Xn, Yn):
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(Xn, dtype=np.float64).reshape(-1, MLP_IN)
    Y = np.ascontiguousarray(Yn, dtype=np.float64).reshape(-1, MLP_OUT)
    g = np.zeros(MLP_NPARAM)
    loss = np.zeros(1)
    lib().or_mlp_loss_grad(_fp(p), X.shape[0], _dp(X), _dp(Y), _dp(g), _dp(loss))
    return float(loss[0]), g


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place FP64 Adam step on float64 arrays."""
    lib().or_adam(p.size, _dp(p), _dp(np.ascontiguousarray(g, dtype=np.float64)), _dp(m), _dp(v),
                  int(t), float(lr), float(b1), float(b2), float(eps))


class OracleGap:
    """One gap instance advanced by the oracle."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self.N = int(cfg["n_cells"])
        self._p = make_params(cfg)
        self._s = lib().or_create(C.byref(self._p))
        if not self._s:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._s:
            lib().or_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, species, xi, u, ids=None):
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        idp = None
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
            idp = ids.ctypes.data_as(C.POINTER(C.c_uint32))
        rc = lib().or_set_particles(self._s, species, _dp(xi), _dp(u), idp, xi.size)
        if rc != OK:
            raise ValueError("or_set_particles failed: %d" % rc)

    def set_predictor(self, params, in_scale, out_scale, bound):
        p = np.ascontiguousarray(params, dtype=np.float32)
        si = np.ascontiguousarray(in_scale, dtype=np.float64)
        so = np.ascontiguousarray(out_scale, dtype=np.float64)
        rc = lib().or_set_predictor(self._s, _fp(p), _dp(si), _dp(so), float(bound))
        if rc != OK:
            raise ValueError("or_set_predictor failed: %d" % rc)

    def step(self, mode, n_steps, tol=1e-12):
        return lib().or_step(self._s, int(mode), int(n_steps), float(tol))

    @property
    def level(self):
        return lib().or_level(self._s)

    def n_live(self, species):
        return lib().or_n_live(self._s, species)

    def tesla_state(self):
        Q = np.zeros(5)
        lib().or_tesla_state(self._s, _dp(Q))
        return Q

    def particles(self, species):
        n = self.n_live(species)
        xi = np.zeros(n)
        u = np.zeros(n)
        ids = np.zeros(n, dtype=np.uint32)
        lib().or_get_particles(self._s, species, _dp(xi), _dp(u),
                               ids.ctypes.data_as(C.POINTER(C.c_uint32)), n)
        return xi, u, (ids if species == IONS else None)

    def grid(self):
        N = self.N
        phi, rho, E = np.zeros(N + 1), np.zeros(N + 1), np.zeros(N)
        G = np.zeros(N + 1, dtype=np.int64)
        lib().or_read_grid(self._s, _dp(phi), _dp(rho), _dp(E), _ip(G))
        return dict(phi=phi, rho=rho, E=E, G=G)

    def history(self):
        n = lib().or_history_len(self._s)
        arr = (OrDiag * n)()
        if n:
            lib().or_read_history(self._s, 0, n, arr)
        return diag_to_dict(arr)


def diag_to_dict(arr):
    """Column view of a ctypes diagnostics array."""
    out = {}
    n = len(arr)
    for name, typ in OrDiag._fields_:
        if name == "absorbed":
            out[name] = np.array([[[arr[k].absorbed[e][s] for s in range(3)] for e in range(2)]
                                  for k in range(n)], dtype=np.int64).reshape(n, 2, 3)
        elif name in ("emitted", "n_live"):
            m = 2 if name == "emitted" else 3
            out[name] = np.array([[getattr(arr[k], name)[j] for j in range(m)] for k in range(n)],
                                 dtype=np.int64).reshape(n, m)
        else:
            dt = np.int64 if typ in (C.c_int64,) else np.float64
            out[name] = np.array([getattr(arr[k], name) for k in range(n)], dtype=dt)
    return out


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")
