"""FP64 oracle of the 2D planar gap (x normal to the electrodes, y periodic).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s
reference legs; the product path never imports it.

The 2D gap extends the paper's 1D cycle (arXiv 2603.24010) in the way its
Poisson problem allows: the electrodes stay equipotential planes, the
transverse direction is periodic, and the circuit sees only the transverse
mean.  Each step follows the 1D order (push, absorption + SEE, beam,
deposit, solve) with:

* deposit: bilinear cloud-in-cell to nodes with per-axis fixed-point
  weights floor(frac 2^16) (corner products sum to 2^32 per macroparticle),
  end nodes in x doubled as in App. E.2 -- plain CIC with positions snapped
  to 2^-16 of a cell per axis, which moves the fields by far less than the
  1e-5 tolerance (tests/test_oracle_deposit_resolution.py);
* solve: the transverse mean of the charge (the integer column sums of the
  grid) is the 1D coupled problem of Sec. 2.4.2/2.4.3 with the circuit row,
  solved by the 1D oracle; the rest is expanded in transverse Fourier modes
  (numpy's FFT as the transform), each mode k != 0 solving the tridiagonal
  system of App. B's x-differences with the discrete transverse eigenvalue
  and phi = 0 on both electrodes;
* fields E_x at (i+1/2, j), E_y at (i, j+1/2); bilinear gather between them
  (half-grid in the staggered direction, clamped at the electrodes as in 1D);
* SEE: as 1D (yield from the impact's full kinetic energy), emitted
  electrons start at the impact's y with normal velocity;
* beam: ions enter at x = d with a Gaussian transverse profile, y = y_c +
  sigma z from a Box-Muller pair of the beam draw's third and fourth words.

Positions are in cell units xi = x/dx, eta = y/dy; velocities u = v_x dt/dx,
w = v_y dt/dy.
"""
import math

import numpy as np

from . import oracle as O

FIX_AXIS = 65536  # 2^16 per axis, 2^32 per macroparticle
GRID_UNITS = FIX_AXIS * FIX_AXIS


def deposit2d(Nx, Ny, xi, eta, sign, G=None):
    """int64 node grid (Nx+1, Ny): bilinear fixed-point weights."""
    if G is None:
        G = np.zeros((Nx + 1, Ny), dtype=np.int64)
    xi = np.asarray(xi, np.float64)
    eta = np.asarray(eta, np.float64)
    i = np.floor(xi).astype(np.int64)
    j = np.floor(eta).astype(np.int64)
    wx1 = np.floor((xi - i) * FIX_AXIS).astype(np.int64)
    wy1 = np.floor((eta - j) * FIX_AXIS).astype(np.int64)
    wx0, wy0 = FIX_AXIS - wx1, FIX_AXIS - wy1
    j1 = (j + 1) % Ny
    for ii, jj, w in ((i, j, wx0 * wy0), (i + 1, j, wx1 * wy0), (i, j1, wx0 * wy1),
                      (i + 1, j1, wx1 * wy1)):
        w = w * np.where((ii == 0) | (ii == Nx), 2, 1)
        np.add.at(G, (ii, jj), sign * w)
    return G


def gather2d(Ex, Ey, xi, eta):
    """E_x, E_y at the particles (Ex: (Nx, Ny) at (i+1/2, j); Ey: (Nx+1, Ny) at (i, j+1/2))."""
    Nx, Ny = Ex.shape
    xi = np.asarray(xi, np.float64)
    eta = np.asarray(eta, np.float64)
    # E_x: half-grid in x (clamped to the end values), nodes in y (periodic)
    s = xi - 0.5
    i = np.floor(s).astype(np.int64)
    t = s - i
    lo = s < 0
    hi = s >= Nx - 1
    i = np.where(lo, 0, np.where(hi, Nx - 1, i))
    t = np.where(lo | hi, 0.0, t)
    i1 = np.minimum(i + 1, Nx - 1)
    j = np.floor(eta).astype(np.int64)
    v = eta - j
    j = j % Ny
    j1 = (j + 1) % Ny
    ex = (1 - v) * ((1 - t) * Ex[i, j] + t * Ex[i1, j]) + v * ((1 - t) * Ex[i, j1] + t * Ex[i1, j1])
    # E_y: nodes in x, half-grid in y (periodic)
    a = np.floor(xi).astype(np.int64)
    fx = xi - a
    a1 = a + 1
    sy = eta - 0.5
    jj = np.floor(sy).astype(np.int64)
    vy = sy - jj
    jj = jj % Ny
    jj1 = (jj + 1) % Ny
    ey = (1 - vy) * ((1 - fx) * Ey[a, jj] + fx * Ey[a1, jj]) + vy * ((1 - fx) * Ey[a, jj1] + fx * Ey[a1, jj1])
    return ex, ey


def cfg_1d(cfg):
    """The 1D problem of the transverse mean (same gap, circuit and weight;
    its charge grid, the column sums, counts 2^32 per macroparticle)."""
    return dict(cfg, grid_units=float(GRID_UNITS))


def solve2d(cfg, mode, G, conv_count, sigma_prev, Qhist, t, phi0_prev, tol=1e-12):
    """phi (Nx+1, Ny), Ex, Ey and the 1D solve's circuit outputs."""
    Nx, Ny = G.shape[0] - 1, G.shape[1]
    dx = cfg["d"] / Nx
    dy = cfg["Ly"] / Ny
    A = cfg["area"]
    Lz = A / cfg["Ly"]
    # transverse mean: the 1D coupled problem with the integer column sums
    G1 = G.sum(axis=1)
    rc, phi0, _, out = O.solve_fields(cfg_1d(cfg), mode, G1, conv_count, sigma_prev, Qhist, t,
                                      tol=tol, phi0_prev=phi0_prev)
    # the other transverse modes, phi = 0 on both electrodes
    scale = cfg["e"] * cfg["weight"] / (dx * dy * Lz * float(GRID_UNITS))
    rho = G.astype(np.float64) * scale
    rho_t = rho - rho.mean(axis=1, keepdims=True)
    R = np.fft.fft(rho_t, axis=1)
    Phi = np.zeros_like(R)
    k = np.arange(Ny)
    kap = (dx / dy) ** 2 * (2.0 - 2.0 * np.cos(2.0 * math.pi * k / Ny))
    n = Nx - 1
    for kk in range(1, Ny):
        # (i-1) - (2 + kappa) (i) + (i+1) = -dx^2 R_i / eps0, i = 1..Nx-1, Dirichlet 0
        ab = np.zeros((3, n), dtype=np.complex128)
        ab[0, 1:] = 1.0
        ab[1, :] = -(2.0 + kap[kk])
        ab[2, :-1] = 1.0
        rhs = -dx * dx * R[1:Nx, kk] / cfg["eps0"]
        Phi[1:Nx, kk] = _banded_solve(ab, rhs)
    phi_t = np.real(np.fft.ifft(Phi, axis=1))
    phi = phi0[:, None] + phi_t
    Ex = (phi[:-1, :] - phi[1:, :]) / dx
    Ey = (phi - np.roll(phi, -1, axis=1)) / dy
    return rc, phi, Ex, Ey, out


def _banded_solve(ab, rhs):
    from scipy.linalg import solve_banded
    return solve_banded((1, 1), ab, rhs)


class Oracle2D:
    """One 2D gap advanced by the oracle (small sizes)."""

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self.Nx = int(cfg["n_cells"])
        self.Ny = int(cfg["Ny"])
        c = self.cfg
        self.dx = c["d"] / self.Nx
        self.dy = c["Ly"] / self.Ny
        dt = c["dt"]
        self.kx = {s: q * c["e"] * dt * dt / (m * self.dx) for s, q, m in
                   ((0, -1, c["m_e"]), (1, 1, c["m_i"]), (2, -1, c["m_e"]))}
        self.ky = {s: q * c["e"] * dt * dt / (m * self.dy) for s, q, m in
                   ((0, -1, c["m_e"]), (1, 1, c["m_i"]), (2, -1, c["m_e"]))}
        self.p = [dict(xi=np.zeros(0), eta=np.zeros(0), u=np.zeros(0), w=np.zeros(0))
                  for _ in range(3)]
        self.ids = np.zeros(0, dtype=np.uint64)
        self.level = 0
        self.pushed = False
        self.solved0 = False
        self.sigma = c.get("sigma0", 0.0)
        self.Qh = np.zeros(4)
        self.phi0_prev = 0.0
        self.beam_base = 0
        self.hist = []
        self.G = None
        self.phi = self.Ex = self.Ey = None

    def set_particles(self, s, xi, eta, u, w, ids=None):
        self.p[s] = dict(xi=np.array(xi, np.float64), eta=np.array(eta, np.float64),
                         u=np.array(u, np.float64), w=np.array(w, np.float64))
        if s == 1:
            n = len(xi)
            self.ids = (np.arange(n, dtype=np.uint64) if ids is None
                        else np.array(ids, dtype=np.uint64))
            self.beam_base = int(self.ids.max()) + 1 if n else 0

    def _deposit_all(self):
        G = np.zeros((self.Nx + 1, self.Ny), dtype=np.int64)
        for s, sign in ((0, -1), (1, 1), (2, -1)):
            if self.p[s]["xi"].size:
                deposit2d(self.Nx, self.Ny, self.p[s]["xi"], self.p[s]["eta"], sign, G)
        return G

    def _solve(self, mode, conv, tol, diag):
        t = self.level * self.cfg["dt"]
        rc, phi, Ex, Ey, out = solve2d(self.cfg, mode, self.G, conv, self.sigma, self.Qh, t,
                                       self.phi0_prev, tol)
        self.phi, self.Ex, self.Ey = phi, Ex, Ey
        self.sigma = out["sigma_n"]
        self.Qh = np.array([out["Q_n"], self.Qh[0], self.Qh[1], self.Qh[2]])
        self.phi0_prev = phi[0, 0]
        d = dict(diag)
        d.update(step=self.level, V_gap=phi[0, 0], I_circ=out["I"], Q_surf=out["sigma_n"] * self.cfg["area"],
                 Q_circ=out["Q_n"], residual=out["residual"],
                 Q_conv=conv * self.cfg["e"] * self.cfg["weight"], conv_count=conv,
                 n_live=[self.p[s]["xi"].size for s in range(3)])
        self.hist.append(d)
        return rc

    def step(self, mode, n_steps, tol=1e-12):
        c = self.cfg
        if not self.solved0:
            self.G = self._deposit_all()
            rc = self._solve(mode, 0, tol, dict(absorbed=np.zeros((2, 3), np.int64),
                                                emitted=[0, 0], injected=0))
            self.solved0 = True
            if rc != O.OK:
                return rc
        Nx, Ny = self.Nx, self.Ny
        for _ in range(n_steps):
            step = self.level
            absorbed = np.zeros((2, 3), np.int64)
            conv = 0
            hits = []  # (id, electrode, u, w, eta) of absorbed ions
            for s in range(3):
                q = self.p[s]
                if q["xi"].size == 0:
                    continue
                ex, ey = gather2d(self.Ex, self.Ey, q["xi"], q["eta"])
                f = 0.5 if not self.pushed else 1.0
                u = q["u"] + f * self.kx[s] * ex
                w = q["w"] + f * self.ky[s] * ey
                xi = q["xi"] + u
                eta = q["eta"] + w
                eta = np.where(eta < 0, eta + Ny, eta)
                eta = np.where(eta >= Ny, eta - Ny, eta)  # (a tiny negative value + Ny rounds to Ny)
                far = ~((eta >= 0) & (eta < Ny))  # more than one period in a step
                eta = np.where(far, eta - Ny * np.floor(eta / Ny), eta)
                eta = np.where((eta >= 0) & (eta < Ny), eta, 0.0)
                gone0 = xi <= 0
                gone1 = ~(xi > 0) | ~(xi < Nx)
                gone1 = gone1 & ~gone0
                absorbed[0, s] = int(gone0.sum())
                absorbed[1, s] = int(gone1.sum())
                if s == 1:
                    for el, m in ((0, gone0), (1, gone1)):
                        for k in np.nonzero(m)[0]:
                            hits.append((int(self.ids[k]), el, u[k], w[k], eta[k]))
                keep = ~(gone0 | gone1)
                self.p[s] = dict(xi=xi[keep], eta=eta[keep], u=u[keep], w=w[keep])
                if s == 1:
                    self.ids = self.ids[keep]
            self.pushed = True
            conv = int(absorbed[0, 1] - absorbed[0, 0] - absorbed[0, 2])
            # secondary emission (Sec. 2.3), normal to the electrode
            emitted = [0, 0]
            se = dict(xi=[], eta=[], u=[], w=[])
            energy_q = 0
            for ion, el, u, w, eta in hits:
                vx = u * self.dx / c["dt"]
                vy = w * self.dy / c["dt"]
                E_eV = 0.5 * c["m_i"] * (vx * vx + vy * vy) / c["e"]
                nse, _ = O.see_count(c, E_eV, ion, step)
                if el == 0:
                    energy_q += int(round(E_eV * 256.0))
                    conv += nse
                emitted[el] += nse
                for jn in range(nse):
                    v, frac = O.see_electron(c, ion, step, jn)
                    use = v * c["dt"] / self.dx
                    x = use * frac if el == 0 else Nx - use * frac
                    x = min(max(x, np.nextafter(0.0, 1.0)), np.nextafter(float(Nx), 0.0))
                    se["xi"].append(x)
                    se["eta"].append(eta)
                    se["u"].append(use if el == 0 else -use)
                    se["w"].append(0.0)
            q = self.p[2]
            self.p[2] = {k: np.concatenate([q[k], np.array(se[k], np.float64)]) for k in q}
            # beam ions entering at x = d with a Gaussian transverse profile
            B = int(c["beam_per_step"])
            if B:
                xs, us, es, ids = [], [], [], []
                for k in range(B):
                    wv = O.philox4x64_10([k, step, 0, 0], [c["seed"], O.TAG_BEAM])
                    frac = O.u01(wv[0])
                    Eb = c["beam_E_eV"] if c["beam_mode"] == 0 else (
                        c["beam_Emin_eV"] + (c["beam_Emax_eV"] - c["beam_Emin_eV"]) * O.u01(wv[1]))
                    ub = math.sqrt(2.0 * Eb * c["e"] / c["m_i"]) * c["dt"] / self.dx
                    z = math.sqrt(-2.0 * math.log(O.u01(wv[2]))) * math.cos(2.0 * math.pi * O.u01(wv[3]))
                    y = (c["beam_yc"] + c["beam_sigma"] * z) / self.dy
                    y = y - Ny * math.floor(y / Ny)
                    if y >= Ny:
                        y = 0.0
                    x = min(max(Nx - ub * frac, np.nextafter(0.0, 1.0)), np.nextafter(float(Nx), 0.0))
                    xs.append(x)
                    us.append(-ub)
                    es.append(y)
                    ids.append(self.beam_base + step * B + k)
                q = self.p[1]
                self.p[1] = dict(xi=np.concatenate([q["xi"], xs]), eta=np.concatenate([q["eta"], es]),
                                 u=np.concatenate([q["u"], us]), w=np.concatenate([q["w"], np.zeros(B)]))
                self.ids = np.concatenate([self.ids, np.array(ids, dtype=np.uint64)])
            self.G = self._deposit_all()
            self.level += 1
            rc = self._solve(mode, conv, tol, dict(absorbed=absorbed, emitted=emitted, injected=B,
                                                   ion_energy_eV=energy_q / 256.0))
            if rc != O.OK:
                return rc
        return O.OK

    def history(self):
        keys = ("V_gap", "I_circ", "Q_surf", "Q_circ", "Q_conv", "residual", "conv_count")
        out = {k: np.array([h[k] for h in self.hist]) for k in keys}
        out["n_live"] = np.array([h["n_live"] for h in self.hist], dtype=np.int64)
        out["absorbed"] = np.array([h["absorbed"] for h in self.hist], dtype=np.int64)
        out["emitted"] = np.array([h["emitted"] for h in self.hist], dtype=np.int64)
        return out
