"""Conservation pins of the oracle on a coupled run with beam, absorption and SEE.

A shortened gap (0.5 mm, 64 cells) lets the 20 keV beam reach the driven
electrode within the run so that ion impacts, secondary emission, electron
loss and circuit charging all happen.  Checked at every time level:

* Gauss at x = 0 (Eq. 1D_Gaussian_app) and the global Gauss balance
  sigma_+ A + Q_space + sigma_- A = 0 with sigma_- from the field at x = d;
* the integer charge grid carries exactly 2^16 per live macroparticle;
* particle and charge ledgers: live counts change only by absorption,
  emission and injection, and circuit-delivered charge = change of the
  surface charge - convection charge (Eq. top_plate_charge), where the
  convection charge is ions + electrons absorbed at x = 0 plus the emitted
  secondaries (Eq. for Q_conv^n);
* the coupled solve's backward error stays below the requested tolerance.
"""
import numpy as np
import pytest

from paper_2603_24010_gb300 import workloads as W


def small_gap(seed=0):
    cfg = W.scaled(W.gap_1d_fp64(seed), d=5e-4, n_cells=64, n_pairs=2000, beam_per_step=8,
                   see_scale=8.0)
    cfg["area"] = cfg["C"] * cfg["d"] / cfg["eps0"]
    cfg["weight"] = cfg["n0"] * cfg["d"] * cfg["area"] / cfg["n_pairs"]
    return cfg


def run(orc, cfg, mode, steps):
    g = orc.OracleGap(cfg)
    xi, ue, ui = W.load_pairs(cfg)
    g.set_particles(orc.ELECTRONS, xi, ue)
    g.set_particles(orc.IONS, xi, ui)
    grids = []
    for _ in range(steps):
        assert g.step(mode, 1) == orc.OK
        grids.append(g.grid())
    h = g.history()
    g.close()
    return h, grids


@pytest.mark.parametrize("mode", [0, 1])
def test_conservation_on_coupled_run(orc, mode):
    cfg = small_gap()
    steps = 420
    h, grids = run(orc, cfg, mode, steps)
    N = cfg["n_cells"]
    dx = cfg["d"] / N
    A, e0 = cfg["area"], cfg["eps0"]
    qw = cfg["e"] * cfg["weight"]
    # the run exercises every path
    assert h["absorbed"][:, 0, 1].sum() > 100  # ions hit x = 0
    assert h["emitted"][:, 0].sum() > 100      # ... and emit secondaries
    assert h["absorbed"][:, :, 0].sum() > 0     # plasma electrons lost
    assert np.all(h["residual"] <= 1e-12)
    for k, gr in enumerate(grids, start=1):
        G, E = gr["G"], gr["E"]
        nl = h["n_live"][k]
        # 2^16 per live macroparticle, boundary nodes counted half
        assert G[0] // 2 + G[1:N].sum() + G[N] // 2 == 2**16 * (nl[1] - nl[0] - nl[2])
        rho = gr["rho"]
        sig_p = h["Q_surf"][k] / A
        scale = abs(sig_p) + abs(qw / A) * (nl.sum() + 1)
        # Gauss at x = 0
        assert abs(e0 * E[0] - (sig_p + dx * rho[0] / 2)) <= 1e-11 * scale
        # global Gauss balance with the grounded electrode's induced charge
        q_space = dx * (rho[0] / 2 + rho[1:N].sum() + rho[N] / 2)
        sig_m = -e0 * E[N - 1] - dx * rho[N] / 2
        assert abs(sig_p + q_space + sig_m) <= 1e-11 * scale
        assert q_space * A == pytest.approx(qw * (nl[1] - nl[0] - nl[2]), rel=1e-12, abs=1e-30)
    # particle ledger
    nl = h["n_live"]
    ab = h["absorbed"]
    np.testing.assert_array_equal(np.diff(nl[:, 0]), -ab[1:, :, 0].sum(axis=1))
    np.testing.assert_array_equal(np.diff(nl[:, 1]), -ab[1:, :, 1].sum(axis=1) + h["injected"][1:])
    np.testing.assert_array_equal(np.diff(nl[:, 2]),
                                  -ab[1:, :, 2].sum(axis=1) + h["emitted"][1:].sum(axis=1))
    # convection charge = ions - electrons absorbed at x = 0 + secondaries emitted there
    conv = ab[:, 0, 1] - ab[:, 0, 0] - ab[:, 0, 2] + h["emitted"][:, 0]
    np.testing.assert_array_equal(h["conv_count"], conv)
    # circuit-delivered charge = surface-charge change - convection charge
    # (Q_circ is the circuit's loop charge in both schemes, zero at rest)
    lhs = h["Q_circ"][-1]
    rhs = h["Q_surf"][-1] - cfg["sigma0"] * A - qw * conv.sum()
    assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-10 * abs(h["Q_surf"]).max())


def test_runs_are_deterministic(orc):
    cfg = small_gap(3)
    h1, g1 = run(orc, cfg, 0, 300)
    h2, g2 = run(orc, cfg, 0, 300)
    np.testing.assert_array_equal(h1["V_gap"], h2["V_gap"])
    np.testing.assert_array_equal(g1[-1]["G"], g2[-1]["G"])
