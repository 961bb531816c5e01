"""Physics pins of the CUDA path against numbers the paper prints.

* Square duct, Bingham, Hg = 432, Bi = 0.4, 63 lu (Secs. 4.3.1-4.3.2): the
  spectral reference gives Re = U_max D / nu_p = 12.6242614; the paper's own
  LBM approaches it to ~1e-3 at high resolution.  Parameters follow the
  paper's scaling: nu = 0.0125, g = 2e-5 (15/63)^3, sigma_y = 3e-5 (15/63)^2.
* Creeping flow past a periodic cylinder array, 80 x 80, D = 32, g = 1.25e-6,
  nu_p = 0.08 (Sec. 4.5.2, Table ParticleCreep): Re, Bn and f for IR and PR,
  within 1 % (the staircase of the cylinder is not specified in the paper).
Values are read from tests/golden/paper_values.json.
"""
import json
import os

import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _run_to_steady(s, chunk, max_steps, rtol, probe):
    prev = probe(s)
    steps = 0
    while steps < max_steps:
        s.step(chunk)
        steps += chunk
        cur = probe(s)
        if abs(cur - prev) <= rtol * abs(cur):
            return cur, steps
        prev = cur
    return prev, steps


def _umax(s):
    _, u = s.fields()
    return float(u[0].max())


@pytest.mark.parametrize("model,storage", [("IR", "F64"), ("PR", "F64"), ("IR", "F32")])
def test_square_duct_spectral_reference(model, storage):
    ref = GOLD["square_duct_spectral"]
    sc = GOLD["duct_convergence_scaling"]
    D = 63
    nu = sc["nu"]
    g = sc["g0"] * (sc["D0"] / D) ** 3
    sy = sc["sigma_y0"] * (sc["D0"] / D) ** 2
    assert abs(g * D ** 3 / nu ** 2 - ref["Hg"]) < 1e-9 * ref["Hg"]
    assert abs(4 * sy / (g * D) - ref["Bi"]) < 1e-12
    s = lbm.Solver("D3Q27", W.duct_mask(1, D + 1, D + 1), model=model, storage=storage,
                   mu_p=nu, sigma_y=sy, m=1e8, g=(g, 0, 0))
    umax, steps = _run_to_steady(s, 50_000, 2_000_000, 1e-6, _umax)
    re = umax * D / nu
    err = abs(re - ref["Re"]) / ref["Re"]
    print(f"duct {model} {storage}: Re {re:.6f} vs spectral {ref['Re']} (rel {err:.2e}) after {steps} steps")
    assert err < 5e-3
    s.close()


@pytest.mark.parametrize("model", ["IR", "PR"])
def test_creeping_cylinder_array_table(model):
    tab = GOLD["creeping_cylinders"]
    L, D, g, nu = tab["L"], tab["D"], tab["g"], tab["nu_p"]
    mask = W.cylinder_mask(L, D)
    nfluid = int((mask == 0).sum())
    assert abs(1 - nfluid / mask.size - 0.1257) < 2e-3      # solid fraction of Sec. 4.5
    for row in tab["rows"]:
        # The printed sigma_y column is 10x smaller than what the table's own
        # Re and Bn columns imply: Bn nu_p U_avg / D = Bn nu_p^2 Re / D^2 gives
        # 1.0e-5, 1.5e-5, 2.0e-5 for the three yield rows (the inertial table's
        # sigma_y, by contrast, is consistent with its Bn).  Reading: the yield
        # stresses are 1e-5, 1.5e-5, 2e-5.
        sy = 10.0 * row["sigma_y"]
        if sy > 0:
            implied = row["IR"]["Bn"] * nu ** 2 * row["IR"]["Re"] / D ** 2
            assert abs(implied - sy) / sy < 0.01
        s = lbm.Solver("D2Q9", mask, model=model, storage="F64", mu_p=nu, sigma_y=sy, m=1e8,
                       g=(g, 0, 0))
        q, steps = _run_to_steady(s, 20_000, 600_000, 1e-7, lambda x: x.flowrate(0))
        # U_avg read as the mean velocity over the fluid cells (the paper's
        # u_bulk of Sec. 4.5.1, superficial velocity / (1 - phi)); the flow
        # rate is sum(u_x) / L_x, so U_avg = flow rate * L_x / N_fluid
        u_avg = q * L / nfluid
        re = u_avg * D / nu
        bn = sy * D / (nu * u_avg)
        f = 2 * D * g / u_avg ** 2
        want = row[model]
        print(f"cylinders {model} sigma_y={sy:g}: Re {re:.4f} ({want['Re']}), Bn {bn:.4f} "
              f"({want['Bn']}), f {f:.3f} ({want['f']}) after {steps} steps")
        # measured agreement is 0.03-0.4 %; the bar leaves room for the
        # unspecified staircase of the cylinder
        assert abs(re - want["Re"]) / want["Re"] < 0.01
        assert abs(f - want["f"]) / want["f"] < 0.01
        if sy > 0:
            assert abs(bn - want["Bn"]) / want["Bn"] < 0.01
        s.close()


def _duct63(model, m=1e8, storage="F64", flags=0, gammadot_c=1e-8):
    sc = GOLD["duct_convergence_scaling"]
    D = 63
    g = sc["g0"] * (sc["D0"] / D) ** 3           # 2.70e-7
    sy = sc["sigma_y0"] * (sc["D0"] / D) ** 2    # 1.70e-6
    return lbm.Solver("D3Q27", W.duct_mask(1, D + 1, D + 1), model=model, storage=storage,
                      mu_p=sc["nu"], sigma_y=sy, m=m, g=(g, 0, 0), flags=flags,
                      gammadot_c=gammadot_c), sy


def test_pr_m_sweep_and_apparent_viscosity():
    """Sec. 4.2.1, Table Rel_error_m: relative U_max error of PR against
    m = 1e14 in the 63 lu square duct (1.37, 1.03e-2, 8.5e-6, 0 for m = 1e3,
    1e6, 1e9, 1e12); the apparent viscosity saturates far below the limit
    nu_p + m sigma_y at large m because of the Burnett d_xx (the paper reads
    ~727), and reaches the limit when d_xx is set to zero.

    The saturation value sigma_y / nu_app ~ 2e-9 is below the printed cut-off
    gdot^C = 1e-8, where a linear interpolation towards nu_0 would stiffen the
    flow (measured: U_max at m = 1e9 drops to 0.64 of its m = 1e6 value and the
    fluid does not yield from rest at m >= 1e12).  The paper's table is
    reproduced with the cut-off below the strain rates of the flow
    (gdot^C = 1e-20), which is how it is pinned here."""
    rows = GOLD["pr_m_sweep_relative_error"]["rows"]
    umax = {}
    nu_max = {}
    for m in (1e3, 1e6, 1e9, 1e12, 1e14):
        s, sy = _duct63("PR", m=m, gammadot_c=1e-20)
        umax[m], steps = _run_to_steady(s, 50_000, 1_500_000, 1e-11, _umax)
        tau = s.get_tau()[s.mask == 0]
        nu_max[m] = (tau.max() - 0.5) / 3.0
        print(f"PR m={m:g}: U_max {umax[m]:.10e}, max nu_app {nu_max[m]:.4g} "
              f"(limit {0.0125 + m * sy:.4g}) after {steps} steps")
        s.close()
    ref = umax[1e14]
    got = {m: abs(umax[m] - ref) / ref for m in umax}
    for m, want in rows:
        print(f"  m={m:g}: rel err {got[m]:.3e} (paper {want:g})")
    # measured: 1.248, 5.3e-3, 5.7e-7, 1.7e-15
    assert abs(got[1e3] - 1.37) / 1.37 < 0.15
    assert 0.4 * 1.03e-2 < got[1e6] < 2.5 * 1.03e-2
    assert got[1e9] < 8.5e-6
    assert got[1e12] < 1e-12
    # saturation (measured ~594 for m >= 1e12; the paper reads ~727)
    assert nu_max[1e12] < 1e-3 * (0.0125 + 1e12 * 1.7e-6)
    assert abs(nu_max[1e14] - nu_max[1e12]) < 0.01 * nu_max[1e12]
    assert 727 / 1.5 < nu_max[1e12] < 727 * 1.5
    # the large-m velocity is the Bingham one: Re near the spectral 12.6242614
    re = umax[1e14] * 63 / 0.0125
    assert abs(re - GOLD["square_duct_spectral"]["Re"]) / GOLD["square_duct_spectral"]["Re"] < 2e-3
    s, sy = _duct63("PR", m=1e9, flags=lbm.LBM_FLAG_BURNETT_X, gammadot_c=1e-20)
    _run_to_steady(s, 50_000, 1_500_000, 1e-10, _umax)
    nu_flag = (s.get_tau()[s.mask == 0].max() - 0.5) / 3.0
    print(f"PR m=1e9 with d_xx = 0: max nu_app {nu_flag:.6g} (limit {0.0125 + 1e9 * sy:.6g})")
    assert abs(nu_flag - (0.0125 + 1e9 * sy)) < 1e-3 * (0.0125 + 1e9 * sy)
    s.close()


def test_ir_transverse_currents_vanish_without_burnett_term():
    """Sec. 4.2.2: IR's deviatoric projection redistributes the Burnett T_xx
    and drives small transverse currents in a Bingham duct; with T_xx = 0
    they vanish and U_max changes only by O(1e-7) relative."""
    res = {}
    for flags in (0, lbm.LBM_FLAG_BURNETT_X):
        s, _ = _duct63("IR", flags=flags)
        u, _ = _run_to_steady(s, 50_000, 1_500_000, 1e-10, _umax)
        _, vel = s.fields()
        res[flags] = (u, np.max(np.abs(vel[1:])))
        s.close()
    (u0, t0), (u1, t1) = res[0], res[lbm.LBM_FLAG_BURNETT_X]
    print(f"IR transverse max {t0:.3e} (with Burnett term) vs {t1:.3e} (T_xx = 0); "
          f"U_max rel diff {abs(u0 - u1) / u1:.2e}")
    assert t0 > 1e-4 * u0 * 1e-3          # present
    assert t1 < 1e-6 * t0 + 1e-18         # gone
    assert abs(u0 - u1) / u1 < 1e-5


def _gpu_startup_stats(model, lat, m, storage="F32", steps=100):
    # the 63-lu duct of Sec. 4.3.3 at the stated scaling (reading 14)
    s = lbm.Solver(lat, W.duct_mask(2, 64, 64), model=model, storage=storage, mu_p=0.0125,
                   sigma_y=3e-5 * (15.0 / 63.0) ** 2, m=m, g=(2e-5 * (15.0 / 63.0) ** 3, 0.0, 0.0))
    d = np.arange(1, 33)
    wiggle, lowest = 0.0, np.inf
    for t in range(1, steps + 1):
        s.step(1)
        if t < 15:
            continue
        _, u = s.fields()
        ux = u[0][d, d, 0]
        inc = np.diff(ux)
        wiggle = max(wiggle, -inc[inc < 0].sum() / ux.max())
        lowest = min(lowest, ux.min() / ux.max())
    s.close()
    return wiggle, lowest


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_startup_transient_pr_fluctuates_ir_damps(lat):
    """Sec. 4.3.3 on the GPU (FP32): in the impulsively started 63-lu duct,
    PR (m = 1e8) reverses the flow locally within the first 100 steps and its
    diagonal profile fluctuates more than 1.5 times as much as IR's, which
    keeps the flow direction (the oracle's figures: 54 % against 31-33 %)."""
    w_pr, low_pr = _gpu_startup_stats("PR", lat, 1e8)
    w_ir, low_ir = _gpu_startup_stats("IR", lat, 0.0)
    assert low_pr < 0.0 < low_ir
    assert w_pr > 1.5 * w_ir


@pytest.mark.parametrize("model,nu,magic,flags", [("PR", 0.1, 3.0 / 16.0, 0),
                                                  ("IR", 0.125, 0.25, lbm.LBM_FLAG_BURNETT_X)])
def test_lattice_choice_transverse_currents(model, nu, magic, flags):
    """Sec. 4.1 on the GPU (FP64): in a Newtonian square duct driven along x,
    D3Q19 shows spurious transverse velocities (its lattice lacks the
    isotropy the cross-section needs) while D3Q27 shows none.  IR runs with
    T_xx = 0: with the Burnett term its deviatoric projection drives
    transverse currents of its own on either lattice (Sec. 4.2.2; 1.5e-7 of
    U_max on D3Q27 here), which would hide the lattice's.  Both lattices are
    also held to the oracle at equal step count, transverse part included."""
    import oracle
    n, g, steps = 24, 1e-5, 8000
    mask = W.duct_mask(2, n, n)
    out = {}
    for lat in ("D3Q19", "D3Q27"):
        s = lbm.Solver(lat, mask, model=model, storage="F64", mu_p=nu, g=(g, 0.0, 0.0),
                       magic=magic, flags=flags)
        s.step(steps)
        _, u = s.fields()
        s.close()
        o = oracle.State(lat, oracle.params(model=model, nu_p=nu, g=(g, 0, 0), magic=magic,
                                            burnett_x=bool(flags)), mask)
        o.step(steps)
        _, uo = o.fields()
        umax = np.max(np.abs(uo[0]))
        assert np.max(np.abs(u - uo)) <= 1e-10 * umax
        out[lat] = np.max(np.abs(u[1:])) / np.max(np.abs(u[0]))
    print(f"{model}: transverse / U_max  D3Q19 {out['D3Q19']:.2e}  D3Q27 {out['D3Q27']:.2e}")
    assert out["D3Q19"] > 1e-7
    assert out["D3Q27"] < 1e-11
