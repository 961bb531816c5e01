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
