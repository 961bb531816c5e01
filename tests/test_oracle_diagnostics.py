"""Pins of the oracle's two diagnostics, State.flowrate and residual, against
what the mathematics fixes (they serve as checkers in the GPU parity tests).

* Flow rate along axis a is the volume flux through one cross-section normal
  to a (Secs. 4.4, 4.5: Q / L^2 = U_avg), averaged over the L_a sections:
  - a uniform plug u = U on a wall-less periodic box carries U_a times the
    section's area, L_b L_c, through every section;
  - the steady plane-Poiseuille channel with TRT Lambda = 3/16 is exactly the
    parabola (g / 2 nu)(h^2 - y^2) on every fluid row, so its flux is the
    discrete sum of that parabola over the 63 fluid rows of one x-section;
  - the steady Bingham channel carries H U_mean with the closed-form mean
    U_mean = (g h^2 / 3 nu_p)(1 - 3 xi / 2 + xi^3 / 2), xi = y_0 / h (Sec. 4.3).
* The residual sqrt(sum |u - u_prev|^2 / sum |u|^2) of 2u against u is 1/2,
  of (1 + eps) u against u is eps / (1 + eps), of u against itself 0, and
  values on solid cells do not enter.

Each pin is also run against planted mistakes (a divisor of another axis,
the fluid-cell count as divisor, a residual normalised by u_prev or missing
its square root): every planted variant must fail at least one pin.
"""
import numpy as np
import pytest

import oracle
from paper_1610_01388_gb300 import workloads as W

NY = 64
H = NY - 1
h = H / 2.0
YC = np.arange(1, NY) - NY / 2.0


# --- planted mistakes, for the pins to catch -------------------------------------

def _flow_other_axis(st, axis=0):
    _, u = st.fields()
    L = (st.ny, st.nz, st.nx)[axis]           # wrong: length of another axis
    return float(np.sum(u[axis][st.mask == 0])) / L


def _flow_per_fluid_cell(st, axis=0):
    _, u = st.fields()
    fl = st.mask == 0
    return float(np.sum(u[axis][fl])) / int(fl.sum())   # wrong: mean velocity


def _residual_by_prev(u, u_prev, fluid):
    du = (u - u_prev)[:, fluid]
    return float(np.sqrt(np.sum(du * du) / np.sum(u_prev[:, fluid] ** 2)))


def _residual_no_sqrt(u, u_prev, fluid):
    du = (u - u_prev)[:, fluid]
    return float(np.sum(du * du) / np.sum(u[:, fluid] ** 2))


def _residual_all_cells(u, u_prev, fluid):
    du = u - u_prev
    return float(np.sqrt(np.sum(du * du) / np.sum(u * u)))


def _good_flow(st, axis=0):
    return st.flowrate(axis)


# --- flow rate: uniform plug through a wall-less box ------------------------------

def _plug_box_errors(flow):
    """Largest relative error of flow(state, axis) against U_a L_b L_c, over
    the three axes of a 5 x 4 x 3 periodic box in uniform motion."""
    nz, ny, nx = 3, 4, 5
    U = np.array([2.0e-3, -1.5e-3, 7.0e-4])
    p = oracle.params(model="IR", nu_p=0.1)              # no body force: u_real = j / rho
    st = oracle.State("D3Q27", p, np.zeros((nz, ny, nx), np.uint8))
    st.f = np.ascontiguousarray(np.repeat(oracle.feq("D3Q27", 1.0, U)[:, None], st.N, axis=1))
    area = (ny * nz, nx * nz, nx * ny)
    return max(abs(flow(st, a) - U[a] * area[a]) / abs(U[a] * area[a]) for a in range(3))


def test_flowrate_uniform_plug_is_velocity_times_section():
    assert _plug_box_errors(_good_flow) < 1e-12


@pytest.mark.parametrize("planted", [_flow_other_axis, _flow_per_fluid_cell])
def test_flowrate_pin_catches_planted_divisor(planted):
    assert _plug_box_errors(planted) > 1e-2


# --- flow rate: steady channels ---------------------------------------------------

def _steady_channel(model, nu, sy, g, steps, m=0.0, magic=0.25):
    p = oracle.params(model=model, nu_p=nu, sigma_y=sy, m=m, g=(g, 0, 0), magic=magic)
    st = oracle.State("D2Q9", p, W.channel_mask(4, NY))
    st.step(steps)
    return st


@pytest.fixture(scope="module")
def poiseuille_state():
    nu = 0.1
    g = W.channel_params(H=H, nu_p=nu, u_newton=0.01, bn=0)["g"]
    return _steady_channel("PR", nu, 0.0, g, 150_000, magic=3.0 / 16.0), g, nu


@pytest.fixture(scope="module")
def bingham_state():
    nu = 0.1
    prm = W.channel_params(H=H, nu_p=nu, u_newton=0.01, bn=1.0)
    return _steady_channel("IR", nu, prm["sigma_y"], prm["g"], 300_000), prm, nu


def _poiseuille_error(flow, poiseuille_state):
    st, g, nu = poiseuille_state
    q_exact = float(np.sum(g / (2 * nu) * (h * h - YC * YC)))   # one x-section, 63 rows
    return abs(flow(st, 0) - q_exact) / q_exact


def _bingham_error(flow, bingham_state):
    st, prm, nu = bingham_state
    g, sy = prm["g"], prm["sigma_y"]
    xi = sy / g / h
    q_exact = H * g * h * h / (3 * nu) * (1 - 1.5 * xi + 0.5 * xi ** 3)
    return abs(flow(st, 0) - q_exact) / q_exact


def test_flowrate_poiseuille_channel_is_discrete_parabola_sum(poiseuille_state):
    assert _poiseuille_error(_good_flow, poiseuille_state) < 1e-10


def test_flowrate_bingham_channel_is_height_times_mean(bingham_state):
    assert _bingham_error(_good_flow, bingham_state) < 2e-3


@pytest.mark.parametrize("planted", [_flow_other_axis, _flow_per_fluid_cell])
def test_flowrate_channel_pins_catch_planted_divisor(planted, poiseuille_state, bingham_state):
    assert _poiseuille_error(planted, poiseuille_state) > 1e-2
    assert _bingham_error(planted, bingham_state) > 1e-2


# --- residual ----------------------------------------------------------------------

def _residual_errors(res):
    """Largest absolute error of res over the closed-form cases, on a field
    with solid cells that hold values which must not enter."""
    rng = np.random.default_rng(5)
    mask = W.duct_mask(4, 9, 7)
    fluid = mask == 0
    u = rng.uniform(-1e-2, 1e-2, (3,) + mask.shape)
    u[:, ~fluid] = 0.0
    junk = u.copy()
    junk[:, ~fluid] = rng.uniform(-1.0, 1.0, (3, int((~fluid).sum())))
    eps = 3.0e-4
    cases = [
        (res(2.0 * u, u, fluid), 0.5),
        (res((1.0 + eps) * u, u, fluid), eps / (1.0 + eps)),
        (res(u, u, fluid), 0.0),
        (res(2.0 * junk, junk, fluid), 0.5),
        (res(2.0 * junk, u, fluid), 0.5),
    ]
    return max(abs(got - want) for got, want in cases)


def test_residual_closed_forms():
    assert _residual_errors(oracle.residual) < 1e-15


@pytest.mark.parametrize("planted", [_residual_by_prev, _residual_no_sqrt, _residual_all_cells])
def test_residual_pin_catches_planted_mistake(planted):
    assert _residual_errors(planted) > 1e-2
