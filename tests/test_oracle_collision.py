"""Single-cell pins of the oracle's PR and IR collisions.

Each check is a relation the paper states (or that follows from its
definitions) rather than a copy of the oracle's formula:

* collision invariants: mass conserved, momentum gains F = rho g per step
  (Sec. 2.4 body-force schemes);
* EDM, eq. (14): an equilibrium state with force relaxes to f_eq(u + du);
* IR: the closed form solves eq. (Vikh_main_short) 1/2 s + T = -sigma; in the
  yielded branch it obeys the Bingham law in s-form, eq. (sigma_vs_s); s and
  sigma are continuous across the yield switch; the post-collision
  non-equilibrium second moment is -sigma_bar + s/2 (eqs. Vikh_postCol,
  Vikh_f_stress, reading R4), and for sigma_y = 0 it is BGK's (eqs. Vikh_4/5);
* PR: the strain rate of a Chapman-Enskog population with prescribed D is
  recovered (eq. LBM_strain_rate); nu_app has the limits of Sec. 3.1; tau_new
  follows eq. (tau_visc); the odd relaxation time satisfies the magic-number
  definition Lambda = (1/2 - tau_odd)(1/2 - tau_even) (Sec. 2.1).
"""
import numpy as np
import pytest

import oracle

LATS = ["D2Q9", "D3Q15", "D3Q19", "D3Q27"]
DIMS = {"D2Q9": 2, "D3Q15": 3, "D3Q19": 3, "D3Q27": 3}


def _rand_state(lat, rng, amp=2e-3, rho=None, u=None):
    c, w, _ = oracle.lattice_info(lat)
    D = DIMS[lat]
    if rho is None:
        rho = 1.0 + 0.05 * (rng.random() - 0.5)
    if u is None:
        u = np.zeros(3)
        u[:D] = 0.05 * (rng.random(D) - 0.5)
    f = oracle.feq(lat, rho, u) + amp * w * (rng.random(len(w)) - 0.5)
    return f


def _g(lat, rng, scale=1e-5):
    g = np.zeros(3)
    g[:DIMS[lat]] = scale * (rng.random(DIMS[lat]) - 0.5)
    return g


def _mom2(lat, f):
    c, _, _ = oracle.lattice_info(lat)
    cf = c.astype(np.float64)
    return np.einsum("ia,ib,i->ab", cf, cf, f)


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_mass_and_momentum_gain(lat, model):
    rng = np.random.default_rng(11)
    c, w, _ = oracle.lattice_info(lat)
    for k in range(8):
        g = _g(lat, rng)
        p = oracle.params(model=model, nu_p=0.05 + 0.2 * rng.random(), sigma_y=1e-4 * rng.random(),
                          m=1e5, g=g)
        f = _rand_state(lat, rng)
        fo, _, _ = oracle.collide(lat, p, f, tau_old=0.5 + 3 * 0.1)
        rho = f.sum()
        assert abs(fo.sum() - rho) < 1e-14
        j = c.T.astype(np.float64) @ f
        jo = c.T.astype(np.float64) @ fo
        assert np.allclose(jo, j + rho * g, atol=1e-15, rtol=0)


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_equilibrium_fixed_point(lat, model):
    rng = np.random.default_rng(5)
    D = DIMS[lat]
    u = np.zeros(3)
    u[:D] = [0.03, -0.02, 0.01][:D]
    f = oracle.feq(lat, 1.02, u)
    p = oracle.params(model=model, nu_p=0.1, sigma_y=1e-3, m=1e4)
    fo, _, d = oracle.collide(lat, p, f, tau_old=0.8)
    assert np.max(np.abs(fo - f)) < 1e-15
    assert np.max(np.abs(d["T"])) < 1e-15


@pytest.mark.parametrize("lat", LATS)
def test_edm_equilibrium_shift(lat):
    """eq. (14) on an equilibrium state: f_eq(u) -> f_eq(u + g)."""
    D = DIMS[lat]
    u = np.zeros(3)
    u[:D] = [0.02, 0.01, -0.015][:D]
    g = np.zeros(3)
    g[:D] = [3e-4, -1e-4, 2e-4][:D]
    p = oracle.params(model="PR", nu_p=0.1, sigma_y=1e-4, m=1e3, g=g)
    fo, _, _ = oracle.collide(lat, p, oracle.feq(lat, 1.1, u), tau_old=0.9)
    assert np.allclose(fo, oracle.feq(lat, 1.1, u + g), atol=1e-15, rtol=0)


@pytest.mark.parametrize("lat", LATS)
def test_ir_implicit_relation_both_branches(lat):
    """eq. (Vikh_main_short): s/2 + T = -sigma in both regimes, and in the
    yielded one sigma = (3 nu_p + sqrt2 sigma_y / |s|) s (eq. sigma_vs_s)."""
    rng = np.random.default_rng(7)
    seen = set()
    for k in range(40):
        nu = 0.01 + 0.3 * rng.random()
        f = _rand_state(lat, rng, amp=4e-3)
        T0 = np.linalg.norm(oracle.collide(lat, oracle.params(model="IR", nu_p=nu), f)[2]["T"])
        sy = T0 / np.sqrt(2.0) * (0.2 + 1.6 * rng.random())   # either side of the switch
        p = oracle.params(model="IR", nu_p=nu, sigma_y=sy, g=_g(lat, rng))
        _, _, d = oracle.collide(lat, p, f)
        T, s, sig = d["T"], d["s"], d["sigma"]
        assert np.allclose(0.5 * s + T, -sig, atol=2e-16, rtol=0)
        seen.add(d["yielded"])
        if d["yielded"]:
            sn = np.sqrt(np.sum(s * s))
            assert np.allclose(sig, (3 * nu + np.sqrt(2) * sy / sn) * s, rtol=1e-12, atol=1e-18)
            # s points against T and has a positive magnitude
            assert np.sum(s * T) < 0
        else:
            assert np.all(s == 0)
    assert seen == {True, False}


def test_ir_continuity_at_yield_switch():
    lat = "D3Q27"
    rng = np.random.default_rng(2)
    f = _rand_state(lat, rng, amp=4e-3)
    nu = 0.1
    T0 = np.linalg.norm(oracle.collide(lat, oracle.params(model="IR", nu_p=nu), f)[2]["T"])
    outs = []
    for eps in (-1e-9, 1e-9):
        p = oracle.params(model="IR", nu_p=nu, sigma_y=T0 / np.sqrt(2.0) * (1 + eps))
        fo, _, d = oracle.collide(lat, p, f)
        outs.append((fo, d))
    (fa, da), (fb, db) = outs
    assert da["yielded"] != db["yielded"]
    # |s| = (|T| - sqrt2 sigma_y) / (1/2 + 3 nu) is ~1e-9 |T| on the yielded side
    assert np.max(np.abs(da["s"] - db["s"])) < 2e-9 * T0
    assert np.max(np.abs(da["sigma"] - db["sigma"])) < 1e-8 * T0
    assert np.max(np.abs(fa - fb)) < 1e-8 * T0


@pytest.mark.parametrize("lat", LATS)
def test_ir_post_collision_second_moment(lat):
    """Second moment of f_pc - f_eq(rho, u) is A = -sigma_bar + s/2; for the
    unyielded branch (s = 0) this is the deviatoric part of T."""
    rng = np.random.default_rng(13)
    D = DIMS[lat]
    for sy in (0.0, 1.0):   # 1.0 = always unyielded for these small T
        p = oracle.params(model="IR", nu_p=0.07, sigma_y=sy, g=_g(lat, rng))
        f = _rand_state(lat, rng)
        fo, _, d = oracle.collide(lat, p, f)
        feq = oracle.feq(lat, d["rho"], d["u"])
        M = _mom2(lat, fo - feq)
        sig = d["sigma"]
        sbar = sig.copy()
        tr = np.trace(sig[:D, :D])
        for a in range(D):
            sbar[a, a] -= tr / D
        assert np.allclose(M, -sbar + 0.5 * d["s"], atol=2e-16, rtol=0)
        if sy == 1.0:
            T = d["T"]
            Tbar = T.copy()
            trT = np.trace(T[:D, :D])
            for a in range(D):
                Tbar[a, a] -= trT / D
            assert not d["yielded"]
            assert np.allclose(M, Tbar, atol=2e-16, rtol=0)


@pytest.mark.parametrize("lat", LATS)
def test_ir_newtonian_limit_is_bgk(lat):
    """eqs. (Vikh_4), (Vikh_5): with sigma_y = 0 the deviatoric part of the
    post-collision non-equilibrium second moment equals BGK's (1 - 1/tau) T
    with tau = 1/2 + 3 nu (eq. tau_visc)."""
    rng = np.random.default_rng(17)
    D = DIMS[lat]
    for nu in (0.01, 0.1, 0.5):
        f = _rand_state(lat, rng)
        p = oracle.params(model="IR", nu_p=nu, sigma_y=0.0)
        fo, _, d = oracle.collide(lat, p, f)
        tau = 0.5 + 3 * nu
        M = _mom2(lat, fo - oracle.feq(lat, d["rho"], d["u"]))
        bgk = (1 - 1 / tau) * d["T"]

        def dev(X):
            Y = X.copy()
            t = np.trace(X[:D, :D])
            for a in range(D):
                Y[a, a] -= t / D
            return Y
        assert np.allclose(dev(M), dev(bgk), atol=2e-16, rtol=0)
        # off-diagonal components are exactly BGK's
        for a in range(D):
            for b in range(D):
                if a != b:
                    assert abs(M[a, b] - bgk[a, b]) < 2e-16


@pytest.mark.parametrize("lat", LATS)
def test_pr_strain_rate_of_chapman_enskog_state(lat):
    """f = f_eq + f^(1) with f^(1)_i = -(tau rho w_i / c_s^2)(c_i c_i - c_s^2 I):D
    has sum c c f^(1) = -2 tau rho c_s^2 D, so eq. (LBM_strain_rate) returns D
    and gdot = sqrt(2 D:D) (eq. strainInvariant)."""
    c, w, _ = oracle.lattice_info(lat)
    D = DIMS[lat]
    rng = np.random.default_rng(23)
    cf = c.astype(np.float64)
    for tau in (0.6, 1.0, 3.0):
        Dm = np.zeros((3, 3))
        X = 1e-4 * (rng.random((D, D)) - 0.5)
        Dm[:D, :D] = X + X.T
        Dm[:D, :D] -= np.trace(Dm[:D, :D]) / D * np.eye(D)   # incompressible
        h = np.einsum("ia,ib,ab->i", cf, cf, Dm) - np.trace(Dm) / 3.0
        f = oracle.feq(lat, 1.0, [0, 0, 0]) - tau * w * h / (1.0 / 3.0)
        p = oracle.params(model="PR", nu_p=0.1, sigma_y=0.0, m=0.0)
        _, _, d = oracle.collide(lat, p, f, tau_old=tau)
        assert abs(d["gdot"] - np.sqrt(2 * np.sum(Dm * Dm))) < 1e-12 * np.sqrt(np.sum(Dm * Dm))


def test_pr_apparent_viscosity_limits():
    """Sec. 3.1: nu_app -> nu_0 = nu_p + m sigma_y / rho as gdot -> 0; the cut-off
    interpolation is continuous at gdot^C; for m gdot >> 1 nu_app is the
    Bingham nu_p + sigma_y/(rho gdot) (eq. muApparent); m = 0 is Newtonian."""
    nu, sy, m, gc = 0.1, 2e-6, 1e8, 1e-8
    p = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=m, gdot_c=gc)
    for rho in (1.0, 1.05):
        nu0 = nu + m * sy / rho
        assert abs(oracle.pr_nu_app(p, 0.0, rho) - nu0) < 1e-12 * nu0
        a = oracle.pr_nu_app(p, gc * (1 - 1e-12), rho)
        b = oracle.pr_nu_app(p, gc, rho)
        assert abs(a - b) < 1e-9 * b
        # below the cut-off the map is linear in gdot
        x1, x2, x3 = 0.2 * gc, 0.5 * gc, 0.8 * gc
        y1, y2, y3 = (oracle.pr_nu_app(p, x, rho) for x in (x1, x2, x3))
        assert abs((y2 - y1) / (x2 - x1) - (y3 - y2) / (x3 - x2)) < 1e-6 * abs((y2 - y1) / (x2 - x1))
        gd = 1e-3   # m gdot = 1e5
        assert abs(oracle.pr_nu_app(p, gd, rho) - (nu + sy / (rho * gd))) < 1e-14
        # small m gdot but above cut-off: regularised value tends to nu_0
        p2 = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=1e4, gdot_c=gc)
        v = oracle.pr_nu_app(p2, 1e-7, rho)
        assert abs(v - (nu + 1e4 * sy / rho)) < 1e-3 * (1e4 * sy / rho)
    p0 = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=0.0, gdot_c=gc)
    for gd in (0.0, 1e-9, 1e-3):
        assert oracle.pr_nu_app(p0, gd) == nu


@pytest.mark.parametrize("lat", LATS)
def test_pr_trt_relaxation_rates(lat):
    """With g = 0 and a non-equilibrium part of zero mass and momentum, the even
    part of f - f_eq decays by 1 - 1/tau_new with tau_new = 1/2 + nu_app / c_s^2
    (eq. tau_visc), and the odd part by 1 - 1/tau_odd where
    (1/2 - tau_odd)(1/2 - tau_new) = Lambda (Sec. 2.1)."""
    c, w, opp = oracle.lattice_info(lat)
    rng = np.random.default_rng(29)
    cf = c.astype(np.float64)
    Q = len(w)
    for lam in (0.25, 3.0 / 16.0):
        n = 1e-4 * w * (rng.random(Q) - 0.5)
        # project out mass and momentum so f_eq is unchanged
        B = np.vstack([np.ones(Q), cf.T])
        n = n - B.T @ np.linalg.lstsq(B @ B.T, B @ n, rcond=None)[0]
        f = w + n
        p = oracle.params(model="PR", nu_p=0.05, sigma_y=3e-6, m=1e5, magic=lam)
        fo, tnew, d = oracle.collide(lat, p, f, tau_old=0.9)
        assert abs(tnew - (0.5 + 3 * d["nu_app"])) < 1e-15 * tnew
        ne, no = 0.5 * (n + n[opp]), 0.5 * (n - n[opp])
        de, do = 0.5 * ((fo - w) + (fo - w)[opp]), 0.5 * ((fo - w) - (fo - w)[opp])
        k = np.argmax(np.abs(ne))
        assert np.allclose(de, (1 - 1 / tnew) * ne, atol=1e-16, rtol=1e-9)
        k = np.argmax(np.abs(no))
        todd = 1.0 / (1.0 - do[k] / no[k])
        assert np.allclose(do, (1 - 1 / todd) * no, atol=1e-16, rtol=1e-8)
        assert abs((0.5 - todd) * (0.5 - tnew) - lam) < 1e-8


def test_pr_uses_previous_tau_for_strain_rate():
    """Sec. 3: the strain rate comes from the previous step's tau, so doubling
    tau_old halves gdot for the same populations."""
    lat = "D3Q19"
    rng = np.random.default_rng(31)
    f = _rand_state(lat, rng)
    p = oracle.params(model="PR", nu_p=0.1, sigma_y=1e-5, m=1e4)
    g1 = oracle.collide(lat, p, f, tau_old=0.8)[2]["gdot"]
    g2 = oracle.collide(lat, p, f, tau_old=1.6)[2]["gdot"]
    assert abs(g1 - 2 * g2) < 1e-12 * g1


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_burnett_suppressed_variant_drops_xx(lat):
    """Secs. 4.2.1-4.2.2: with d_xx = 0 (PR) / T_xx = 0 (IR), a unidirectional
    shear D_xy plus any xx non-equilibrium perturbation gives the strain rate
    of the shear alone, and the IR stress has no xx component."""
    c, w, _ = oracle.lattice_info(lat)
    cf = c.astype(np.float64)
    tau = 0.9
    Dm = np.zeros((3, 3))
    Dm[0, 1] = Dm[1, 0] = 3e-5
    h = np.einsum("ia,ib,ab->i", cf, cf, Dm) - np.trace(Dm) / 3.0
    pert = 1e-5 * w * (cf[:, 0] ** 2 - 1.0 / 3.0)          # an xx-only second moment
    f = oracle.feq(lat, 1.0, [0, 0, 0]) - tau * w * h * 3.0 + pert
    shear = np.sqrt(2 * np.sum(Dm * Dm))
    pr_on = oracle.params(model="PR", nu_p=0.1, sigma_y=1e-6, m=1e6, burnett_x=True)
    pr_off = oracle.params(model="PR", nu_p=0.1, sigma_y=1e-6, m=1e6)
    g_on = oracle.collide(lat, pr_on, f, tau_old=tau)[2]["gdot"]
    g_off = oracle.collide(lat, pr_off, f, tau_old=tau)[2]["gdot"]
    assert abs(g_on - shear) < 1e-12 * shear
    assert g_off > shear * (1 + 1e-3)
    ir_on = oracle.params(model="IR", nu_p=0.1, sigma_y=1e-9, burnett_x=True)
    d = oracle.collide(lat, ir_on, f)[2]
    assert d["T"][0, 0] == 0.0 and d["sigma"][0, 0] == 0.0


def _ce_state(lat, D_target, tau, rho=1.0):
    """Chapman-Enskog population with strain rate D_target at relaxation time
    tau: sum c c f^(1) = -2 tau rho c_s^2 D (see the strain-rate pin above)."""
    c, w, _ = oracle.lattice_info(lat)
    cf = c.astype(np.float64)
    h = np.einsum("ia,ib,ab->i", cf, cf, D_target) - np.trace(D_target) / 3.0
    return oracle.feq(lat, rho, [0, 0, 0]) - tau * rho * w * h / (1.0 / 3.0)


def _shear(gdot):
    """Simple shear D_xy = D_yx with sqrt(2 D:D) = gdot."""
    Dm = np.zeros((3, 3))
    Dm[0, 1] = Dm[1, 0] = gdot / 2.0
    return Dm


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("m,sy,gdot", [
    (1e4, 1e-5, 3e-3),     # yielded, m gdot = 30
    (1e6, 1e-6, 2e-6),     # transition, m gdot = 2
    (1e8, 1e-5, 1e-3),     # strongly regularised, stiff in tau
    (1e6, 1e-6, 5e-9),     # below the cut-off gdot_C = 1e-8 (linear branch)
])
def test_pr_newton_recovers_consistent_tau(lat, m, sy, gdot):
    """Sec. 3, implicit update: for a Chapman-Enskog state built with strain
    rate gdot at tau* = 1/2 + nu_app(gdot)/c_s^2 (eqs. Pap_reg_1, tau_visc), the
    consistent relaxation time is tau* itself.  Newton iterations from a tau_old
    that is far off must return it, and converge quadratically: the error
    after k + 1 iterations is far below the one after k.  The explicit update
    (0 iterations) returns the viscosity of the lagged strain rate instead."""
    nu, rho = 0.1, 1.0
    p0 = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=m)
    tstar = 0.5 + 3.0 * oracle.pr_nu_app(p0, gdot, rho)
    f = _ce_state(lat, _shear(gdot), tstar, rho)
    errs = []
    for k in range(0, 40):
        p = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=m, newton=k)
        _, tn, d = oracle.collide(lat, p, f, tau_old=0.5 + 0.5 * (tstar - 0.5))
        errs.append(abs(tn - tstar) / tstar)
    assert errs[0] > 1e-3                      # lagged tau is off
    assert errs[-1] < 1e-11
    assert abs(d["gdot"] - gdot) < 1e-9 * gdot
    k = next(i for i, e in enumerate(errs) if e < 1e-4)
    assert k < 30
    assert errs[k + 1] < 10 * errs[k] ** 1.5 + 1e-14     # superlinear once close


@pytest.mark.parametrize("rho", [1.0, 1.05])
def test_pr_newton_bingham_closed_form(rho):
    """For m gdot >> 1, nu_app = nu_p + sigma_y / (rho gdot) (eq. muApparent), so
    the consistency tau = 1/2 + 3 nu_app(a / tau) with a = tau gdot (the
    tau-independent product given by T) is linear in tau:
    tau = (1/2 + 3 nu_p) / (1 - 3 sigma_y / (rho a)).  Eq. (LBM_strain_rate) as
    printed has no rho (reading R7), so the state built with rho and strain
    rate gd carries a = rho tau gd."""
    lat = "D3Q27"
    nu, sy, m = 0.1, 2e-6, 1e12
    for tau_ce, gd in ((0.8, 4e-5), (1.7, 1e-4)):
        f = _ce_state(lat, _shear(gd), tau_ce, rho)
        a = rho * tau_ce * gd
        exact = (0.5 + 3 * nu) / (1 - 3 * sy / (rho * a))
        p = oracle.params(model="PR", nu_p=nu, sigma_y=sy, m=m, newton=12)
        tn = oracle.collide(lat, p, f, tau_old=0.6)[1]
        assert abs(tn - exact) < 1e-11 * exact


def test_pr_newton_newtonian_in_one_iteration():
    """sigma_y = 0: tau does not depend on the strain rate, the consistency
    condition is linear and one Newton iteration lands on tau = 1/2 + 3 nu_p,
    with the strain rate that tau implies."""
    lat = "D3Q19"
    rng = np.random.default_rng(37)
    f = _rand_state(lat, rng)
    p = oracle.params(model="PR", nu_p=0.07, sigma_y=0.0, m=1e6, newton=1)
    _, tn, d = oracle.collide(lat, p, f, tau_old=2.5)
    assert abs(tn - (0.5 + 3 * 0.07)) < 1e-15
    g_lag = oracle.collide(lat, oracle.params(model="PR", nu_p=0.07), f, tau_old=2.5)[2]["gdot"]
    assert abs(d["gdot"] - g_lag * 2.5 / tn) < 1e-12 * d["gdot"]
