"""Pins of the oracle's velocity sets and equilibrium against exact identities.

The weights are not printed in the paper (Sec. 4.1 names the lattices only);
what fixes them is that the lattice moments reproduce the isotropic tensors
up to fourth order with c_s^2 = 1/3, which is what eq. (MomentsEqLBM)
requires of the equilibrium of eq. (f_eq).  A wrong weight, a missing or
duplicated velocity fails one of these identities.
"""
import itertools

import numpy as np
import pytest

import oracle

LATS = {"D2Q9": (9, 2), "D3Q15": (15, 3), "D3Q19": (19, 3), "D3Q27": (27, 3)}
CS2 = 1.0 / 3.0


def _delta(D):
    d = np.zeros((3, 3))
    d[:D, :D] = np.eye(D)
    return d


@pytest.mark.parametrize("lat", list(LATS))
def test_velocity_set_shape_and_opposites(lat):
    c, w, opp = oracle.lattice_info(lat)
    Q, D = LATS[lat]
    assert c.shape == (Q, 3) and w.shape == (Q,)
    assert len({tuple(v) for v in c}) == Q
    assert np.all(np.abs(c) <= 1)
    if D == 2:
        assert np.all(c[:, 2] == 0)
    for i in range(Q):
        assert np.array_equal(c[opp[i]], -c[i])
        assert opp[opp[i]] == i
    assert np.all(w > 0)


@pytest.mark.parametrize("lat", list(LATS))
def test_isotropy_to_fourth_order(lat):
    c, w, _ = oracle.lattice_info(lat)
    Q, D = LATS[lat]
    c = c.astype(np.float64)
    d = _delta(D)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * d, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("lat", list(LATS))
def test_equilibrium_moments(lat):
    """eq. (MomentsEqLBM): sum f_eq = rho, sum c f_eq = rho u,
    sum c c f_eq = rho c_s^2 I + rho u u."""
    c, w, _ = oracle.lattice_info(lat)
    Q, D = LATS[lat]
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 0.8 + 0.4 * rng.random()
        u = np.zeros(3)
        u[:D] = 0.1 * (rng.random(D) - 0.5)
        f = oracle.feq(lat, rho, u)
        cf = c.astype(np.float64)
        assert abs(f.sum() - rho) < 1e-14
        assert np.allclose(cf.T @ f, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("ia,ib,i->ab", cf, cf, f),
                           rho * CS2 * _delta(D) + rho * np.outer(u, u), atol=1e-15)


def test_equilibrium_is_second_order_expansion():
    """f_eq for u = 0 is rho w_i; the u-derivative is rho w_i c_i / c_s^2."""
    c, w, _ = oracle.lattice_info("D3Q27")
    assert np.allclose(oracle.feq("D3Q27", 1.3, [0, 0, 0]), 1.3 * w, rtol=0, atol=1e-16)
    eps = 1e-6
    d = (oracle.feq("D3Q27", 1.0, [eps, 0, 0]) - oracle.feq("D3Q27", 1.0, [-eps, 0, 0])) / (2 * eps)
    assert np.allclose(d, w * c[:, 0] / CS2, atol=1e-9)
