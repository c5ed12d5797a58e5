"""Pins for the spherical-glass oracle (Sec. 3.1, Eq. 14-18) and for the
reversed-gravity equation of motion used to relax glasses.

Pins: the stereographic map's closed values and round trip; the compact
volume of Eq. 18 against direct quadrature of the 3-sphere's volume element and
against the 3-sphere's total volume 2 pi^2 R^3; equal compact volumes of the
constant-volume shells; total mass equal to the mean density times the
simulated volume (Eq. 16-17); placement inside each shell with the sin^2
distribution in omega (Kolmogorov-Smirnov) and isotropic directions; the
reversed pair term equal to minus the ordinary one, and a uniform comoving
sphere with no peculiar acceleration under reversed gravity too.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from oracle import glass

RHO = 0.3 * 3.0 / (8.0 * math.pi)


def test_projection_closed_values_and_round_trip():
    D = 60.0
    assert glass.omega_of_r(0.0, D) == 0.0
    assert glass.omega_of_r(D, D) == pytest.approx(math.pi / 2, rel=1e-15)   # tan(pi/4) = 1
    assert glass.r_of_omega(math.pi / 2, D) == pytest.approx(D, rel=1e-15)
    r = np.geomspace(1e-3, 1e5, 200)
    w = glass.omega_of_r(r, D)
    assert np.all(np.diff(w) > 0) and w[-1] < math.pi
    np.testing.assert_allclose(glass.r_of_omega(w, D), r, rtol=1e-12)


def test_compact_volume_against_quadrature():
    """V(omega) = int_0^omega 4 pi R^3 sin^2 w dw with R = D_s/2 is the form of Eq. 18."""
    D = 100.0
    R = D / 2
    for w in (0.05, 0.7, 1.9, 3.0):
        q, _ = integrate.quad(lambda x: 4 * math.pi * R ** 3 * math.sin(x) ** 2, 0.0, w, epsabs=0, epsrel=1e-13)
        assert glass.compact_volume(w, D) == pytest.approx(q, rel=1e-12)
    assert glass.compact_volume(math.pi, D) == pytest.approx(2 * math.pi ** 2 * R ** 3, rel=1e-14)


def test_constant_volume_edges_and_total_mass():
    D, R_sim, nr, ns = 100.0, 342.45, 40, 96
    edges, m, n_in, m_in = glass.layout(1, D, R_sim, nr, ns, 0.0, RHO)
    assert edges[0] == 0.0 and edges[-1] == pytest.approx(glass.omega_of_r(R_sim, D), rel=1e-15)
    dv = np.diff(glass.compact_volume(edges, D))
    np.testing.assert_allclose(dv, dv.mean(), rtol=1e-10)
    assert n_in == 0
    assert (m * ns).sum() == pytest.approx(RHO * 4 / 3 * math.pi * R_sim ** 3, rel=1e-12)
    assert np.all(np.diff(m) > 0)            # particle mass grows outwards


def test_constant_domega_edges_inner_ball_and_total_mass():
    D, R_sim, r_c, nr, ns = 60.0, 342.45, 45.0, 30, 64
    edges, m, n_in, m_in = glass.layout(0, D, R_sim, nr, ns, r_c, RHO)
    np.testing.assert_allclose(np.diff(edges), np.diff(edges).mean(), rtol=1e-12)
    assert edges[0] == pytest.approx(glass.omega_of_r(r_c, D), rel=1e-15)
    assert edges[-1] == pytest.approx(glass.omega_of_r(R_sim, D), rel=1e-15)
    assert m_in == m[0]                      # mass continuous at r_c
    m_ball = RHO * 4 / 3 * math.pi * r_c ** 3
    assert n_in == math.floor(m_ball / m_in)  # Eq. 17
    total = (m * ns).sum() + n_in * m_in
    shells = RHO * 4 / 3 * math.pi * (R_sim ** 3 - r_c ** 3)
    assert (m * ns).sum() == pytest.approx(shells, rel=1e-12)
    assert m_ball - m_in < n_in * m_in <= m_ball and total <= RHO * 4 / 3 * math.pi * R_sim ** 3


@pytest.mark.parametrize("scheme", [0, 1])
def test_placement_inside_shells_with_the_compact_volume_law(scheme):
    D, R_sim, r_c, nr, ns = 60.0, 200.0, 30.0, 12, 4000
    edges, m, n_in, m_in = glass.layout(scheme, D, R_sim, nr, ns, r_c, RHO)
    n = n_in + nr * ns
    u = np.random.default_rng(11).random((n, 3))
    pos, mass = glass.place(scheme, D, R_sim, nr, ns, r_c, RHO, u)
    r = np.linalg.norm(pos, axis=1)
    if n_in:
        assert np.all(r[:n_in] <= r_c * (1 + 1e-14)) and np.all(mass[:n_in] == m_in)
        # uniform in the real-space ball: (r / r_c)^3 is uniform
        assert stats.kstest((r[:n_in] / r_c) ** 3, "uniform").pvalue > 1e-3
    F = lambda w: 2 * w - np.sin(2 * w)
    for k in (0, nr // 2, nr - 1):
        sl = slice(n_in + k * ns, n_in + (k + 1) * ns)
        w = glass.omega_of_r(r[sl], D)
        lo, hi = edges[k], edges[k + 1]
        assert np.all(w >= lo - 1e-12) and np.all(w <= hi + 1e-12)
        assert np.all(mass[sl] == m[k])
        # sin^2 law within the shell: its CDF is (F(w) - F(lo)) / (F(hi) - F(lo))
        cdf = (F(w) - F(lo)) / (F(hi) - F(lo))
        assert stats.kstest(cdf, "uniform").pvalue > 1e-3
        unit = pos[sl] / r[sl, None]
        assert np.linalg.norm(unit.mean(0)) < 5.0 / math.sqrt(ns)
    # the inverse CDF hits the shell edges at u = 0 and u -> 1
    u2 = np.zeros((n, 3))
    u2[:, 0] = 0.0
    p0, _ = glass.place(scheme, D, R_sim, nr, ns, r_c, RHO, u2)
    u2[:, 0] = 1.0 - 2.0 ** -53
    p1, _ = glass.place(scheme, D, R_sim, nr, ns, r_c, RHO, u2)
    r0 = np.linalg.norm(p0[n_in:], axis=1).reshape(nr, ns)
    r1 = np.linalg.norm(p1[n_in:], axis=1).reshape(nr, ns)
    redges = glass.r_of_omega(edges, D)
    np.testing.assert_allclose(r0[:, 0], redges[:-1], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r1[:, 0], redges[1:], rtol=1e-9)


def test_reversed_gravity_flips_the_pair_term():
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(300, 3))
    m = rng.uniform(0.5, 2, 300)
    h = np.full(300, 0.05)
    a = oracle.KDK(pos, np.zeros_like(pos), m, h, oracle.cosmo(comoving=True))
    b = oracle.KDK(pos, np.zeros_like(pos), m, h, oracle.cosmo(reversed=True))
    assert b.c.comoving == 1 and b.c.reversed == 1
    np.testing.assert_array_equal(b.acc, -a.acc)


def test_uniform_comoving_sphere_at_rest_under_reversed_gravity():
    """With gravity reversed the pair sum pushes a uniform sphere apart and the
    reversed background term pulls it back: still no peculiar acceleration
    (a sign error in either term gives a ratio near +-2)."""
    rng = np.random.default_rng(5)
    n, R, Om = 16384, 10.0, 1.0
    rho = Om * 3 / (8 * math.pi)
    p = rng.uniform(-1, 1, (4 * n, 3))
    p = p[(p ** 2).sum(1) <= 1][:n] * R
    m = np.full(n, rho * 4 / 3 * math.pi * R ** 3 / n)
    h = np.full(n, 1e-3)
    a = 0.5
    kd = oracle.KDK(p, np.zeros_like(p), m, h, oracle.cosmo(Om=Om, OL=0.0, reversed=True), a0=a)
    dt = 1e-7
    kd.step(dt)
    A = kd.vel / dt
    r = np.linalg.norm(p, axis=1)
    inner = r < 0.5 * R
    ar = (A[inner] * p[inner]).sum(1) / r[inner]
    bg = 4 * math.pi / 3 * rho * r[inner] / a ** 3
    assert abs(ar.mean() / bg.mean()) < 0.05
