"""Pins for the oracle's spline kernel, pair potential and pair sum.

Each pin comes from outside the oracle's own formulas: Gauss's law applied to
the cubic-spline density the paper's kernel derives from, closed values of
Eq. 4 at its branch points, the shell theorem, Newton's third law, and a
40-digit brute-force sum that builds the kernel from the density instead of
Eq. 4.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import integrate

import oracle


def m4_density(r, h):
    """Cubic-spline (M4) density of unit mass with support radius h
    (Monaghan & Lattanzio 1985, the kernel Eq. 4 cites)."""
    u = r / h
    c = 8.0 / (math.pi * h ** 3)
    if u <= 0.5:
        return c * (1.0 - 6.0 * u * u + 6.0 * u ** 3)
    if u <= 1.0:
        return c * 2.0 * (1.0 - u) ** 3
    return 0.0


def force_from_density(r, h):
    """Gauss's law: F(r) = M(<r) / r^2 for the unit-mass M4 density."""
    pts = [p for p in (0.5 * h, h) if p < r]
    m, _ = integrate.quad(lambda s: 4.0 * math.pi * s * s * m4_density(s, h), 0.0, r,
                          points=pts or None, epsabs=0.0, epsrel=1e-13, limit=200)
    return m / (r * r)


def test_m4_density_has_unit_mass():
    m, _ = integrate.quad(lambda s: 4 * math.pi * s * s * m4_density(s, 0.7), 0, 0.7,
                          points=[0.35], epsabs=0, epsrel=1e-13)
    assert abs(m - 1.0) < 1e-12


@pytest.mark.parametrize("h", [0.01, 0.3, 1.0, 7.5])
def test_spline_equals_gauss_law_of_m4_density(h):
    # a dropped term, a wrong coefficient or a swapped branch in Eq. 4 fails here
    for u in [1e-3, 0.05, 0.2, 0.37, 0.4999, 0.5, 0.5001, 0.63, 0.8, 0.95, 0.9999, 1.0, 1.3, 4.0]:
        r = u * h
        ref = force_from_density(r, h)
        got = oracle.spline_F(r, h)
        assert abs(got - ref) <= 1e-11 * abs(ref), (u, got, ref)


def test_spline_closed_values_and_limits():
    for h in [0.1, 1.0, 3.0]:
        # continuous at r = h/2 with value 38/(15 h^2) from both sides
        assert math.isclose(oracle.spline_F(0.5 * h * (1 - 1e-12), h), 38 / (15 * h * h), rel_tol=1e-9)
        assert math.isclose(oracle.spline_F(0.5 * h, h), 38 / (15 * h * h), rel_tol=1e-12)
        # Newtonian from r = h on: 1/h^2 at the boundary (also the limit from below)
        assert math.isclose(oracle.spline_F(h, h), 1 / (h * h), rel_tol=1e-15)
        assert math.isclose(oracle.spline_F(h * (1 - 1e-12), h), 1 / (h * h), rel_tol=1e-9)
        assert oracle.spline_F(2 * h, h) == 1 / (4 * h * h)
        # linear near the centre: F ~ (4 pi/3) rho(0) r = 32 r / (3 h^3)
        r = 1e-6 * h
        assert math.isclose(oracle.spline_F(r, h), 32 * r / (3 * h ** 3), rel_tol=1e-9)
        assert oracle.spline_F(0.0, h) == 0.0


@pytest.mark.parametrize("H", [0.05, 1.0])
def test_pair_potential(H):
    # W(0) = -2.8/H: the depth that makes the Plummer-equivalent softening H/2.8
    assert math.isclose(oracle.pair_W(0.0, H), -2.8 / H, rel_tol=1e-15)
    for u in [1.0, 1.5, 10.0]:
        assert math.isclose(oracle.pair_W(u * H, H), -1.0 / (u * H), rel_tol=1e-15)
    # dW/dr = F everywhere, including across both branch points
    for u in [0.1, 0.3, 0.49, 0.5, 0.51, 0.7, 0.99, 1.0, 1.01, 2.0]:
        r = u * H
        d = 1e-6 * H
        dW = (oracle.pair_W(r + d, H) - oracle.pair_W(r - d, H)) / (2 * d)
        assert math.isclose(dW, force_from_density(r, H), rel_tol=1e-7), u
    # W(r) = -int_r^inf F by quadrature of the density-derived force
    for u in [0.0, 0.25, 0.75]:
        r = u * H
        inner, _ = integrate.quad(lambda s: force_from_density(s, H), r, H, points=[0.5 * H],
                                  epsrel=1e-12, epsabs=0)
        assert math.isclose(oracle.pair_W(r, H), -(inner + 1.0 / H), rel_tol=1e-9)


def test_softening_eq7():
    m = np.array([3.0, 1.5, 1.5 * 27, 1.5 * 8])
    h = oracle.softening(m, 0.01)
    np.testing.assert_allclose(h, [0.01 * 2 ** (1 / 3), 0.01, 0.03, 0.02], rtol=1e-15)


def test_single_pair_closed_form():
    G = 2.5
    pos = np.array([[0.1, -0.2, 0.3], [0.1 + 0.3, -0.2 + 0.4, 0.3]])  # separation 0.5 along (0.6, 0.8, 0)
    m = np.array([2.0, 3.0])
    for h in ([0.1, 0.1], [0.2, 0.4], [0.3, 0.1]):  # Newtonian, spline-inner, spline-outer
        h = np.array(h, dtype=float)
        acc = oracle.pair_acc(pos, m, h, G)
        H = h.sum()
        mag1 = G * m[1] * force_from_density(0.5, H)
        mag0 = G * m[0] * force_from_density(0.5, H)
        np.testing.assert_allclose(acc[0], mag1 * np.array([0.6, 0.8, 0.0]), rtol=1e-11, atol=1e-300)
        np.testing.assert_allclose(acc[1], -mag0 * np.array([0.6, 0.8, 0.0]), rtol=1e-11, atol=1e-300)
    # coincident particles exert nothing on each other
    acc = oracle.pair_acc(np.zeros((2, 3)), m, np.array([0.1, 0.1]), G)
    assert np.all(acc == 0.0)


def _m4_force_closed(r, h):
    """Enclosed-mass force of the M4 density, integrated exactly with mpmath
    polynomials (independent of Eq. 4's printed coefficients)."""
    r = mpmath.mpf(r)
    h = mpmath.mpf(h)
    if r >= h:
        return 1 / (r * r)
    c = 32 / h ** 3  # 4 pi * 8/(pi h^3)
    def inner(s):  # int_0^s x^2 (1 - 6 x^2/h^2 + 6 x^3/h^3) dx
        return s ** 3 / 3 - 6 * s ** 5 / (5 * h * h) + s ** 6 / h ** 3
    def outer(s):  # int x^2 2 (1 - x/h)^3 dx, antiderivative
        return 2 * (s ** 3 / 3 - 3 * s ** 4 / (4 * h) + 3 * s ** 5 / (5 * h * h) - s ** 6 / (6 * h ** 3))
    if r <= h / 2:
        M = c * inner(r)
    else:
        M = c * (inner(h / 2) + outer(r) - outer(h / 2))
    return M / (r * r)


def test_brute_force_40_digits():
    mpmath.mp.dps = 40
    rng = np.random.default_rng(11)
    n = 48
    pos = rng.normal(size=(n, 3)) * 0.3
    pos[5] = pos[4] + 1e-3  # a close pair deep in the spline core
    m = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.02, 0.2, n)
    G = 0.7
    acc = oracle.pair_acc(pos, m, h, G)
    for i in range(n):
        ref = [mpmath.mpf(0)] * 3
        for j in range(n):
            if j == i:
                continue
            d = [mpmath.mpf(float(pos[j, k])) - mpmath.mpf(float(pos[i, k])) for k in range(3)]
            r = mpmath.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            f = G * mpmath.mpf(float(m[j])) * _m4_force_closed(r, mpmath.mpf(float(h[i])) + mpmath.mpf(float(h[j]))) / r
            for k in range(3):
                ref[k] += f * d[k]
        ref = np.array([float(x) for x in ref])
        assert np.linalg.norm(acc[i] - ref) <= 1e-12 * np.linalg.norm(ref), i


def test_third_law_static():
    rng = np.random.default_rng(3)
    n = 500
    pos = rng.normal(size=(n, 3))
    m = rng.lognormal(size=n)
    h = 0.05 * np.cbrt(m)
    acc = oracle.pair_acc(pos, m, h, 1.0)
    net = (m[:, None] * acc).sum(0)
    scale = (m[:, None] * np.abs(acc)).sum()
    assert np.all(np.abs(net) <= 1e-13 * scale)


def fibonacci_shell(n, R):
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    phi = math.pi * (1 + 5 ** 0.5) * k
    s = np.sqrt(1 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], 1) * R


def test_shell_theorem():
    n, R, M = 20000, 1.0, 3.0
    shell = fibonacci_shell(n, R)
    probes = np.array([[0.3, 0, 0], [0, 0.6, 0], [0.2, -0.3, 0.4], [2.0, 0, 0], [0, 0, -5.0], [3.0, 3.0, 0]])
    pos = np.concatenate([shell, probes])
    m = np.concatenate([np.full(n, M / n), np.zeros(len(probes))])
    h = np.full(len(pos), 1e-4)
    tg = np.arange(n, len(pos))
    acc = oracle.pair_acc(pos, m, h, 1.0, targets=tg)
    r = np.linalg.norm(probes, axis=1)
    inside = r < R
    # interior: no net force (up to the lattice's discreteness)
    assert np.all(np.linalg.norm(acc[inside], axis=1) < 1e-3 * M / R ** 2)
    # exterior: point-mass force G M / r^2 pointing at the centre
    expect = -M * probes[~inside] / r[~inside, None] ** 3
    err = np.linalg.norm(acc[~inside] - expect, axis=1) / np.linalg.norm(expect, axis=1)
    assert np.all(err < 1e-6)
