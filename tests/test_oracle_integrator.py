"""Pins for the oracle's KDK integrator (Eq. 9-11), RK4 scale factor (Eq. 1),
the comoving equation of motion (Eq. 8) and the pair counts.

Pins: Kepler's period and second-order convergence of KDK, energy conservation
in a static background, the flat-LambdaCDM closed form a(t), a uniform
comoving sphere that must feel no peculiar acceleration, and pair counts from
an independent k-d tree.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1811_05903_gb300 import workloads


def kepler(e, dt, periods):
    """Two equal masses, G = M = 1, semi-major axis 1, released at apocentre."""
    ra = 1.0 + e
    vrel = math.sqrt((1.0 - e) / (1.0 + e))
    pos = np.array([[0.5 * ra, 0, 0], [-0.5 * ra, 0, 0]])
    vel = np.array([[0, 0.5 * vrel, 0], [0, -0.5 * vrel, 0]])
    m = np.array([0.5, 0.5])
    h = np.array([1e-4, 1e-4])
    kd = oracle.KDK(pos, vel, m, h, oracle.cosmo(comoving=False))
    e0 = kd.energy()
    nsteps = int(round(periods * 2 * math.pi / dt))
    de_max = 0.0
    for _ in range(nsteps):
        kd.step(dt)
        de_max = max(de_max, abs(kd.energy() - e0) / abs(e0))
    return kd, de_max, pos


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kepler_period_and_second_order(e):
    errs = []
    for dt in (2 * math.pi / 400, 2 * math.pi / 800):
        kd, de, pos0 = kepler(e, dt, 10)
        # after whole periods the bodies are back at the start (period 2 pi sqrt(a^3/GM))
        dx = np.linalg.norm(kd.pos - pos0)
        errs.append((de, dx))
    (de1, dx1), (de2, dx2) = errs
    assert dx1 < 0.2 and dx2 < dx1
    # second order: halving dt cuts the phase error and the (bounded, oscillating)
    # energy error ~4x; on a circular orbit the energy error is at rounding level
    assert 3.0 < dx1 / dx2 < 5.0
    if e > 0:
        assert 3.0 < de1 / de2 < 5.0
    assert de2 < 1e-3


def test_static_energy_conservation_small_system():
    p = workloads.static_ball(seed=1)
    h = oracle.softening(p.mass, p.h_min)
    des = []
    for dt in (1e-3, 5e-4):
        kd = oracle.KDK(p.pos, p.vel, p.mass, h, oracle.cosmo(comoving=False))
        e0 = kd.energy()
        for _ in range(int(round(0.01 / dt))):
            kd.step(dt)
        des.append(abs(kd.energy() - e0) / abs(e0))
        # momentum stays zero in the static mode (Newton's third law)
        _, pmom = oracle.kinetic(kd.vel, kd.m)
        assert np.linalg.norm(pmom) < 1e-11 * (kd.m.sum() * np.abs(kd.vel).max() + 1e-300) + 1e-12
    # the heavy outer shells dominate E; at dt = 1e-3 the drift is ~2e-4 and
    # falls as dt^2 (KDK is second order)
    assert des[0] < 1e-3
    assert 3.5 < des[0] / des[1] < 4.5


def test_rk4_matches_flat_lcdm_closed_form():
    c = oracle.cosmo(Om=0.3, OL=0.7, comoving=True)
    a_sched, dts = workloads.loga_schedule(0.02, 1.0, 200, 0.3, 0.7)
    a = a_sched[0]
    for n, dt in enumerate(dts):
        a = oracle.rk4_a(a, dt, c)
        assert abs(a - a_sched[n + 1]) <= 1e-9 * a_sched[n + 1]
    # Eq. 1 itself: H(a=1) = H0 and the matter era limit
    assert math.isclose(oracle.hubble(1.0, c), 1.0, rel_tol=1e-15)
    assert math.isclose(oracle.hubble(0.5, c), math.sqrt(0.3 * 8 + 0.7), rel_tol=1e-15)


def test_uniform_comoving_sphere_has_no_peculiar_acceleration():
    """Eq. 8 with the background term (4 pi G/3) rho_bar x / a^3: inside a
    uniform sphere of mean density rho_bar the pair sum and the background
    cancel at any a.  A sign error gives a ratio near 2, a missing 1/a^3 a
    ratio near 1 - a^-3."""
    rng = np.random.default_rng(5)
    n, R, Om = 16384, 10.0, 0.3
    rho = Om * 3 / (8 * math.pi)
    pos = rng.uniform(-1, 1, (4 * n, 3))
    pos = pos[(pos ** 2).sum(1) <= 1][:n] * R
    m = np.full(n, rho * 4 / 3 * math.pi * R ** 3 / n)
    h = np.full(n, 1e-3)
    a = 0.5
    c = oracle.cosmo(Om=Om, OL=1 - Om, comoving=True)
    kd = oracle.KDK(pos, np.zeros_like(pos), m, h, c, a0=a)
    dt = 1e-7
    kd.step(dt)
    A = kd.vel / dt  # ~ the Eq. 8 acceleration at rest
    r = np.linalg.norm(pos, axis=1)
    inner = r < 0.5 * R
    ar = (A[inner] * pos[inner]).sum(1) / r[inner]
    bg = 4 * math.pi / 3 * rho * r[inner] / a ** 3
    ratio = ar.mean() / bg.mean()
    assert abs(ratio) < 0.05, ratio


def test_paircount_matches_kdtree():
    rng = np.random.default_rng(9)
    n = 1500
    scale = 2 ** 16
    q = rng.integers(-scale, scale, size=(n, 3)).astype(np.int32)
    # squared edges in integer units, log spaced
    edges = np.geomspace(2000.0, 60000.0, 13)
    edge2 = np.ceil(edges ** 2).astype(np.int64)
    dd = oracle.paircount(q, edge2)
    tree = cKDTree(q.astype(np.float64))
    # an integer d^2 < E  <=>  d <= sqrt(E - 1/2); no integer distance sits on that radius
    cum = np.array([(tree.count_neighbors(tree, math.sqrt(E - 0.5)) - n) // 2 for E in edge2])
    np.testing.assert_array_equal(dd.astype(np.int64), np.diff(cum))


def test_ball_pair_cdf_against_sampled_pairs():
    """RR normalisation P(2R) = 1, P(0) = 0, monotone; and the CDF against the
    distances of independently sampled uniform pairs (Kolmogorov bound)."""
    R = 3.0
    assert oracle.ball_pair_cdf(0.0, R) == 0.0 and oracle.ball_pair_cdf(2 * R, R) == 1.0
    s = np.linspace(0, 2 * R, 1001)
    assert np.all(np.diff(oracle.ball_pair_cdf(s, R)) >= 0)
    rng = np.random.default_rng(12)
    def ball(k):
        u = rng.uniform(-1, 1, (3 * k, 3))
        return u[(u ** 2).sum(1) <= 1][:k] * R
    m = 400_000
    d = np.sort(np.linalg.norm(ball(m) - ball(m), axis=1))
    emp = np.arange(1, m + 1) / m
    ks = np.max(np.abs(emp - oracle.ball_pair_cdf(d, R)))
    assert ks < 1.63 / math.sqrt(m) * 1.5, ks  # well inside the 1% Kolmogorov quantile


def test_xi_of_poisson_ball_is_zero():
    """Pair counts of a uniform ball through the oracle: xi = 0 within the noise
    of a U-statistic (a Poisson term 1/sqrt(RR) plus a term of order 1/sqrt(n)
    from pairs that share a point)."""
    rng = np.random.default_rng(13)
    n, R = 2500, 50.0
    u = rng.uniform(-1, 1, (3 * n, 3))
    pts = u[(u ** 2).sum(1) <= 1][:n] * R
    step = R / 2 ** 20
    q = np.rint(pts / step).astype(np.int32)
    edges = np.geomspace(5.0, 90.0, 9)
    dd = oracle.paircount(q, np.ceil((edges / step) ** 2).astype(np.int64))
    rr = oracle.rr_ball(n, R, edges)
    xi = oracle.xi_natural(dd, n, R, edges)
    assert np.all(np.abs(xi) < 5 / np.sqrt(rr) + 4 / math.sqrt(n)), xi


# ---------------------------------------------------------------- Eq. 12 ----

def test_timestep_bound_pair_closed_form():
    """Two bodies far outside their softening: |A_1| = G m_2 / r^2, |A_2| = G m_1 / r^2,
    so dt = min_i sqrt(2 * 2.8 h_i * eps * r^2 / (G m_other))."""
    G, r, eps = 1.7, 3.0, 0.02
    pos = np.array([[0.0, 0.0, 0.0], [0.0, r, 0.0]])
    m = np.array([2.0, 0.5])
    h = np.array([1e-3, 4e-3])
    acc = oracle.pair_acc(pos, m, h, G)
    c = oracle.cosmo(G=G, comoving=False)
    dt = oracle.timestep(pos, np.zeros_like(pos), acc, h, eps, 1e9, 1.0, c)
    want = min(math.sqrt(2 * 2.8 * h[0] * eps * r * r / (G * m[1])),
               math.sqrt(2 * 2.8 * h[1] * eps * r * r / (G * m[0])))
    assert dt == pytest.approx(want, rel=1e-13)
    # dt_max wins when smaller; a finite time left wins when smaller still; never below 0
    assert oracle.timestep(pos, np.zeros_like(pos), acc, h, eps, 0.5 * want, 1.0, c) == 0.5 * want
    assert oracle.timestep(pos, np.zeros_like(pos), acc, h, eps, 1e9, 1.0, c, t_left=0.25 * want) == 0.25 * want
    assert oracle.timestep(pos, np.zeros_like(pos), acc, h, eps, 1e9, 1.0, c, t_left=-1.0) == 0.0


def test_timestep_comoving_background_and_friction_terms():
    """A lone particle (no pair term) in comoving mode: at rest off-centre it feels
    only the background term (1/2) Om H0^2 x / a^3; moving through the centre only
    the friction -2 H(a) v.  Both give dt in closed form; at rest at the centre
    nothing limits the step and dt = dt_max."""
    c = oracle.cosmo(G=1.0, H0=1.0, Om=0.3, OL=0.7, comoving=True)
    a, eps, hh = 0.25, 0.01, np.array([0.05])
    x = np.array([[3.0, -4.0, 0.0]])
    zero = np.zeros((1, 3))
    dt = oracle.timestep(x, zero, zero, hh, eps, 1e9, a, c)
    A = 0.5 * 0.3 * 5.0 / a ** 3
    assert dt == pytest.approx(math.sqrt(2 * 2.8 * 0.05 * eps / A), rel=1e-13)
    v = np.array([[0.0, 0.0, 2.0]])
    H = math.sqrt(0.3 / a ** 3 + 0.7)
    dt = oracle.timestep(zero, v, zero, hh, eps, 1e9, a, c)
    assert dt == pytest.approx(math.sqrt(2 * 2.8 * 0.05 * eps / (2 * H * 2.0)), rel=1e-13)
    assert oracle.timestep(zero, zero, zero, hh, eps, 0.125, a, c) == 0.125


def test_adaptive_kepler_energy_error_scales_with_eps():
    """Eq. 12 makes dt proportional to sqrt(eps); KDK's energy error goes as dt^2,
    so on an eccentric orbit it must fall about 4x when eps falls 4x."""
    def run(eps):
        e = 0.6
        ra = 1.0 + e
        vrel = math.sqrt((1.0 - e) / (1.0 + e))
        pos = np.array([[0.5 * ra, 0, 0], [-0.5 * ra, 0, 0]])
        vel = np.array([[0, 0.5 * vrel, 0], [0, -0.5 * vrel, 0]])
        m = np.array([0.5, 0.5])
        h = np.array([1e-3, 1e-3])
        kd = oracle.KDK(pos, vel, m, h, oracle.cosmo(comoving=False))
        e0 = kd.energy()
        t_end = 4 * math.pi
        de, steps = 0.0, 0
        while kd.t.value < t_end:
            dt = kd.adaptive_step(eps, 0.05, t_end)
            steps += 1
            de = max(de, abs(kd.energy() - e0) / abs(e0))
            assert dt > 0
        assert kd.t.value == pytest.approx(t_end, abs=1e-12)
        return de, steps
    de1, n1 = run(0.04)
    de2, n2 = run(0.01)
    assert 1.7 < n2 / n1 < 2.3          # sqrt(4) more steps
    assert 3.0 < de1 / de2 < 5.0, (de1, de2)
