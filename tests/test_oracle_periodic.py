"""Pins for the oracle's periodic pair term (Sec. 2.2: Eq. 2 with the image sum
of Eq. 5, cut at |x - nL| < 2.6 L, and the quasi-periodic leading term) and
its KDK step.

Pins: a perfect cubic lattice feels no force (every image set is inversion
symmetric); forces are invariant under a translation of all particles modulo
the box; Newton's third law; the quasi-periodic term of a cluster whose pairs
are all closer than L/2 is the open-boundary pair sum; and the cut sits at
2.6 L -- moving a pair so that exactly one image crosses the cut sphere changes
the force by that image's Newtonian term, G m / (2.6 L)^2 along the image's
direction, and by nothing else.
"""
import math

import numpy as np
import pytest

import oracle


def lattice(k, L):
    g = (np.arange(k) + 0.5) * L / k
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


@pytest.mark.parametrize("images", [0, 1])
def test_cubic_lattice_feels_no_force(images):
    # k = 7: 6.76 k^2 = 331.24 is not an integer, so no lattice vector lies on
    # the cut sphere (with k = 5 some do, and rounding would decide them)
    L, k = 3.0, 7
    pos = lattice(k, L)
    n = pos.shape[0]
    m = np.ones(n)
    h = np.full(n, 0.05)
    acc = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    one_term = 1.0 / (L / k) ** 2
    assert np.abs(acc).max() < 1e-12 * one_term * n


@pytest.mark.parametrize("images", [0, 1])
def test_translation_invariance_and_third_law(images):
    rng = np.random.default_rng(4)
    L, n = 2.0, 120
    pos = rng.random((n, 3)) * L
    m = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.01, 0.05, n)
    a0 = oracle.pair_acc_periodic(pos, m, h, 1.3, L, images)
    shifted = (pos + np.array([0.731, 1.377, 0.25])) % L
    a1 = oracle.pair_acc_periodic(shifted, m, h, 1.3, L, images)
    scale = np.abs(a0).max()
    assert np.abs(a1 - a0).max() < 1e-10 * scale
    net = np.abs((m[:, None] * a0).sum(0))
    assert np.all(net < 1e-12 * (m[:, None] * np.abs(a0)).sum())


def test_quasi_periodic_cluster_is_the_open_sum():
    rng = np.random.default_rng(8)
    L, n = 10.0, 200
    pos = 3.5 + rng.random((n, 3)) * 3.0          # all separations < 3*sqrt(3) < L/2
    m = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.01, 0.3, n)
    a = oracle.pair_acc_periodic(pos, m, h, 1.0, L, 1)
    b = oracle.pair_acc(pos, m, h, 1.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(b).max())


def test_cut_sits_at_two_point_six_box_lengths():
    """Particle j at x_i - delta*u along a generic direction u; at delta* one
    image n* has |delta* u - n*| = 2.6 exactly while every other image is far
    from the cut.  Crossing delta* adds exactly that image's Newtonian term."""
    L, G, mj = 1.0, 1.0, 0.7
    u = np.array([1.0, 0.37, 0.21])
    u /= np.linalg.norm(u)
    grid = np.arange(-5, 6)
    ns = np.stack(np.meshgrid(grid, grid, grid, indexing="ij"), -1).reshape(-1, 3).astype(float)
    found = None
    for nstar in ns:
        # |delta u - n|^2 = 2.6^2 -> delta^2 - 2 delta (u.n) + |n|^2 - 6.76 = 0
        b, c = u @ nstar, nstar @ nstar - 6.76
        disc = b * b - c
        if disc <= 0:
            continue
        for delta in (b - math.sqrt(disc), b + math.sqrt(disc)):
            if not 0.05 < delta < 0.95:
                continue
            dist = np.linalg.norm(delta * u - ns, axis=1)
            others = np.abs(dist - 2.6)[np.any(ns != nstar, axis=1)]
            if others.min() > 1e-3:
                found = (nstar, delta)
                break
        if found:
            break
    assert found is not None
    nstar, delta = found
    xi = np.array([0.5, 0.5, 0.5])
    h = np.array([1e-3, 1e-3])
    m = np.array([1.0, mj])

    def acc(dl):
        pos = np.stack([xi, (xi - dl * u) % L])
        return oracle.pair_acc_periodic(pos, m, h, G, L, 0)[0]

    eps = 1e-9
    jump = acc(delta + eps) - acc(delta - eps)
    d = delta * u - nstar                  # the image's separation x_i - x_j - n L at the crossing
    term = -G * mj * d / np.linalg.norm(d) ** 3
    inside_after = np.linalg.norm((delta + eps) * u - nstar) < 2.6
    expected = term if inside_after else -term
    np.testing.assert_allclose(jump, expected, rtol=1e-5, atol=1e-6 * np.linalg.norm(term))


def test_periodic_kdk_wraps_and_conserves_momentum():
    rng = np.random.default_rng(2)
    L, n = 1.0, 64
    pos = rng.random((n, 3)) * L
    vel = rng.normal(size=(n, 3)) * 0.5
    vel -= vel.mean(0)
    m = np.ones(n)
    h = np.full(n, 0.02)
    kd = oracle.KDKPeriodic(pos, vel, m, h, L, 0, Om=1.0, OL=0.0, a0=0.5)
    for _ in range(5):
        kd.step(0.01)
    assert np.all((kd.pos >= 0) & (kd.pos < L))
    # the pair term conserves momentum; the friction term scales it by the same factor for every particle
    p = (m[:, None] * kd.vel).sum(0)
    assert np.abs(p).max() < 1e-12 * (m[:, None] * np.abs(kd.vel)).sum()


@pytest.mark.parametrize("images", [0, 1])
def test_target_subset_equals_full_rows(images):
    """The sampled-target form used at large N returns exactly the rows of the
    full evaluation (same loops, same order)."""
    rng = np.random.default_rng(6)
    L, n = 1.5, 150
    pos = rng.random((n, 3)) * L
    m = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.01, 0.05, n)
    full = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    tg = np.array([0, 7, 33, 149, 7])
    sub = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images, targets=tg)
    assert np.array_equal(sub, full[tg])


@pytest.mark.parametrize("images", [0, 1])
def test_brute_force_newtonian_image_sum(images):
    """Tiny softening (every pair Newtonian): the oracle equals a direct Python
    sum of G m_j d / |d|^3 over the images the definition keeps, enumerated
    over a wide cube of n."""
    rng = np.random.default_rng(12)
    L, n, G = 1.3, 6, 0.8
    pos = rng.random((n, 3)) * L
    m = rng.uniform(0.5, 2.0, n)
    h = np.full(n, 1e-6)
    got = oracle.pair_acc_periodic(pos, m, h, G, L, images)
    rng4 = range(-4, 5)
    want = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            if j == i:
                continue
            d0 = pos[i] - pos[j]
            if images == 1:
                nv = np.floor(d0 / L + 0.5)
                d = d0 - nv * L
                want[i] -= G * m[j] * d / np.linalg.norm(d) ** 3
                continue
            for a in rng4:
                for b in rng4:
                    for c in rng4:
                        d = d0 - np.array([a, b, c]) * L
                        r = np.linalg.norm(d)
                        if r < 2.6 * L:
                            want[i] -= G * m[j] * d / r ** 3
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())

