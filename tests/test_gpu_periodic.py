"""GPU parity of the periodic mode (Sec. 2.2: Eq. 2 with the image sum of Eq. 5,
cut at |x - nL| < 2.6 L, and the quasi-periodic leading term) against the FP64
oracle, on the same seeded inputs.

The FP32 path carries pair separations to ~1 ulp and re-takes, in FP64, every
include/exclude decision that falls within a thin band of the cut sphere or of
the half-box faces; the tests place pairs right on those boundaries.
Tolerances: FP64 path 1e-12 per element; FP32 path rms <= 1e-6 and per element
2e-5, as for the open-boundary force (a wrong decision would cost a whole
image's term, orders of magnitude above these).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05903_gb300 import steps

pytestmark = pytest.mark.gpu

RMS_TOL, MAX_TOL = 1e-6, 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    steps.load(build_if_missing=True)


def clumpy_box(seed, n, L):
    """A few Gaussian clumps plus a uniform background, wrapped into [0, L)^3."""
    rng = np.random.default_rng(seed)
    k = n // 2
    centres = rng.random((6, 3)) * L
    clump = centres[rng.integers(0, 6, k)] + rng.normal(size=(k, 3)) * 0.06 * L
    pos = np.concatenate([clump, rng.random((n - k, 3)) * L]) % L
    m = rng.uniform(0.5, 1.5, n)
    h = rng.uniform(0.002, 0.01, n) * L
    return pos, m, h


def periodic_sim(pos, m, h, L, images, prec, vel=None, a0=1.0, resort_every=8, variant=None):
    tile = 0 if variant is None else steps.steps_variants().index(variant) + 1
    cfg = steps.make_config(mode=steps.STEPS_PERIODIC, prec=prec, G=1.0, Om=1.0, OL=0.0, box=L, images=images,
                            resort_every=resort_every, tile_override=tile)
    return steps.Simulation(pos, np.zeros_like(pos) if vel is None else vel, m, soft=h, a0=a0, cfg=cfg)


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("images", [0, 1])
@pytest.mark.parametrize("n", [700, 3000])
def test_periodic_forces_match_oracle(images, n):
    L = 2.0
    pos, m, h = clumpy_box(10 + n + images, n, L)
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F64)
    e = rel_err(sim.forces(), ref)
    sim.close()
    assert e.max() <= 1e-12, e.max()
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP)
    e = rel_err(sim.forces(), ref)
    sim.close()
    rms = math.sqrt(np.mean(e ** 2))
    print("n=%d images=%d FP32 rms %.2e max %.2e" % (n, images, rms, e.max()))
    assert rms <= RMS_TOL and e.max() <= MAX_TOL, (rms, e.max())


@pytest.mark.parametrize("variant", ["comp_ki4_w4_u4", "exp_ki6_w4_u4"])
@pytest.mark.parametrize("images", [0, 1])
def test_periodic_tile_sizes(variant, images):
    """128- and 192-particle tiles (one image per warp step, 4 or 6 targets per
    lane) against the oracle; the default at these sizes is 64-particle tiles
    with two image slots per warp."""
    L, n = 2.0, 3000
    pos, m, h = clumpy_box(40 + images, n, L)
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP, variant=variant)
    e = rel_err(sim.forces(), ref)
    sim.close()
    rms = math.sqrt(np.mean(e ** 2))
    print("%s images=%d FP32 rms %.2e max %.2e" % (variant, images, rms, e.max()))
    assert rms <= RMS_TOL and e.max() <= MAX_TOL, (rms, e.max())


@pytest.mark.parametrize("kind", ["uniform", "clumpy"])
def test_periodic_16k_sampled_targets(kind):
    """The size the periodic throughput is measured at (N = 16,384, L = 1, cut
    image sum): FP32 against the oracle on 64 sampled targets.  Here the far
    images dominate (~53 of the ~74 images per pair lie wholly inside the cut
    sphere) and the sum cancels heavily in the uniform box."""
    L, n = 1.0, 16384
    rng = np.random.default_rng(16)
    if kind == "uniform":
        pos = rng.random((n, 3)) * L
        m = np.full(n, 1.0 / n)
        h = np.full(n, 0.02 * L / n ** (1.0 / 3.0))
    else:
        pos, m, h = clumpy_box(16, n, L)
    tg = np.sort(rng.choice(n, 64, replace=False))
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, 0, targets=tg)
    sim = periodic_sim(pos, m, h, L, 0, steps.STEPS_F32_COMP)
    e = rel_err(sim.forces()[tg], ref)
    sim.close()
    rms = math.sqrt(np.mean(e ** 2))
    print("N=16384 %s FP32 rms %.2e max %.2e" % (kind, rms, e.max()))
    assert rms <= RMS_TOL and e.max() <= MAX_TOL, (rms, e.max())


@pytest.mark.parametrize("images", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 63, 65])
def test_periodic_small_and_ragged(images, n):
    """Degenerate and ragged sizes: one particle (no pair; its own images are
    excluded, so no force), two particles, and tile counts one below and above
    a 64-particle tile."""
    L = 1.5
    rng = np.random.default_rng(70 + n + images)
    pos = rng.random((n, 3)) * L
    m = rng.uniform(0.5, 1.5, n)
    h = rng.uniform(0.002, 0.01, n) * L
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    for prec in (steps.STEPS_F64, steps.STEPS_F32_COMP):
        sim = periodic_sim(pos, m, h, L, images, prec)
        got = sim.forces()
        sim.close()
        if n == 1:
            assert np.all(got == 0.0) and np.all(ref == 0.0)
            continue
        e = rel_err(got, ref)
        assert e.max() <= (1e-12 if prec == steps.STEPS_F64 else MAX_TOL), (prec, e.max())


@pytest.mark.parametrize("images", [0, 1])
@pytest.mark.parametrize("n", [127, 128, 129, 511, 513, 2000])
def test_periodic_symmetric_ragged_tiles(n, images):
    """The default path of both sums (the symmetric kernel on 128-particle
    tiles, padding to 512): sizes around one tile and one padded block, every
    target against the oracle."""
    L = 1.0
    pos, m, h = clumpy_box(300 + n + images, n, L)
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images)
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP)
    got = sim.forces()
    sim.close()
    e = rel_err(got, ref)
    rms = math.sqrt(np.mean(e ** 2))
    assert rms <= RMS_TOL and e.max() <= MAX_TOL, (n, rms, e.max())


@pytest.mark.parametrize("images", [0, 1])
def test_periodic_symmetric_third_law_bitwise_and_per_target_kernel(images):
    """Each Newtonian (tile pair, image) is evaluated once and added to both
    particles in 64-bit fixed point: the net force vanishes to rounding (no
    pair of these random positions sits exactly on a half-box face, where the
    quasi-periodic sum is not antisymmetric), two evaluations agree bit for
    bit, and the per-target kernel on the same 128-particle tiles (each order
    of every pair evaluated separately) agrees within the FP32 contract."""
    L, n = 2.0, 4000
    pos, m, h = clumpy_box(77 + images, n, L)
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP)
    a1 = sim.forces()
    a2 = sim.forces()
    sim.close()
    assert np.array_equal(a1, a2)
    net = np.abs((m[:, None] * a1).sum(0))
    scale = (m[:, None] * np.abs(a1)).sum()
    assert np.all(net <= 1e-6 * scale), net / scale
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP, variant="comp_ki4_w4_u4")
    b = sim.forces()
    sim.close()
    e = rel_err(a1, b)
    assert math.sqrt(np.mean(e ** 2)) <= RMS_TOL and e.max() <= MAX_TOL, (math.sqrt(np.mean(e ** 2)), e.max())


@pytest.mark.parametrize("images", [0, 1])
def test_periodic_65k_sampled_targets(images):
    """N = 65,536 (1,024 tiles, 19 source chunks per target tile): FP32 against
    the oracle on 32 sampled targets of a clumpy box."""
    L, n = 1.0, 65536
    pos, m, h = clumpy_box(65, n, L)
    tg = np.sort(np.random.default_rng(66).choice(n, 32, replace=False))
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, images, targets=tg)
    sim = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP)
    e = rel_err(sim.forces()[tg], ref)
    sim.close()
    rms = math.sqrt(np.mean(e ** 2))
    print("N=65536 images=%d FP32 rms %.2e max %.2e" % (images, rms, e.max()))
    assert rms <= RMS_TOL and e.max() <= MAX_TOL, (rms, e.max())


def test_pairs_on_the_cut_sphere():
    """Pairs whose separation puts one image within ~1e-8 of 2.6 L, on both sides:
    the FP32 path must make the definition's FP64 decision for every one."""
    L = 1.0
    u = np.array([1.0, 0.37, 0.21])
    u /= np.linalg.norm(u)
    grid = np.arange(-5, 6)
    ns = np.stack(np.meshgrid(grid, grid, grid, indexing="ij"), -1).reshape(-1, 3).astype(float)
    deltas = []
    for nstar in ns:
        b, c = u @ nstar, nstar @ nstar - 6.76
        disc = b * b - c
        if disc > 0:
            deltas += [d for d in (b - math.sqrt(disc), b + math.sqrt(disc)) if 0.05 < d < 0.95]
    rng = np.random.default_rng(3)
    pts = []
    for k, d in enumerate(sorted(deltas)[:40]):
        base = rng.random(3) * L
        for off in (-3e-8, 3e-8):
            pts += [base, (base - (d + off) * u) % L]
    pos = np.array(pts)
    n = pos.shape[0]
    m = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 1e-4)
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, 0)
    for prec, tol in ((steps.STEPS_F64, 1e-12), (steps.STEPS_F32_COMP, 2e-5)):
        sim = periodic_sim(pos, m, h, L, 0, prec)
        e = rel_err(sim.forces(), ref)
        sim.close()
        assert e.max() <= tol, (prec, e.max())


def test_pairs_on_the_half_box_faces():
    """Quasi-periodic: pairs separated by L/2 +- 1e-9 along an axis, where the
    leading image flips from one side to the other."""
    L = 3.0
    rng = np.random.default_rng(5)
    pts = []
    for k in range(60):
        base = rng.random(3) * L
        axis = k % 3
        off = np.zeros(3)
        off[axis] = 0.5 * L + (1e-9 if k % 2 else -1e-9) * (1 + k)
        off[(axis + 1) % 3] = rng.uniform(-0.3, 0.3)
        pts += [base, (base + off) % L]
    pos = np.array(pts)
    n = pos.shape[0]
    m = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 1e-4)
    ref = oracle.pair_acc_periodic(pos, m, h, 1.0, L, 1)
    for prec, tol in ((steps.STEPS_F64, 1e-12), (steps.STEPS_F32_COMP, 2e-5)):
        sim = periodic_sim(pos, m, h, L, 1, prec)
        e = rel_err(sim.forces(), ref)
        sim.close()
        assert e.max() <= tol, (prec, e.max())


@pytest.mark.parametrize("images", [0, 1])
@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-9), (steps.STEPS_F32_COMP, 2e-5)])
def test_periodic_steps_match_oracle(images, prec, tol):
    """Six KDK steps of Eq. 2 (no background term, positions wrapped into the box)
    from a = 0.5 in EdS, with velocities that carry particles across the box
    faces.  Light particles and a large softening keep the six steps far from
    collapse or close encounters, which would amplify any difference ~10-100x per
    step and compare chaos rather than arithmetic."""
    L, n, dt = 2.0, 1500, 0.005
    pos, m, h = clumpy_box(77 + images, n, L)
    m = m * 1e-3      # dynamical time ~2, far longer than the six steps: no violent collapse
    h = np.random.default_rng(12).uniform(0.03, 0.06, n) * L
    vel = np.random.default_rng(9).normal(size=(n, 3)) * 0.5
    kd = oracle.KDKPeriodic(pos, vel, m, h, L, images, Om=1.0, OL=0.0, a0=0.5)
    sim = periodic_sim(pos, m, h, L, images, prec, vel=vel, a0=0.5, resort_every=3)
    for _ in range(6):
        kd.step(dt)
        sim.step(dt)
    p1, v1, _, t1, a1 = sim.state()
    assert np.all((p1 >= 0) & (p1 < L))
    assert a1 == pytest.approx(kd.a.value, rel=1e-12)
    d = p1 - kd.pos
    d -= L * np.round(d / L)                  # compare modulo the box
    crossed = np.any(np.abs(kd.pos - pos) > 0.5 * L, axis=1)
    assert crossed.sum() > 10
    # the force errors act on the displacement the accelerations (gravity and
    # friction) produce, x - x0 - v0 T, not on the ballistic part
    da = kd.pos - pos - vel * 6 * dt
    da = np.linalg.norm(da - L * np.round(da / L), axis=1)
    err = np.linalg.norm(d, axis=1) / np.maximum(da, 1e-2 * np.median(da))
    assert err.max() <= tol, err.max()
    sim.close()


@pytest.mark.parametrize("images", [0, 1])
def test_periodic_graph_run_equals_single_steps_bitwise(images):
    """steps_kdk_run replays captured steps (periodic force kernels, drift with
    the wrap into the box, re-sorts): bit-identical to single steps."""
    L, n = 2.0, 1500
    pos, m, h = clumpy_box(91 + images, n, L)
    m = m * 1e-3
    vel = np.random.default_rng(19).normal(size=(n, 3)) * 0.5
    dts = np.full(9, 0.005)
    s1 = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP, vel=vel, a0=0.5, resort_every=4)
    s2 = periodic_sim(pos, m, h, L, images, steps.STEPS_F32_COMP, vel=vel, a0=0.5, resort_every=4)
    for dt in dts:
        s1.step(dt)
    s2.run(dts)
    r1, r2 = s1.state(), s2.state()
    for x1, x2 in zip(r1[:3], r2[:3]):
        assert np.array_equal(x1, x2)
    assert r1[3] == r2[3] and r1[4] == r2[4]
    s1.close()
    s2.close()


def test_periodic_configuration_errors():
    pos, m, h = clumpy_box(1, 200, 1.0)
    for kw, status in ((dict(box=0.0), steps.STEPS_EINVAL), (dict(box=1.0, images=2), steps.STEPS_EINVAL),
                       (dict(box=1.0, prec=steps.STEPS_F32_NAIVE), steps.STEPS_EUNSUPPORTED)):
        args = dict(mode=steps.STEPS_PERIODIC, prec=steps.STEPS_F32_COMP, Om=1.0, OL=0.0)
        args.update(kw)
        with pytest.raises(steps.StepsError) as e:
            steps.Simulation(pos, np.zeros_like(pos), m, soft=h, cfg=steps.make_config(**args))
        assert e.value.status == status
    sim = periodic_sim(pos, m, h, 1.0, 0, steps.STEPS_F32_COMP)
    with pytest.raises(steps.StepsError) as e:
        steps.steps_forces_subset(sim.ctx, np.arange(4))
    assert e.value.status == steps.STEPS_EUNSUPPORTED
    sim.close()
