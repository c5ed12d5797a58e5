"""GPU parity of the spherical-glass path (Sec. 3.1): shell placement
(Eq. 14-18) against the oracle from the same uniform random numbers, KDK
steps under reversed gravity (Eq. 8 with both gravity terms negated) against
the oracle, and the relaxation's purpose -- a much smaller net force.

Tolerances: placement is FP64 bisection on 2w - sin 2w plus trigonometry on
both sides; the device and host sin/tan differ by an ulp or two, which moves a
root by ~1e-12 relative where the compact-volume density sin^2 w is small, so
positions are compared to 1e-9 relative and masses to 1e-12.  Reversed steps use
the integrator tests' bounds (1e-10 for FP64 forces, 2e-5 for FP32).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import glass as og
from paper_1811_05903_gb300 import glass, steps

pytestmark = pytest.mark.gpu

RHO = glass.RHO_EDS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    steps.load(build_if_missing=True)


@pytest.mark.parametrize("scheme,D,R,nr,ns,rc", [(0, 60.0, 342.45, 24, 300, 45.0), (1, 100.0, 342.45, 30, 257, 0.0)])
def test_placement_matches_oracle(scheme, D, R, nr, ns, rc):
    spec = steps.glass_spec(scheme, D, R, nr, ns, rc, RHO)
    n = steps.steps_glass_layout(spec)[0]
    n_inner = steps.steps_glass_layout(spec)[1]
    u = np.random.default_rng(100 + scheme).random((n, 3))
    # draws on the edges of shell 3 (and the centre of the inner ball)
    k = n_inner + 3 * ns
    u[k:k + 5, 0] = [0.0, 0.5, 1 - 1e-12, 1 - 2.0 ** -53, 0.25]
    if n_inner:
        u[:2, 0] = [0.0, 1e-300]
    pos, mass = steps.steps_glass_place(spec, u)
    ref_pos, ref_mass = og.place(scheme, D, R, nr, ns, rc, RHO, u)
    np.testing.assert_allclose(mass, ref_mass, rtol=1e-12)
    scale = np.maximum(np.linalg.norm(ref_pos, axis=1), 1e-300)
    err = np.linalg.norm(pos - ref_pos, axis=1) / scale
    assert err.max() <= 1e-9, err.max()


def test_placement_from_device_buffers_and_size_check():
    import torch
    spec = steps.glass_spec(1, 50.0, 200.0, 6, 128, 0.0, RHO)
    n = steps.steps_glass_layout(spec)[0]
    u = torch.rand((n, 3), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    pos = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.empty(n, dtype=torch.float64, device="cuda")
    steps.steps_glass_place(spec, u, pos, mass)
    ref_pos, ref_mass = og.place(1, 50.0, 200.0, 6, 128, 0.0, RHO, u.cpu().numpy())
    np.testing.assert_allclose(pos.cpu().numpy(), ref_pos, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(mass.cpu().numpy(), ref_mass, rtol=1e-12)
    with pytest.raises(steps.StepsError) as e:
        steps.steps_glass_place(spec, np.zeros((n + 1, 3)))
    assert e.value.status == steps.STEPS_EINVAL


@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-10), (steps.STEPS_F32_COMP, 2e-5)])
def test_reversed_gravity_steps_match_oracle(prec, tol):
    pos, mass = glass.place(0, 60.0, 300.0, 10, 200, 40.0, RHO, seed=5)
    h_min = glass.default_h_min(pos, mass)
    h = oracle.softening(mass, h_min)
    a0 = 0.1
    t = glass.eds_time(np.geomspace(a0, 0.2, 9))
    kd = oracle.KDK(pos, np.zeros_like(pos), mass, h, oracle.cosmo(Om=1.0, OL=0.0, reversed=True), a0=a0,
                    t0=float(t[0]))
    cfg = steps.make_config(mode=steps.STEPS_COMOVING_REVERSED, prec=prec, G=1.0, Om=1.0, OL=0.0, resort_every=3)
    sim = steps.Simulation(pos, np.zeros_like(pos), mass, h_min=h_min, t0=float(t[0]), a0=a0, cfg=cfg)
    # the reversed pair term is the ordinary one negated
    acc = sim.forces()
    ref = oracle.pair_acc(pos, mass, h, -1.0)
    e = np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert e.max() <= (1e-12 if prec == steps.STEPS_F64 else 2e-5)
    for dt in np.diff(t):
        kd.step(float(dt))
    sim.run(np.diff(t))
    p1, v1, _, t1, a1 = sim.state()
    assert t1 == pytest.approx(kd.t.value, rel=1e-14) and a1 == pytest.approx(kd.a.value, rel=1e-12)
    moved = np.linalg.norm(kd.pos - pos, axis=1)
    err = np.linalg.norm(p1 - kd.pos, axis=1) / np.maximum(moved, 1e-300)
    assert err.max() <= tol, err.max()
    sim.close()


@pytest.mark.parametrize("scheme,rc", [(0, 40.0), (1, 0.0)])
def test_relaxation_reduces_the_net_force(scheme, rc):
    """Sec. 3.1's purpose: after relaxing under reversed gravity the net
    (ordinary-gravity) force on the particles away from the outer edge is far
    smaller than for the random placement; the oracle, run on a 2,000-particle
    version of the same recipe, gives ratios 0.09 and 0.22."""
    D, R, nr, ns = 60.0, 300.0, 16, 1024
    pos0, mass = glass.place(scheme, D, R, nr, ns, rc, RHO, seed=7)
    h_min = glass.default_h_min(pos0, mass)
    pos1 = glass.relax(pos0, mass, h_min, a_start=0.1, a_end=1.0, nsteps=100)
    f0 = glass.peculiar_acceleration(pos0, mass, h_min)
    f1 = glass.peculiar_acceleration(pos1, mass, h_min)
    inner0 = np.linalg.norm(pos0, axis=1) < 0.6 * R
    inner1 = np.linalg.norm(pos1, axis=1) < 0.6 * R
    ratio = math.sqrt(np.mean(f1[inner1] ** 2) / np.mean(f0[inner0] ** 2))
    print("scheme %d: n=%d rms net force relaxed/random = %.3f" % (scheme, pos0.shape[0], ratio))
    assert np.isfinite(pos1).all()
    assert ratio < 0.35, ratio
