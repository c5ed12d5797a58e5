"""GPU parity of the adaptive step length (Eq. 12) and of adaptive KDK runs.

The device computes dt = min(dt_max, min_i sqrt(2 * 2.8 h_i * eps / |A_i|))
with a block-min reduction over the kick's acceleration; the oracle does the
same sum of the definition in FP64 on the CPU.  With FP64 forces the two agree
to rounding (1e-12); with FP32 compensated forces dt inherits half the
relative error of the limiting particle's acceleration (per-element force
bound 2e-5), so 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05903_gb300 import steps, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    steps.load(build_if_missing=True)


def make_sim(p, prec, resort_every=8):
    cfg = steps.make_config(mode=steps.STEPS_COMOVING if p.comoving else steps.STEPS_STATIC,
                            prec=prec, G=p.G, Om=p.Om, OL=p.OL, resort_every=resort_every)
    return steps.Simulation(p.pos, p.vel, p.mass, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfg)


def oracle_kdk(p):
    h = oracle.softening(p.mass, p.h_min)
    c = oracle.cosmo(G=p.G, Om=p.Om, OL=p.OL, comoving=p.comoving)
    return oracle.KDK(p.pos, p.vel, p.mass, h, c, a0=p.a0, t0=p.t0)


@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-12), (steps.STEPS_F32_COMP, 1e-5)])
def test_timestep_static_ball(prec, tol):
    p = workloads.static_ball(seed=1)
    kd = oracle_kdk(p)
    sim = make_sim(p, prec)
    for eps in (1e-3, 0.02):
        want = kd.timestep(eps, 1e9)
        got = sim.timestep(eps, 1e9)
        assert got == pytest.approx(want, rel=tol), (eps, got, want)
    # dt_max and the time left limit it; past t_end the step is 0
    assert sim.timestep(0.02, 1e-7) == 1e-7
    assert sim.timestep(0.02, 1e9, t_end=p.t0 + 2e-6) == pytest.approx(2e-6, rel=1e-12)
    assert sim.timestep(0.02, 1e9, t_end=p.t0 - 1.0) == 0.0
    sim.close()


@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-12), (steps.STEPS_F32_COMP, 1e-5)])
def test_timestep_comoving_with_velocities(prec, tol):
    """Compactified set with Zel'dovich velocities: friction and background terms
    enter |A_i|, and the limiting particle is found among 16,384."""
    p = workloads.compactified(31, 8192, 64, 128)
    kd = oracle_kdk(p)
    sim = make_sim(p, prec)
    want = kd.timestep(0.01, 1e9)
    got = sim.timestep(0.01, 1e9)
    assert got == pytest.approx(want, rel=tol), (got, want)
    sim.close()


@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-10), (steps.STEPS_F32_COMP, 2e-5)])
def test_adaptive_run_matches_oracle(prec, tol):
    """Eight adaptive KDK steps (device-chosen lengths, graph-replayed) against the
    oracle taking Eq. 12 then Eq. 11 at every step; the sixth step is cut at t_end
    and the last two have length 0."""
    p = workloads.static_ball(seed=1)
    eps, dt_max = 0.02, 5e-3
    probe = oracle_kdk(p)
    dts = [probe.adaptive_step(eps, dt_max) for _ in range(6)]
    t_end = p.t0 + sum(dts[:5]) + 0.5 * dts[5]
    kd = oracle_kdk(p)
    for _ in range(8):
        kd.adaptive_step(eps, dt_max, t_end)
    sim = make_sim(p, prec, resort_every=3)
    t = sim.run_adaptive(8, eps, dt_max, t_end)
    assert t == pytest.approx(t_end, rel=1e-14)
    assert kd.t.value == pytest.approx(t_end, rel=1e-14)
    pos, vel, _, _, _ = sim.state()
    moved = np.linalg.norm(kd.pos - p.pos, axis=1)
    e = np.linalg.norm(pos - kd.pos, axis=1) / np.maximum(moved, 1e-300)
    assert e.max() <= tol, e.max()
    dv = np.linalg.norm(kd.vel - p.vel, axis=1)
    ev = np.linalg.norm(vel - kd.vel, axis=1) / np.maximum(dv, 1e-300)
    assert ev.max() <= 10 * tol, ev.max()
    sim.close()


def test_adaptive_run_equals_host_driven_steps():
    """steps_kdk_run_adaptive (device-chosen dt, graph replay) is bitwise the same
    as host-driven steps_timestep + steps_kdk_step with the returned dt."""
    p = workloads.compactified(32, 4096, 16, 128)
    a = make_sim(p, steps.STEPS_F32_COMP, resort_every=4)
    b = make_sim(p, steps.STEPS_F32_COMP, resort_every=4)
    a.run_adaptive(10, 0.01, 1e-2)
    for _ in range(10):
        b.step(b.timestep(0.01, 1e-2))
    sa, sb = a.state(), b.state()
    for x, y in zip(sa[:3], sb[:3]):
        assert np.array_equal(x, y)
    assert sa[3] == sb[3] and sa[4] == sb[4]
    a.close()
    b.close()


@pytest.mark.parametrize("eps,dt_max,t_end", [(0.0, 1.0, math.inf), (-1.0, 1.0, math.inf), (0.01, 0.0, math.inf),
                                              (0.01, math.inf, math.inf), (0.01, 1.0, math.nan),
                                              (math.nan, 1.0, math.inf)])
def test_timestep_rejects_bad_arguments(eps, dt_max, t_end):
    p = workloads.static_ball(seed=1, n_ball=256, n_shells=2, per_shell=32)
    sim = make_sim(p, steps.STEPS_F32_COMP)
    with pytest.raises(steps.StepsError) as e:
        sim.timestep(eps, dt_max, t_end)
    assert e.value.status == steps.STEPS_EINVAL
    with pytest.raises(steps.StepsError):
        sim.run_adaptive(2, eps, dt_max, t_end)
    sim.close()
