"""GPU parity of the FP64 KDK integrator (Eq. 9-11) with the comoving
acceleration (Eq. 8) and the RK4 scale factor (Eq. 1), plus determinism,
checkpoint/resume, diagnostics and the failure paths of the C ABI."""
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


def make_sim(p, prec=steps.STEPS_F32_COMP, resort_every=8, soft=None):
    cfg = steps.make_config(mode=steps.STEPS_COMOVING if p.comoving else steps.STEPS_STATIC,
                            prec=prec, G=p.G, Om=p.Om, OL=p.OL, resort_every=resort_every)
    return steps.Simulation(p.pos, p.vel, p.mass, soft=soft, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfg)


def traj_err(x, ref, x0):
    """Per-particle position error relative to how far the particle moved."""
    moved = np.linalg.norm(ref - x0, axis=1)
    return np.linalg.norm(x - ref, axis=1) / np.maximum(moved, 1e-300)


@pytest.mark.parametrize("prec,tol", [(steps.STEPS_F64, 1e-10), (steps.STEPS_F32_COMP, 2e-5)])
def test_static_ball_ten_steps(prec, tol):
    p = workloads.static_ball(seed=1)
    h = oracle.softening(p.mass, p.h_min)
    kd = oracle.KDK(p.pos, p.vel, p.mass, h, oracle.cosmo(comoving=False))
    sim = make_sim(p, prec)
    for _ in range(10):
        kd.step(1e-3)
        sim.step(1e-3)
    pos, vel, acc, t, a = sim.state()
    sim.close()
    e = traj_err(pos, kd.pos, p.pos)
    assert np.sqrt(np.mean(e ** 2)) <= tol / 10 and e.max() <= tol, (np.sqrt(np.mean(e ** 2)), e.max())
    assert abs(t - 0.01) < 1e-15


def test_comoving_steps_and_scale_factor():
    p = workloads.compactified(31, 4096, 32, 64)
    h = oracle.softening(p.mass, p.h_min)
    c = oracle.cosmo(Om=p.Om, OL=p.OL, comoving=True)
    a_sched, dts = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
    kd = oracle.KDK(p.pos, p.vel, p.mass, h, c, a0=p.a0, t0=p.t0)
    sim = make_sim(p, steps.STEPS_F64)
    sim32 = make_sim(p, steps.STEPS_F32_COMP)
    for k in range(6):
        kd.step(dts[k])
        a_gpu = sim.step(dts[k], want_a=True)
        sim32.step(dts[k])
        assert abs(a_gpu - kd.a.value) <= 1e-14 * kd.a.value
        assert abs(a_gpu - a_sched[k + 1]) <= 1e-9 * a_sched[k + 1]
    pos, vel, acc, t, a = sim.state()
    pos32, vel32, _, _, _ = sim32.state()
    e = traj_err(pos, kd.pos, p.pos)
    assert e.max() <= 1e-9, e.max()
    e32 = traj_err(pos32, kd.pos, p.pos)
    assert e32.max() <= 1e-5, e32.max()
    ev = np.linalg.norm(vel - kd.vel, axis=1) / np.linalg.norm(kd.vel, axis=1)
    assert ev.max() <= 1e-9
    sim.close()
    sim32.close()


def test_run_graph_equals_single_steps_bitwise():
    p = workloads.compactified(41, 3000, 16, 64)
    a_sched, dts = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
    s1 = make_sim(p, resort_every=4)
    s2 = make_sim(p, resort_every=4)
    for k in range(11):
        s1.step(dts[k])
    s2.run(dts[:11])
    r1, r2 = s1.state(), s2.state()
    for x1, x2 in zip(r1[:3], r2[:3]):
        assert np.array_equal(x1, x2)
    assert r1[3] == r2[3] and r1[4] == r2[4]
    s1.close()
    s2.close()


def test_checkpoint_resume_is_bit_identical():
    p = workloads.compactified(51, 3000, 16, 64)
    _, dts = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
    ref = make_sim(p, resort_every=3)
    ref.run(dts[:5])
    blob = steps.steps_checkpoint_save(ref.ctx)
    ref.run(dts[5:12])
    other = make_sim(p, resort_every=3)
    steps.steps_checkpoint_load(other.ctx, blob)
    other.run(dts[5:12])
    for x1, x2 in zip(ref.state(), other.state()):
        assert np.array_equal(np.asarray(x1), np.asarray(x2))
    ref.close()
    other.close()


def test_diagnostics_match_oracle():
    p = workloads.static_ball(seed=1)
    h = oracle.softening(p.mass, p.h_min)
    sim = make_sim(p, steps.STEPS_F64)
    for _ in range(3):
        sim.step(1e-3)
    pos, vel, _, _, _ = sim.state()
    ek, ep, mom = steps.steps_diagnostics(sim.ctx)
    ek_ref, mom_ref = oracle.kinetic(vel, p.mass)
    ep_ref = oracle.pair_potential(pos, p.mass, h, p.G)
    assert abs(ek - ek_ref) <= 1e-12 * ek_ref
    assert abs(ep - ep_ref) <= 1e-12 * abs(ep_ref)
    assert np.all(np.abs(mom - mom_ref) <= 1e-12 * (p.mass.sum() * np.abs(vel).max()))
    sim.close()


def test_static_energy_second_order_on_gpu():
    p = workloads.static_ball(seed=1)
    des = []
    for dt in (1e-3, 5e-4):
        sim = make_sim(p, steps.STEPS_F32_COMP)
        ek0, ep0, _ = steps.steps_diagnostics(sim.ctx)
        for _ in range(int(round(0.01 / dt))):
            sim.step(dt)
        ek, ep, mom = steps.steps_diagnostics(sim.ctx)
        des.append(abs((ek + ep) - (ek0 + ep0)) / abs(ek0 + ep0))
        sim.close()
    assert des[0] < 1e-3 and 3.5 < des[0] / des[1] < 4.5, des


def test_wait_limit_timeout_path_and_recovery():
    p = workloads.compactified(61, 4096, 16, 64)
    sim = make_sim(p)
    steps.steps_set_wait_limit(sim.ctx, 0)       # every bounded wait gives up at once
    with pytest.raises(steps.StepsError) as e:
        sim.forces()
    assert e.value.status == steps.STEPS_ETIMEOUT
    steps.steps_set_wait_limit(sim.ctx, 2_000_000_000)
    h = oracle.softening(p.mass, p.h_min)
    ref = oracle.pair_acc(p.pos, p.mass, h, p.G)
    acc = sim.forces()
    e = np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.sqrt(np.mean(e ** 2)) <= 1e-6
    sim.close()


def test_memory_limit_gives_enomem():
    p = workloads.static_ball(seed=1, n_ball=256, n_shells=2, per_shell=32)
    steps.steps_set_memory_limit(4096)
    try:
        with pytest.raises(steps.StepsError) as e:
            make_sim(p)
        assert e.value.status == steps.STEPS_ENOMEM
    finally:
        steps.steps_set_memory_limit(0)
    make_sim(p).close()


@pytest.mark.parametrize("what", ["nan_pos", "zero_mass", "neg_soft", "inf_vel"])
def test_invalid_inputs_rejected(what):
    p = workloads.static_ball(seed=1, n_ball=256, n_shells=2, per_shell=32)
    pos, vel, m = p.pos.copy(), p.vel.copy(), p.mass.copy()
    soft = None
    if what == "nan_pos":
        pos[5, 1] = np.nan
    elif what == "zero_mass":
        m[3] = 0.0
    elif what == "neg_soft":
        soft = np.full(p.n, 0.01)
        soft[7] = -1.0
    elif what == "inf_vel":
        vel[2, 0] = np.inf
    with pytest.raises(steps.StepsError) as e:
        steps.Simulation(pos, vel, m, soft=soft, h_min=p.h_min)
    assert e.value.status == steps.STEPS_EINVAL


def test_config2_full_run_forces_stay_within_contract():
    """The StePS-like compactified LCDM run of N = 262,144 (131,072 central
    particles + 64 shells x 2,048) taken through all 200 log-a KDK steps from
    a = 0.02 to a = 1 in the graph-replayed loop.  Trajectories are chaotic, so
    the run is checked where the oracle can follow it one target at a time: the
    scale factor reaches 1 (RK4 against the closed form), the state stays
    finite, and the mixed-precision pair term on 512 seeded targets of the
    evolved, clustered state meets the same contract as on the initial state."""
    import time
    p = workloads.lcdm_262k()
    a_sched, dts = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
    sim = make_sim(p)
    t0 = time.perf_counter()
    sim.run(dts)
    pos, vel, acc, t, a = sim.state()
    secs = time.perf_counter() - t0
    sim.close()
    print("262,144 particles, 200 steps: %.2f s, %.3e interactions/s" % (secs, 200 * p.n ** 2 / secs))
    assert abs(a - 1.0) <= 1e-9
    assert np.isfinite(pos).all() and np.isfinite(vel).all() and np.isfinite(acc).all()
    h = oracle.softening(p.mass, p.h_min)
    tg = np.sort(np.random.default_rng(2002).choice(p.n, 512, replace=False))
    ref = oracle.pair_acc(pos, p.mass, h, p.G, targets=tg)
    e = np.linalg.norm(acc[tg] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(e ** 2))
    print("evolved state: rms %.2e max %.2e" % (rms, e.max()))
    assert rms <= 1e-6 and e.max() <= 2e-5, (rms, e.max())
