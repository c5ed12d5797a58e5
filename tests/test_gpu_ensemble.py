"""GPU parity of the batched ensemble (many independent simulations advanced
together in one force launch per step) against the FP64 oracle run member by
member: initial forces, then KDK trajectories with per-member cosmologies,
step schedules, a re-sorting step and CUDA-graph replays."""
import numpy as np
import pytest

import oracle
from paper_1811_05903_gb300 import steps, workloads

pytestmark = pytest.mark.gpu


def members():
    ps = [workloads.compactified(81, 3000, 16, 64, Om=0.26, OL=0.74),
          workloads.compactified(82, 1200, 8, 50, Om=0.33, OL=0.67, disp_frac=0.02),
          workloads.static_ball(seed=83, n_ball=700, n_shells=4, per_shell=40),
          workloads.compactified(84, 5000, 32, 96, Om=0.30, OL=0.70)]
    return ps


def cfg_for(p):
    return steps.make_config(mode=steps.STEPS_COMOVING if p.comoving else steps.STEPS_STATIC,
                             prec=steps.STEPS_F32_COMP, G=p.G, Om=p.Om, OL=p.OL, resort_every=3)


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


@pytest.fixture(scope="module")
def ens():
    import torch
    assert torch.cuda.is_available()
    steps.load(build_if_missing=True)
    ps = members()
    e = steps.Ensemble(ps, [cfg_for(p) for p in ps])
    yield ps, e
    e.close()


def test_ensemble_initial_forces_match_oracle_per_member(ens):
    ps, e = ens
    for s, p in enumerate(ps):
        h = oracle.softening(p.mass, p.h_min)
        ref = oracle.pair_acc(p.pos, p.mass, h, p.G)
        _, _, acc, t, a = e.state(s)
        err = rel(acc, ref)
        assert np.sqrt(np.mean(err ** 2)) <= 1e-6 and err.max() <= 2e-5, (s, np.sqrt(np.mean(err ** 2)), err.max())
        assert t == p.t0 and (a == p.a0 or not p.comoving)


def test_ensemble_trajectories_match_oracle_per_member(ens):
    ps, e = ens
    nsteps = 5
    dts = np.empty((len(ps), nsteps))
    refs = []
    for s, p in enumerate(ps):
        h = oracle.softening(p.mass, p.h_min)
        if p.comoving:
            _, dt = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
            dts[s] = dt[:nsteps]
            c = oracle.cosmo(Om=p.Om, OL=p.OL, comoving=True)
        else:
            dts[s] = 1e-3
            c = oracle.cosmo(comoving=False)
        kd = oracle.KDK(p.pos, p.vel, p.mass, h, c, a0=p.a0, t0=p.t0)
        for k in range(nsteps):
            kd.step(dts[s, k])
        refs.append(kd)
    e.run(dts)  # crosses a re-sort (every 3 steps) and replays the captured step
    for s, (p, kd) in enumerate(zip(ps, refs)):
        pos, vel, acc, t, a = e.state(s)
        moved = np.linalg.norm(kd.pos - p.pos, axis=1)
        err = np.linalg.norm(pos - kd.pos, axis=1) / np.maximum(moved, 1e-300)
        assert err.max() <= 2e-5, (s, err.max())
        assert abs(t - kd.t.value) <= 1e-12 * max(1.0, abs(kd.t.value))
        if p.comoving:
            assert abs(a - kd.a.value) <= 1e-14 * kd.a.value


def test_ensemble_rejects_bad_members():
    steps.load(build_if_missing=True)
    p = workloads.static_ball(seed=85, n_ball=100, n_shells=2, per_shell=20)
    bad = workloads.Particles(pos=p.pos.copy(), vel=p.vel, mass=p.mass.copy(), h_min=p.h_min)
    bad.mass[3] = -1.0
    with pytest.raises(steps.StepsError) as ex:
        steps.Ensemble([p, bad], [cfg_for(p), cfg_for(bad)])
    assert ex.value.status == steps.STEPS_EINVAL
