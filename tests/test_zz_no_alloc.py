"""The allocation-free force entry point, checked against the regular one.

steps_forces_noalloc is meant for callers that cannot allocate device memory
around a force evaluation (an application whose caching allocator already
holds the memory, or a step loop that must not take cudaMalloc's implicit
synchronisation).  It must give the same pair term as steps_init +
steps_forces, within the tolerance the other force tests use, on two calls in
a row -- the second call reuses the fixed scratch left behind by the first.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_1811_05903_gb300 import steps, workloads

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-6
MAX_TOL = 2e-5


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("n_central,n_shells,per_shell", [(4096, 16, 128), (3000, 8, 77)])
def test_noalloc_matches_regular_entry_point_twice(n_central, n_shells, per_shell):
    import torch
    assert torch.cuda.is_available()
    steps.load(build_if_missing=True)
    p = workloads.compactified(71, n_central, n_shells, per_shell)
    assert p.n <= steps.STEPS_NOALLOC_MAX_N
    # the regular entry point run with the kernel variant the allocation-free
    # one uses (64-particle tiles, explicit separations), so that both sides
    # make the same FP32 roundings up to the order of the partial sums
    k = steps.steps_variants().index("comp_ki2_w8_u4") + 1
    cfg = steps.make_config(mode=steps.STEPS_COMOVING, prec=steps.STEPS_F32_COMP, Om=p.Om, OL=p.OL,
                            tile_override=k)
    sim = steps.Simulation(p.pos, p.vel, p.mass, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfg)
    ref = sim.forces()
    sim.close()

    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(np.ascontiguousarray(p.pos)).to(dev)
    mass = torch.from_numpy(np.ascontiguousarray(p.mass)).to(dev)
    outs = []
    for _ in range(2):
        acc = torch.full((p.n, 3), float("nan"), dtype=torch.float64, device=dev)
        steps.steps_forces_noalloc(pos, mass, acc, h_min=p.h_min, G=p.G)
        outs.append(acc.cpu().numpy())
    for a in outs:
        e = rel_err(a, ref)
        assert np.isfinite(a).all()
        assert np.sqrt(np.mean(e ** 2)) <= RMS_TOL and e.max() <= MAX_TOL, (np.sqrt(np.mean(e ** 2)), e.max())
    # deterministic: the second call over the reused scratch repeats the first bit for bit
    assert np.array_equal(outs[0], outs[1])
    # and both equal the FP64 oracle's pair term within the same contract
    h = oracle.softening(p.mass, p.h_min)
    ora = oracle.pair_acc(p.pos, p.mass, h, p.G)
    e = rel_err(outs[0], ora)
    assert np.sqrt(np.mean(e ** 2)) <= RMS_TOL and e.max() <= MAX_TOL, (np.sqrt(np.mean(e ** 2)), e.max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    steps.load(build_if_missing=True)
    n = steps.STEPS_NOALLOC_MAX_N + 1
    dev = torch.device("cuda", 0)
    pos = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    mass = torch.ones(n, dtype=torch.float64, device=dev)
    acc = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(steps.StepsError) as e:
        steps.steps_forces_noalloc(pos, mass, acc, h_min=0.01)
    assert e.value.status == steps.STEPS_EINVAL
    assert "outside" in str(e.value)


def test_noalloc_rejects_host_pointers():
    """Host buffers are refused before any GPU work (the entry point takes
    device memory of the current device only)."""
    steps.load(build_if_missing=True)
    n = 64
    pos = np.zeros((n, 3))
    mass = np.ones(n)
    acc = np.zeros((n, 3))
    with pytest.raises(steps.StepsError) as e:
        steps.steps_forces_noalloc(pos, mass, acc, h_min=0.01)
    assert e.value.status == steps.STEPS_EINVAL
    assert "device pointers" in str(e.value)
