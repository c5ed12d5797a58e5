"""Benchmark: pair interactions/s of the StePS direct-summation step on GB300.

Workload (default): the N = 2^20 compactified precision-study set (524,288
central particles in 50 Mpc/h + 64 shells x 8,192 out to 4,000 Mpc/h),
comoving LambdaCDM, FP32 pair arithmetic with tile-relative coordinates and
compensated sums, FP64 integrator.  One step = one full kick-drift-kick step
(kick, drift, RK4 a(t), staging, pair-force kernel, fixup, kick; spatial
re-sort every 8 steps), i.e. N^2 pair interactions.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead;
--ensemble-only and --periodic-only time the batched ensemble or the
periodic-mode force evaluations alone (their own JSON line, not the bench line).
Multi-GPU (torchrun): the path does not shard; each rank runs an independent
replica and the job value is the sum of all ranks' interactions over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair interactions/s at N=2^20: mixed vs FP64 GPU at <=1e-6 rms rel force err"
UNIT = "interactions/s"
FLOP_PER_INTERACTION = 20  # the usual direct N-body convention
FP64_FMA_PER_SM_CLK = 2    # GB300 FP64 pipe: 2 DFMA per SM and cycle (ncu's peak table)
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one far-field
# launch, measured by ncu (one pass, the launch-list run of this bench command)
# for the named variant at the named size, with the kernel source as committed
# alongside; any other variant or size reports null.
FAR_TRAFFIC_BYTES = {("sym_ki8s_w4", 1048576): 64_272_000,  # mean of 13 launches, 64.06-64.59 MB
                     ("sym_ki8_w4", 1048576): 61_091_000}   # mean of 4 launches, 60.93-61.23 MB


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flop x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, r in rows:
            for nm, v in zip(names, r[1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(local_seconds: float, units_per_rank: float, device=None):
    """Whole-job value of independent replicas: the units every rank processed
    over the slowest rank's time (max over ranks); (value, seconds).  A single
    process (no process group) is its own job."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    seconds = float(local_seconds)
    if ws > 1:
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return units_per_rank * ws / seconds, seconds


def build_workload(name: str):
    from paper_1811_05903_gb300 import workloads
    if name == "precision_1m":
        return workloads.precision_1m(), "StePS compactified LCDM, N=1,048,576 (524,288 central in 50 Mpc/h + 64 shells x 8,192 to 4,000 Mpc/h), a=0.02"
    if name == "lcdm_262k":
        return workloads.lcdm_262k(), "StePS compactified LCDM, N=262,144 (131,072 central + 64 shells x 2,048), a=0.02"
    raise SystemExit("unknown workload " + name)


def run_reference(args):
    """The FP64 CPU oracle on a bounded sample of the same workload."""
    import oracle
    from paper_1811_05903_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    p, desc = build_workload(args.workload)
    h = oracle.softening(p.mass, p.h_min)
    nt = args.ref_targets
    rng = np.random.default_rng(12345)
    for _ in range(args.warmup):
        oracle.pair_acc(p.pos, p.mass, h, p.G, targets=np.sort(rng.choice(p.n, nt, replace=False)))
    times = []
    for _ in range(args.steps):
        tg = np.sort(rng.choice(p.n, nt, replace=False))
        t0 = time.perf_counter()
        oracle.pair_acc(p.pos, p.mass, h, p.G, targets=tg)
        times.append(time.perf_counter() - t0)
    value = args.steps * nt * p.n / sum(times)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "n": p.n, "sample_targets": nt},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d seeded targets x all %d sources per step (FP64 direct sum, OpenMP)" % (nt, p.n)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ensemble_throughput(stream, steps_mod, workloads_mod):
    """Config 4: 64 compactified members (uneven N, differing Om and sigma8)
    advanced together in one ensemble vs the same members run one after
    another; both arms time the complete 100-step runs (CUDA events), after
    initialisation (which includes each arm's autotuning)."""
    import torch
    ens = workloads_mod.ensemble(seed=4)
    ps = ens.sims
    nsteps_run = 100
    cfgs = [steps_mod.make_config(mode=steps_mod.STEPS_COMOVING, prec=steps_mod.STEPS_F32_COMP, G=p.G,
                                  Om=p.Om, OL=p.OL, resort_every=8) for p in ps]
    dts = np.stack([workloads_mod.loga_schedule(p.a0, 1.0, nsteps_run, p.Om, p.OL)[1] for p in ps])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e = steps_mod.Ensemble(ps, cfgs, stream=stream.cuda_stream)
    variant = steps_mod.steps_variants()[e.variant()]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
    e.run(dts)
    with torch.cuda.stream(stream):
        ev1.record(stream)
    ev1.synchronize()
    t_ens = ev0.elapsed_time(ev1) * 1e-3
    total, nnear, nall = e.stats()
    e.close()
    t_seq = 0.0
    seq_variants = set()
    for s, p in enumerate(ps):
        sim = steps_mod.Simulation(p.pos, p.vel, p.mass, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfgs[s],
                                   stream=stream.cuda_stream)
        seq_variants.add(steps_mod.steps_variants()[steps_mod.steps_get_variant(sim.ctx)])
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
        sim.run(dts[s])
        with torch.cuda.stream(stream):
            ev1.record(stream)
        ev1.synchronize()
        t_seq += ev0.elapsed_time(ev1) * 1e-3
        sim.close()
    inter = float(sum(int(p.n) ** 2 for p in ps)) * nsteps_run
    return {"workload": "64 compactified LCDM members, N ~ U[8192, 131072] (sum %d), Om ~ U[0.25, 0.35], "
                        "sigma8 ~ U[0.7, 0.9], 100 KDK steps from a = 0.02 to 1" % sum(p.n for p in ps),
            "sims_per_hour": len(ps) * 3600.0 / t_ens,
            "sims_per_hour_sequential": len(ps) * 3600.0 / t_seq,
            "batched_over_sequential": t_seq / t_ens,
            "run_s": t_ens, "run_s_sequential": t_seq,
            "ms_per_step": 1e3 * t_ens / nsteps_run, "ms_per_step_sequential": 1e3 * t_seq / nsteps_run,
            "interactions_per_s": inter / t_ens, "timed_steps": nsteps_run,
            "variant": variant, "variants_sequential": sorted(seq_variants),
            "near_field_fraction": nnear / max(nall, 1)}


def periodic_throughput(steps_mod, n=16384, L=1.0, seed=21):
    """Periodic mode (Eq. 2 with Eq. 5): one FP32 force evaluation of a uniform
    random box, cut image sum (|x - nL| < 2.6 L) and quasi-periodic; CUDA events
    around the force kernels.  Work counted as N^2 x (4 pi / 3) 2.6^3 pair-image
    terms for the cut sum (the expected number of images inside the cut sphere)
    and N^2 for the quasi-periodic sum."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = fp32_peak_tflops(props.multi_processor_count, float(peaks().get("sm_max_mhz", 2070.0)))
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    m = np.full(n, 1.0 / n)
    h = np.full(n, 0.02 * L / n ** (1.0 / 3.0))
    out = {"workload": "uniform random box, N=%d, L=%g, FP32 compensated" % (n, L)}
    for images, name, terms in ((0, "cut_2p6L", 4.0 * math.pi / 3.0 * 2.6 ** 3), (1, "quasi", 1.0)):
        cfg = steps_mod.make_config(mode=steps_mod.STEPS_PERIODIC, prec=steps_mod.STEPS_F32_COMP, Om=1.0, OL=0.0,
                                    box=L, images=images)
        sim = steps_mod.Simulation(pos, np.zeros_like(pos), m, soft=h, cfg=cfg)
        steps_mod.steps_forces(sim.ctx)
        steps_mod.steps_profile_read(sim.ctx, reset=True)
        steps_mod.steps_profile_enable(sim.ctx, True)
        for _ in range(3):
            steps_mod.steps_forces(sim.ctx)
        far_ms, far_launches = steps_mod.steps_profile_read_far(sim.ctx)
        ms, launches, _ = steps_mod.steps_profile_read(sim.ctx, reset=True)
        sim.close()
        per = ms * 1e-3 / max(launches, 1)
        far = far_ms * 1e-3 / max(far_launches, 1)
        tflops = 20 * terms * n * n / per / 1e12
        out[name] = {"ms_per_evaluation": 1e3 * per, "pair_image_terms_per_s": terms * n * n / per,
                     "fp32_tflops_at_20_flop": tflops, "frac_of_fp32_peak": tflops / peak,
                     # the image kernel alone (the symmetric kernel; the per-target one keeps softened images)
                     "kernel": "psym_far_kernel",
                     "kernel_ms": 1e3 * far, "kernel_share": far / per if per > 0 else None}
    return out


def cpu_workloads(stream, steps_mod, workloads_mod):
    """The FP64 oracle on the host cores on the planned baseline workloads:
    the small static system (4,096 particles) in full -- one force evaluation
    and 10 KDK steps at dt = 1e-3 -- and the N = 262,144 compactified LCDM run
    (200 steps from a = 0.02 to 1, advanced on the GPU) at three checkpoints,
    4,096 seeded targets each against all sources, with the GPU's error there."""
    import torch
    import oracle
    out = []
    p = workloads_mod.static_ball(seed=1)
    h = oracle.softening(p.mass, p.h_min)
    t0 = time.perf_counter()
    oracle.pair_acc(p.pos, p.mass, h, p.G)
    kd = oracle.KDK(p.pos, p.vel, p.mass, h, oracle.cosmo(comoving=False))
    for _ in range(10):
        kd.step(1e-3)
    dt_cpu = time.perf_counter() - t0
    inter = 11.0 * p.n * p.n  # the evaluation plus one per KDK step
    out.append({"workload": "static ball + 16 shells, N=%d: 1 force evaluation + 10 KDK steps" % p.n,
                "interactions_per_s": inter / dt_cpu, "s": dt_cpu})
    q = workloads_mod.lcdm_262k()
    hq = oracle.softening(q.mass, q.h_min)
    _, dts = workloads_mod.loga_schedule(q.a0, 1.0, 200, q.Om, q.OL)
    cfg = steps_mod.make_config(mode=steps_mod.STEPS_COMOVING, prec=steps_mod.STEPS_F32_COMP, G=q.G, Om=q.Om,
                                OL=q.OL, resort_every=8)
    sim = steps_mod.Simulation(q.pos, q.vel, q.mass, h_min=q.h_min, t0=q.t0, a0=q.a0, cfg=cfg,
                               stream=stream.cuda_stream)
    tg = workloads_mod.precision_targets(q.n)
    done = 0
    for stop in (0, 100, 200):
        if stop > done:
            sim.run(dts[done:stop])
            done = stop
        torch.cuda.synchronize()
        pos = np.empty((q.n, 3))
        acc = np.empty((q.n, 3))
        _, a_now = steps_mod.steps_get_state(sim.ctx, pos=pos, acc=acc)
        t0 = time.perf_counter()
        ref = oracle.pair_acc(pos, q.mass, hq, q.G, targets=tg)
        dt_cpu = time.perf_counter() - t0
        e = np.linalg.norm(acc[tg] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        out.append({"workload": "compactified LCDM N=%d after %d of 200 steps (a = %.3f): %d targets x all "
                                "sources" % (q.n, stop, a_now, tg.size),
                    "interactions_per_s": tg.size * q.n / dt_cpu, "s": dt_cpu,
                    "gpu_rms_rel_err": float(np.sqrt(np.mean(e ** 2))), "gpu_max_rel_err": float(e.max())})
    sim.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1811_05903_gb300.build as libbuild
    from paper_1811_05903_gb300 import steps, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    libbuild.build()
    steps.load()
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)

    p, desc = build_workload(args.workload)
    n = p.n
    a_sched, dts = workloads.loga_schedule(p.a0, 1.0, 200, p.Om, p.OL)
    stream = torch.cuda.Stream(device=dev)
    cfg = steps.make_config(mode=steps.STEPS_COMOVING, prec=steps.STEPS_F32_COMP, G=p.G, Om=p.Om, OL=p.OL,
                            resort_every=8, tile_override=args.variant)
    sim = steps.Simulation(p.pos, p.vel, p.mass, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfg,
                           stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    variant_name = steps.steps_variants()[steps.steps_get_variant(sim.ctx)]

    # ---- accuracy at the initial positions (mixed, naive, FP64 GPU) ----
    acc_mixed = np.empty((n, 3))
    steps.steps_get_state(sim.ctx, acc=acc_mixed)
    tg = workloads.precision_targets(n)
    acc64 = steps.steps_forces_subset(sim.ctx, tg)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    big_tg = np.sort(np.random.default_rng(7).choice(n, min(n, args.f64_targets), replace=False))
    with torch.cuda.stream(stream):
        ev0.record(stream)
    steps.steps_forces_subset(sim.ctx, big_tg)
    with torch.cuda.stream(stream):
        ev1.record(stream)
    ev1.synchronize()
    f64_ms = ev0.elapsed_time(ev1)
    f64_rate = big_tg.size * n / (f64_ms * 1e-3)

    cfg_naive = steps.make_config(mode=steps.STEPS_COMOVING, prec=steps.STEPS_F32_NAIVE, G=p.G, Om=p.Om,
                                  OL=p.OL)
    naive = steps.Simulation(p.pos, p.vel, p.mass, h_min=p.h_min, t0=p.t0, a0=p.a0, cfg=cfg_naive,
                             stream=stream.cuda_stream)
    acc_naive = np.empty((n, 3))
    steps.steps_get_state(naive.ctx, acc=acc_naive)
    steps.steps_profile_enable(naive.ctx, True)
    for _ in range(2):
        steps.steps_forces(naive.ctx)
    naive_ms, naive_launches, _ = steps.steps_profile_read(naive.ctx)
    naive_rate = naive_launches * n * n / (naive_ms * 1e-3)
    naive.close()

    # ---- CPU baseline: the FP64 oracle on the seeded targets (rank 0 only) ----
    cpu = None
    err = {}
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        h = oracle.softening(p.mass, p.h_min)
        t0 = time.perf_counter()
        ref = oracle.pair_acc(p.pos, p.mass, h, p.G, targets=tg)
        cpu_s = time.perf_counter() - t0
        cpu = {"value": tg.size * n / cpu_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d seeded targets x all %d sources (FP64 direct sum, OpenMP), %.1f s" % (tg.size, n, cpu_s)}
        nrm = np.linalg.norm(ref, axis=1)
        for name, a in (("f32_comp", acc_mixed[tg]), ("f32_naive", acc_naive[tg]), ("f64_gpu", acc64)):
            e = np.linalg.norm(a - ref, axis=1) / nrm
            err[name] = {"rms": float(np.sqrt(np.mean(e ** 2))), "max": float(e.max())}

    # ---- warm-up and timed KDK steps ----
    for k in range(args.warmup):
        sim.step(dts[k])
    torch.cuda.synchronize()
    steps.steps_profile_read(sim.ctx, reset=True)
    steps.steps_force_stats(sim.ctx)  # restart the near/far tile-pair counts
    steps.steps_profile_enable(sim.ctx, True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                      # L2 flush between timed steps (not timed)
                starts[k].record(stream)
            sim.step(dts[args.warmup + k])
            with torch.cuda.stream(stream):
                ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    far_ms, far_launches = steps.steps_profile_read_far(sim.ctx)
    force_ms, force_launches, kernel_launches = steps.steps_profile_read(sim.ctx, reset=True)
    near_pairs, all_pairs = steps.steps_force_stats(sim.ctx)
    steps.steps_profile_enable(sim.ctx, False)
    value, total_s = job_throughput(sum(step_ms) * 1e-3, args.steps * n * n, device=dev)

    # ---- end to end through the C ABI with host buffers ----
    pos_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    vel_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    acc_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    t_now, a_now = steps.steps_get_state(sim.ctx, pos=pos_h.numpy(), vel=vel_h.numpy())
    steps.steps_set_state(sim.ctx, pos_h.numpy(), vel_h.numpy(), t_now, a_now)  # warm
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        steps.steps_set_state(sim.ctx, pos_h.numpy(), vel_h.numpy(), t_now, a_now)  # H2D + sort + forces
        steps.steps_get_state(sim.ctx, acc=acc_h.numpy())                         # D2H of the result
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_steps * n * n * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 2 * 3 * 8 * n, "d2h_bytes_per_step": 3 * 8 * n,
           "what": "steps_set_state(host pos, vel) + steps_get_state(host acc): one force evaluation per step"}
    sim.close()
    evolved = None
    if rank == 0 and not args.no_cpu:
        # the pair term at the state reached after the warm-up and timed steps
        ref_ev = oracle.pair_acc(pos_h.numpy(), p.mass, h, p.G, targets=tg)
        e = np.linalg.norm(acc_h.numpy()[tg] - ref_ev, axis=1) / np.linalg.norm(ref_ev, axis=1)
        evolved = {"rms": float(np.sqrt(np.mean(e ** 2))), "max": float(e.max()), "a": a_now,
                   "steps": args.warmup + args.steps}
    workloads_cpu = None
    if rank == 0 and not args.no_cpu:
        workloads_cpu = cpu_workloads(stream, steps, workloads)
    ensemble = None
    if rank == 0 and not args.no_ensemble:
        ensemble = ensemble_throughput(stream, steps, workloads)
    periodic = None
    if rank == 0 and not args.no_periodic:
        periodic = periodic_throughput(steps)

    if rank != 0:
        dist.destroy_process_group()
        return
    clocks = clk.summary()
    force_avg_s = force_ms * 1e-3 / max(force_launches, 1)
    far_avg_s = far_ms * 1e-3 / max(far_launches, 1)
    near_frac = near_pairs / max(all_pairs, 1)
    # the far-field kernel evaluates every tile pair not marked near: all its
    # targets against all sources of those tiles (N^2 (1 - near fraction) at
    # equal tile sizes); the near-field kernel does the rest
    far_interactions = n * n * (1.0 - near_frac)
    achieved = FLOP_PER_INTERACTION * far_interactions / far_avg_s / 1e12
    pk = peaks()
    max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(props.multi_processor_count, max_mhz)
    fp64_peak = props.multi_processor_count * FP64_FMA_PER_SM_CLK * 2 * max_mhz * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n": n, "prec": "f32 pairs, compensated sums, fp64 integrator",
                   "parallelism": "replicas" if ws > 1 else "single gpu",
                   "l2": "flushed between timed steps (%d MiB write)" % (L2_FLUSH_BYTES >> 20),
                   "variant": variant_name},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": FAR_TRAFFIC_BYTES.get((variant_name, n)),
                     "kernel": "%s (far field, %s)" % ("sym_far_kernel" if variant_name.startswith("sym") else "force_f32_kernel", variant_name),
                     "basis": "%d flop/interaction x N^2 (1 - near fraction %.4f of the tile pairs, or of their 128 x 128 "
                              "sub-blocks for sym_ki8s) per launch / mean far-field "
                              "launch time (CUDA events on the launching stream, %d launches); peak = %d SMs x 128 FP32 "
                              "lanes x 2 x %.0f MHz (FP32 FMA pipe, no measured FP32 peak on file)"
                              % (FLOP_PER_INTERACTION, near_frac, far_launches, props.multi_processor_count, max_mhz),
                     "pair_force_evaluation_tflops": FLOP_PER_INTERACTION * n * n / force_avg_s / 1e12,
                     "frac_at_observed_clock": (achieved / fp32_peak_tflops(props.multi_processor_count, clocks["sm_mhz"])
                                                if clocks.get("sm_mhz") else None)},
        "cpu_baseline": dict(cpu, workloads=workloads_cpu) if cpu else None,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(kernel_launches),
        "comparison": {
            "f32_comp": {"interactions_per_s": value / ws, "force_kernel_interactions_per_s": n * n / force_avg_s,
                         **err.get("f32_comp", {})},
            "f32_naive": {"force_kernel_interactions_per_s": naive_rate, **err.get("f32_naive", {})},
            "f64_gpu": {"interactions_per_s": f64_rate, "sample": "%d targets x %d sources" % (big_tg.size, n),
                        "kernel": "force_f64_list_kernel (FP64, one warp per target, lane-strided sources, shuffle-tree sum)",
                        "fp64_tflops_at_20_flop": FLOP_PER_INTERACTION * f64_rate / 1e12,
                        "fp64_peak_tflops": fp64_peak,
                        "frac_of_fp64_peak_at_20_flop": FLOP_PER_INTERACTION * f64_rate / 1e12 / fp64_peak,
                        "mixed_over_fp64": (value / ws) / f64_rate,
                        **err.get("f64_gpu", {})},
            "f32_comp_evolved": evolved,
            "error_targets": int(tg.size),
        },
        "near_field_fraction": near_frac,
        "ensemble": ensemble,
        "periodic": periodic,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision_1m")
    ap.add_argument("--variant", type=int, default=0, help="force-kernel variant (1-based), 0 = auto")
    ap.add_argument("--f64-targets", type=int, default=16384)
    ap.add_argument("--ref-targets", type=int, default=512)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-periodic", action="store_true")
    ap.add_argument("--periodic-only", action="store_true",
                    help="time only the periodic-mode force evaluations (one JSON line; not the bench line)")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="time only the batched ensemble against its members run one by one (one JSON line; "
                         "not the bench line)")
    args = ap.parse_args()
    if args.periodic_only or args.ensemble_only:
        import torch

        import paper_1811_05903_gb300.build as libbuild
        from paper_1811_05903_gb300 import steps, workloads
        torch.cuda.set_device(0)
        libbuild.build()
        steps.load()
        if args.periodic_only:
            print(json.dumps({"periodic": periodic_throughput(steps)}))
        else:
            print(json.dumps({"ensemble": ensemble_throughput(torch.cuda.Stream(), steps, workloads)}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
