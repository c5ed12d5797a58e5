"""Correlation-function emulator: batched compactified runs -> exact pair
counts of the central sphere -> xi(r) -> a small network trained by the
library's kernels -> error on held-out plain simulations.

The simulations are run for the statistics of the density field (Sec. 1;
opening of Sec. 3).  The emulator answers "what xi(r) would a run at these
cosmological parameters give" in microseconds instead of a simulation, which
is what a parameter fit needs; the plain batched simulation remains the
measure of its error.  Every numerical step runs in libsteps: the N-body runs
(steps_ensemble_*), the pair counts (steps_paircount) and the network's
training and inference (steps_emu_*).  This module marshals: it draws the
parameter sets and initial conditions (``workloads``), maps features and
targets to and from the network's normalised units, and scores the result.

    python -m paper_1811_05903_gb300.emulator --train 512 --test 64

prints one JSON line.  Readings: xi is measured on the central particles
within R_XI = 40 Mpc/h of the centre at a = 1 (inside the constant-resolution
sphere of radius 50), natural estimator DD/RR - 1 with the analytic RR of a
uniform ball; the network sees (Om, sigma8, h, n_s, ln r) scaled to [-1, 1]
and predicts asinh(xi), standardised bin by bin over the training runs (so
that the small variations of the large-separation bins weigh as much as the
large ones of the small-separation bins).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import time

import numpy as np

from . import steps, workloads

R_XI = 40.0
NBINS = 24
R_MIN, R_MAX = 0.5, 20.0
FIXED_POINT_BITS = 20  # positions quantised to R_XI / 2^20


def bin_edges() -> np.ndarray:
    return R_MIN * (R_MAX / R_MIN) ** (np.arange(NBINS + 1) / NBINS)


def bin_centres() -> np.ndarray:
    e = bin_edges()
    return np.sqrt(e[1:] * e[:-1])


def _ball_pair_fraction(s, R):
    """Fraction of pairs of uniform points in a ball of radius R closer than s."""
    x = np.clip(np.asarray(s, dtype=np.float64) / R, 0.0, 2.0)
    return x ** 3 - 9.0 / 16.0 * x ** 4 + x ** 6 / 32.0


def xi_from_counts(dd, n_in, R=R_XI, edges=None):
    """Natural estimator xi = DD/RR - 1 per set; returns (xi, RR)."""
    edges = bin_edges() if edges is None else edges
    n_in = np.asarray(n_in, dtype=np.float64)[:, None]
    rr = 0.5 * n_in * (n_in - 1) * np.diff(_ball_pair_fraction(edges, R))[None, :]
    return np.asarray(dd, dtype=np.float64) / rr - 1.0, rr


def _make_run(args):
    seed, theta, kw = args
    return workloads.emulator_run(seed, *[float(v) for v in theta], **kw)


def generate_runs(thetas, seed0: int, processes: int = 0, fixed_phases: bool = True, **kw):
    """Initial conditions of one run per parameter set (host, in parallel;
    'spawn' so that no worker inherits a CUDA context).  With fixed_phases
    every run shares one random realisation (lattice offset and white-noise
    field), so that runs differ by their parameters alone and the sample
    variance of a 40 Mpc/h sphere does not enter the emulator's targets."""
    jobs = [(seed0 if fixed_phases else seed0 * 100003 + k, th, kw) for k, th in enumerate(thetas)]
    if processes == 1 or len(jobs) < 4:
        return [_make_run(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes or min(16, mp.cpu_count())) as pool:
        return pool.map(_make_run, jobs, chunksize=4)


def simulate(runs, n_steps: int, batch: int = 64, resort_every: int = 8):
    """Advance every run from its a0 to a = 1 in n_steps log-a KDK steps,
    ``batch`` runs per ensemble launch.  Returns the central particles'
    positions at a = 1 and the wall seconds spent in the library."""
    out, secs = [], 0.0
    for b0 in range(0, len(runs), batch):
        members = runs[b0:b0 + batch]
        cfgs = [steps.make_config(mode=steps.STEPS_COMOVING, prec=steps.STEPS_F32_COMP, G=p.G,
                                  Om=p.Om, OL=p.OL, resort_every=resort_every) for p in members]
        dts = np.stack([workloads.loga_schedule(p.a0, 1.0, n_steps, p.Om, p.OL)[1] for p in members])
        t0 = time.perf_counter()
        ens = steps.Ensemble(members, cfgs)
        ens.run(dts)
        for s, p in enumerate(members):
            pos, _, _, _, a = ens.state(s)
            out.append(pos[:p.n_central].copy())
        ens.close()
        secs += time.perf_counter() - t0
    return out, secs


def measure_xi(central_positions, R: float = R_XI):
    """Exact pair counts of the particles within R of the centre, all sets in
    one library call; returns (xi [nsets][NBINS], DD, RR, n_in)."""
    sel = [p[np.einsum("ij,ij->i", p, p) < R * R] for p in central_positions]
    n_in = np.array([len(p) for p in sel], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(n_in)]).astype(np.int64)
    step = R / 2 ** FIXED_POINT_BITS
    edge2 = np.ceil((bin_edges() / step) ** 2).astype(np.int64)
    dd = steps.steps_paircount(offsets, np.concatenate(sel), np.zeros((len(sel), 3)), step, edge2)
    xi, rr = xi_from_counts(dd, n_in, R)
    return xi, dd, rr, n_in


class XiEmulator:
    """(Om, sigma8, h, n_s) -> xi in NBINS bins, on the library's network."""

    def __init__(self, seed: int = 0, batch: int = 1024):
        self.ranges = np.array(list(workloads.EMU_RANGES.values()))
        self.lnr = np.log(bin_centres())
        self.batch = batch
        self.params0 = self._init_params(seed)
        self.net = None
        self.mu, self.sd = np.zeros(NBINS), np.ones(NBINS)

    @staticmethod
    def _init_params(seed):
        """He-uniform weights, zero biases (packed in the library's order)."""
        rng = np.random.Generator(np.random.PCG64(seed))
        widths = (steps.STEPS_EMU_IN, 256, 256, 256, 1)
        out = []
        for fo, fi in zip(widths[1:], widths[:-1]):
            lim = math.sqrt(6.0 / fi)
            out += [rng.uniform(-lim, lim, fo * fi), np.zeros(fo)]
        return np.concatenate(out).astype(np.float32)

    def features(self, thetas) -> np.ndarray:
        th = np.asarray(thetas, dtype=np.float64).reshape(-1, 4)
        lo, hi = self.ranges[:, 0], self.ranges[:, 1]
        u = 2.0 * (th - lo) / (hi - lo) - 1.0
        v = 2.0 * (self.lnr - math.log(R_MIN)) / (math.log(R_MAX) - math.log(R_MIN)) - 1.0
        X = np.concatenate([np.repeat(u, NBINS, axis=0), np.tile(v, len(th))[:, None]], axis=1)
        return X.astype(np.float32)

    def fit(self, thetas, xi, n_steps: int = 4000, lr: float = 1e-3, seed: int = 1):
        """Adam with a cosine learning-rate schedule on shuffled epochs.
        Targets: asinh(xi) standardised bin by bin over the training runs.
        (Scaling each bin by the error measure's own denominator instead,
        max(|xi|, sigma_P) in asinh units, was measured on the 512-run
        pipeline: held-out rms 0.281 against 0.268, so it is not used.)"""
        y = np.arcsinh(np.asarray(xi, dtype=np.float64)).reshape(-1, NBINS)
        self.mu = y.mean(axis=0)
        self.sd = np.where(y.std(axis=0) > 0, y.std(axis=0), 1.0)
        X = self.features(thetas)
        t = ((y - self.mu) / self.sd).reshape(-1).astype(np.float32)
        self.net = steps.Emulator(self.params0, batch=self.batch)
        self.net.set_data(X, t)
        rng = np.random.Generator(np.random.PCG64(seed))
        n = X.shape[0]
        per_epoch = max(1, n // self.batch)
        rows = []
        while len(rows) < n_steps:
            perm = rng.permutation(n)
            rows += [perm[k * self.batch:(k + 1) * self.batch] for k in range(per_epoch)
                     if (k + 1) * self.batch <= n]
            if n < self.batch:
                rows.append(rng.integers(0, n, self.batch))
        rows = np.stack(rows[:n_steps]).astype(np.int32)
        lrs = (lr * 0.5 * (1.0 + np.cos(np.pi * np.arange(n_steps) / n_steps))).astype(np.float32)
        t0 = time.perf_counter()
        losses = self.net.train(rows, lrs)
        self.train_seconds = time.perf_counter() - t0
        return losses

    def predict(self, thetas) -> np.ndarray:
        y = self.net.predict(self.features(thetas)).astype(np.float64).reshape(-1, NBINS)
        return np.sinh(y * self.sd + self.mu)

    def close(self):
        if self.net is not None:
            self.net.close()
            self.net = None


def scaled_errors(xi_pred, xi_true, dd):
    """(xi_pred - xi_true) / max(|xi_true|, sigma_P), sigma_P = (1 + xi) / sqrt(DD)
    the Poisson error of the counts."""
    sig = (1.0 + xi_true) / np.sqrt(np.maximum(np.asarray(dd, dtype=np.float64), 1.0))
    return (xi_pred - xi_true) / np.maximum(np.abs(xi_true), np.abs(sig))


def error_breakdown(err, err_nn, xi_true, dd):
    """Where the scaled errors come from: per bin (rms of the emulator and of
    the nearest-neighbour run, median |xi| and median Poisson scale), per
    held-out run, and the share of the squared error carried by the worst 1%
    of (run, bin) entries."""
    sig = (1.0 + xi_true) / np.sqrt(np.maximum(np.asarray(dd, dtype=np.float64), 1.0))
    sq = (err ** 2).ravel()
    k = max(1, sq.size // 100)
    worst = np.sort(sq)[::-1]
    return {
        "per_bin_rms": [float(v) for v in np.sqrt(np.mean(err ** 2, axis=0))],
        "per_bin_rms_nearest_neighbour": [float(v) for v in np.sqrt(np.mean(err_nn ** 2, axis=0))],
        "per_bin_median_abs_xi": [float(v) for v in np.median(np.abs(xi_true), axis=0)],
        "per_bin_median_sigma_poisson": [float(v) for v in np.median(sig, axis=0)],
        "per_run_rms": [float(v) for v in np.sqrt(np.mean(err ** 2, axis=1))],
        "worst_1pct_share_of_squared_error": float(worst[:k].sum() / max(sq.sum(), 1e-300)),
    }


def nearest_neighbour(theta_train, xi_train, theta_test, ranges):
    """xi of the training run nearest in normalised parameter space."""
    lo, hi = ranges[:, 0], ranges[:, 1]
    a = (np.asarray(theta_train) - lo) / (hi - lo)
    b = (np.asarray(theta_test) - lo) / (hi - lo)
    d = ((b[:, None, :] - a[None, :, :]) ** 2).sum(-1)
    return np.asarray(xi_train)[d.argmin(axis=1)]


def fit_demo(emu: XiEmulator, xi_obs, dd_obs, theta_true, ngrid: int = 81):
    """Least-squares (Om, sigma8) on a grid, h and n_s held at their true
    values, with the emulator as the model and Poisson errors."""
    lo, hi = emu.ranges[:2, 0], emu.ranges[:2, 1]
    om = np.linspace(lo[0], hi[0], ngrid)
    s8 = np.linspace(lo[1], hi[1], ngrid)
    OM, S8 = np.meshgrid(om, s8, indexing="ij")
    th = np.stack([OM.ravel(), S8.ravel(), np.full(OM.size, theta_true[2]), np.full(OM.size, theta_true[3])], 1)
    t0 = time.perf_counter()
    pred = emu.predict(th)
    secs = time.perf_counter() - t0
    sig = (1.0 + xi_obs) / np.sqrt(np.maximum(dd_obs, 1.0))
    chi2 = (((pred - xi_obs[None, :]) / sig[None, :]) ** 2).sum(1)
    k = int(chi2.argmin())
    return {"Om_true": float(theta_true[0]), "sigma8_true": float(theta_true[1]),
            "Om_fit": float(th[k, 0]), "sigma8_fit": float(th[k, 1]), "grid": ngrid * ngrid,
            "seconds": secs}


def run(n_train=512, n_test=64, n_central=16384, n_shells=32, per_shell=512, n_steps=200, ngrid=128,
        train_steps=8000, batch=1024, lr=1e-3, seed=5, processes=0, fixed_phases=True, save=None):
    t_all = time.perf_counter()
    th_train = workloads.latin_hypercube(n_train, seed)
    th_test = workloads.latin_hypercube(n_test, seed + 1)
    kw = dict(n_central=n_central, n_shells=n_shells, per_shell=per_shell, ngrid=ngrid)
    t0 = time.perf_counter()
    runs_train = generate_runs(th_train, seed, processes, fixed_phases, **kw)
    runs_test = generate_runs(th_test, seed if fixed_phases else seed + 1, processes, fixed_phases, **kw)
    t_ic = time.perf_counter() - t0
    steps.load()
    cen_train, s_train = simulate(runs_train, n_steps)
    cen_test, s_test = simulate(runs_test, n_steps)
    t0 = time.perf_counter()
    xi_tr, dd_tr, rr_tr, n_tr = measure_xi(cen_train)
    xi_te, dd_te, rr_te, n_te = measure_xi(cen_test)
    t_xi = time.perf_counter() - t0
    if save:
        np.savez(save, theta_train=th_train, xi_train=xi_tr, dd_train=dd_tr, n_train=n_tr,
                 theta_test=th_test, xi_test=xi_te, dd_test=dd_te, n_test=n_te)
    emu = XiEmulator(seed, batch)
    losses = emu.fit(th_train, xi_tr, train_steps, lr, seed)
    pred = emu.predict(th_test)
    err = scaled_errors(pred, xi_te, dd_te)
    nn = nearest_neighbour(th_train, xi_tr, th_test, emu.ranges)
    err_nn = scaled_errors(nn, xi_te, dd_te)
    # latency of one query (NBINS bins of one parameter set), host in and out
    emu.predict(th_test[:1])
    reps = 200
    t0 = time.perf_counter()
    for _ in range(reps):
        emu.predict(th_test[:1])
    us_eval = (time.perf_counter() - t0) / reps * 1e6
    demo = fit_demo(emu, xi_te[0], dd_te[0], th_test[0])
    emu.close()
    return {
        "workload": "emulator: %d train + %d held-out runs, N=%d (%d central), %d log-a steps 0.02->1"
                    % (n_train, n_test, n_central + n_shells * per_shell, n_central, n_steps),
        "phases": "one shared realisation" if fixed_phases else "independent realisations",
        "xi_bins": "%d log bins %.1f-%.1f Mpc/h, central particles within %.0f Mpc/h at a=1"
                   % (NBINS, R_MIN, R_MAX, R_XI),
        "emulator_rms_scaled_err": float(np.sqrt(np.mean(err ** 2))),
        "nearest_neighbour_rms_scaled_err": float(np.sqrt(np.mean(err_nn ** 2))),
        "emulator_median_abs_scaled_err": float(np.median(np.abs(err))),
        "train_loss_first_last": [float(losses[0]), float(np.mean(losses[-50:]))],
        "train_seconds": emu.train_seconds, "train_steps": train_steps, "batch": batch,
        "emulator_us_per_query": us_eval,
        "sim_seconds_per_run": (s_train + s_test) / (n_train + n_test),
        "sim_seconds_total": s_train + s_test, "ic_seconds": t_ic, "paircount_seconds": t_xi,
        "central_in_R_mean": float(np.mean(np.concatenate([n_tr, n_te]))),
        "xi_mean_train": [float(v) for v in xi_tr.mean(0)],
        "breakdown": error_breakdown(err, err_nn, xi_te, dd_te),
        "fit_demo": demo, "total_seconds": time.perf_counter() - t_all,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--n-central", type=int, default=16384)
    ap.add_argument("--n-shells", type=int, default=32)
    ap.add_argument("--per-shell", type=int, default=512)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--ngrid", type=int, default=128)
    ap.add_argument("--train-steps", type=int, default=8000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--processes", type=int, default=0)
    ap.add_argument("--random-phases", action="store_true", help="an independent realisation per run")
    ap.add_argument("--save", default=None, help="write the measured xi and counts to this .npz")
    a = ap.parse_args(argv)
    res = run(a.train, a.test, a.n_central, a.n_shells, a.per_shell, a.steps, a.ngrid, a.train_steps,
              a.batch, a.lr, a.seed, a.processes, not a.random_phases, a.save)
    print(json.dumps(res))
    return res


if __name__ == "__main__":
    main()
