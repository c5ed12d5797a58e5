"""Spherical glasses for StePS initial conditions (Sec. 3.1), made on the GPU.

A glass is a particle set that represents a uniform density with as little
net force on each particle as possible.  The recipe of Sec. 3.1:

1. slice the compactified space (Eq. 14-15) into shells -- constant delta-omega
   with a united inner ball (Eq. 17), or constant compact volume (Eq. 18) -- and
   place n_shell particles at random in each (``steps_glass_place``; the
   uniform random numbers are drawn here and passed in);
2. integrate Eq. 8 with gravity reversed in an Einstein-de Sitter background
   (``STEPS_COMOVING_REVERSED``, Om = 1, OL = 0, G = H0 = 1) until the particles
   settle; KDK steps uniform in ln a from ``a_start`` to ``a_end``.

The relaxation uses the EdS mean density rho_crit = 3/(8 pi) for the masses
(so that the background term balances the pair term); the returned masses are
rescaled to the requested mean density (Eq. 16 for the target cosmology).
Placement, forces and integration run in the library's kernels; this module
draws the random numbers, builds the step schedule and evaluates the
net-force diagnostic.
"""
from __future__ import annotations

import math

import numpy as np

from . import steps

RHO_EDS = 3.0 / (8.0 * math.pi)  # rho_crit for G = H0 = 1, Om = 1


def eds_time(a):
    """Cosmic time of scale factor a in Einstein-de Sitter with H0 = 1."""
    return 2.0 / 3.0 * np.asarray(a, dtype=np.float64) ** 1.5


def place(scheme: int, D_s: float, R_sim: float, n_radial: int, n_shell: int, r_c: float = 0.0,
          rho_bar: float = RHO_EDS, seed: int = 0):
    """Shell layout and random placement (Eq. 14-18): positions [n][3], masses [n]."""
    spec = steps.glass_spec(scheme, D_s, R_sim, n_radial, n_shell, r_c, rho_bar)
    n = steps.steps_glass_layout(spec)[0]
    u = np.random.default_rng(seed).random((n, 3))
    return steps.steps_glass_place(spec, u)


def relax(pos, mass, h_min: float, a_start: float = 0.1, a_end: float = 1.0, nsteps: int = 100,
          prec: int = steps.STEPS_F32_COMP, stream=None):
    """Reversed-gravity relaxation in EdS (Sec. 3.1); returns the new positions.
    ``mass`` must carry the EdS mean density (``RHO_EDS``) for the background
    term to balance the pair term."""
    cfg = steps.make_config(mode=steps.STEPS_COMOVING_REVERSED, prec=prec, G=1.0, Om=1.0, OL=0.0)
    t = eds_time(np.geomspace(a_start, a_end, nsteps + 1))
    sim = steps.Simulation(pos, np.zeros_like(pos), mass, h_min=h_min, t0=float(t[0]), a0=a_start, cfg=cfg,
                           stream=stream)
    try:
        sim.run(np.diff(t))
        return sim.state()[0]
    finally:
        sim.close()


def make_glass(scheme: int, D_s: float, R_sim: float, n_radial: int, n_shell: int, r_c: float = 0.0,
               rho_bar: float = RHO_EDS, h_min: float | None = None, seed: int = 0, **relax_kw):
    """Place and relax a spherical glass; masses scaled to ``rho_bar``."""
    pos, mass = place(scheme, D_s, R_sim, n_radial, n_shell, r_c, RHO_EDS, seed)
    if h_min is None:
        h_min = default_h_min(pos, mass)
    pos = relax(pos, mass, h_min, **relax_kw)
    return pos, mass * (rho_bar / RHO_EDS)


def default_h_min(pos, mass) -> float:
    """Softening of the lightest particle: 1/20 of its mean spacing at the mean density."""
    return 0.05 * (float(np.min(mass)) / RHO_EDS) ** (1.0 / 3.0)


def peculiar_acceleration(pos, mass, h_min: float, rho_bar: float = RHO_EDS):
    """|pair term + (4 pi G / 3) rho_bar x| per particle under ordinary gravity
    (the net force a glass minimises), from the library's FP32 force path."""
    cfg = steps.make_config(mode=steps.STEPS_STATIC, prec=steps.STEPS_F32_COMP, G=1.0)
    sim = steps.Simulation(pos, np.zeros_like(pos), mass, h_min=h_min, cfg=cfg)
    try:
        acc = sim.forces()
    finally:
        sim.close()
    return np.linalg.norm(acc + 4.0 * math.pi / 3.0 * rho_bar * np.asarray(pos), axis=1)
