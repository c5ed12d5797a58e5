"""Seeded synthetic inputs for the StePS direct-summation path.

This module only *builds inputs*: particle positions, velocities and masses
with the shapes, sizes and mass spectra of the paper's compactified
simulations, plus the step schedule.  It holds none of the method's
arithmetic (no force kernel, no softening rule, no integrator); the CUDA
library and the CPU oracle each implement those on their own and both read
their inputs from here.

Units throughout: length Mpc/h, time 1/H0 (so H0 = 1), G = 1, hence
rho_crit = 3 / (8 pi).  All randomness comes from numpy PCG64 with fixed seeds.

Recipes (shell construction after the paper's Sec. 3, simplified to log-radius
shells of random particles instead of a relaxed glass):
  * ``static_ball``      -- 2,048 unit-mass particles uniform in the unit ball
                            plus 16 shells x 128 particles at radii 20^(k/15);
                            shell masses keep the mean density continuous.
  * ``compactified``     -- a constant-resolution central sphere (r <= 50)
                            and log-spaced shells out to 4,000 Mpc/h whose
                            particle mass grows with shell volume (Eq. 16 of
                            the paper), Gaussian displacements with rms 1% of
                            the local spacing and Zel'dovich-like velocities.
  * ``ensemble``         -- 64 such runs of uneven N and differing Om, sigma8.
  * ``emulator_run``     -- a compactified run whose central sphere is a
                            lattice displaced by a Gaussian random field with
                            a BBKS spectrum (Om, sigma8, h, n_s), for the
                            correlation-function emulator's training set;
                            ``latin_hypercube`` draws the parameter sets.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RHO_CRIT = 3.0 / (8.0 * math.pi)  # 3 H0^2 / (8 pi G) with H0 = G = 1


@dataclasses.dataclass
class Particles:
    pos: np.ndarray          # [n, 3] float64
    vel: np.ndarray          # [n, 3] float64
    mass: np.ndarray         # [n] float64
    h_min: float             # softening of the lightest particle (Eq. 7 input)
    G: float = 1.0
    comoving: bool = False
    Om: float = 0.3
    OL: float = 0.7
    a0: float = 1.0
    t0: float = 0.0
    n_central: int = 0
    r_central: float = 0.0

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _uniform_ball(rng, n, radius):
    """Rejection sampling from the enclosing cube."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        c = rng.uniform(-1.0, 1.0, size=(2 * n + 16, 3))
        c = c[np.einsum("ij,ij->i", c, c) <= 1.0]
        out = np.concatenate([out, c])
    return out[:n] * radius


def static_ball(seed: int = 1, n_ball: int = 2048, n_shells: int = 16, per_shell: int = 128,
                r_outer: float = 20.0) -> Particles:
    """Small static (non-comoving) test system, G = 1, zero velocities.

    Shell k sits at radius r_k = r_outer^(k/(n_shells-1)); its particles share
    the mass of the volume between geometric-midpoint edges (inner edge 1,
    outer edge r_last * r_outer^(1/(2(n_shells-1)))) at the ball's density.
    Softening is Eq. 7 with h_min = 0.02 (the lightest mass is 1), i.e.
    eps_i = 0.02 m_i^(1/3).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ball = _uniform_ball(rng, n_ball, 1.0)
    rho = n_ball / (4.0 / 3.0 * math.pi)
    k = np.arange(n_shells)
    radii = r_outer ** (k / (n_shells - 1))
    edges = np.empty(n_shells + 1)
    edges[0] = 1.0
    edges[1:-1] = np.sqrt(radii[:-1] * radii[1:])
    edges[-1] = radii[-1] * r_outer ** (1.0 / (2 * (n_shells - 1)))
    dv = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    shell_pos = np.concatenate([_unit_vectors(rng, per_shell) * r for r in radii])
    shell_m = np.repeat(rho * dv / per_shell, per_shell)
    pos = np.concatenate([ball, shell_pos])
    mass = np.concatenate([np.ones(n_ball), shell_m])
    return Particles(pos=pos, vel=np.zeros_like(pos), mass=mass, h_min=0.02, G=1.0,
                     comoving=False, a0=1.0, n_central=n_ball, r_central=1.0)


def flat_lcdm_time(a, Om: float, OL: float):
    """Cosmic time of a flat LambdaCDM universe (Or = Ok = 0), H0 = 1:
    t(a) = 2 / (3 sqrt(OL)) asinh(sqrt(OL/Om) a^(3/2)).  Used to lay out the
    step schedule; the integrators advance a(t) on their own."""
    a = np.asarray(a, dtype=np.float64)
    return 2.0 / (3.0 * math.sqrt(OL)) * np.arcsinh(math.sqrt(OL / Om) * a ** 1.5)


def loga_schedule(a_start: float, a_end: float, n_steps: int, Om: float, OL: float):
    """Steps uniform in ln a; returns (a_n [n_steps+1], dt_n [n_steps])."""
    a = a_start * (a_end / a_start) ** (np.arange(n_steps + 1) / n_steps)
    t = flat_lcdm_time(a, Om, OL)
    return a, np.diff(t)


def _growth_rate_hubble(a, Om, OL):
    """f(a) H(a) for the Zel'dovich velocity, f = Om(a)^0.55 (IC recipe)."""
    E2 = Om / a ** 3 + OL
    om_a = Om / a ** 3 / E2
    return om_a ** 0.55 * math.sqrt(E2)


def compactified(seed: int, n_central: int, n_shells: int, per_shell: int,
                 r_central: float = 50.0, r_max: float = 4000.0, Om: float = 0.3,
                 OL: float = 0.7, a0: float = 0.02, disp_frac: float = 0.01,
                 h_min_frac: float = 1.0 / 50.0) -> Particles:
    """StePS-like compactified LambdaCDM particle set (comoving coordinates).

    * central sphere: n_central equal-mass particles uniform in r <= r_central,
      m_c = Om rho_crit (4 pi/3) r_central^3 / n_central;
    * n_shells shells with edges log-spaced from r_central to r_max, per_shell
      particles each, uniform in volume inside the shell, mass
      Om rho_crit V_shell / per_shell (particle mass grows ~ r^2 dr);
    * i.i.d. Gaussian displacement with rms |Psi| = disp_frac x local spacing
      (V_particle^(1/3)), velocity dx/dt = f(a0) H(a0) Psi;
    * h_min = h_min_frac x central spacing (Eq. 7 input).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = Om * RHO_CRIT
    vc = 4.0 / 3.0 * math.pi * r_central ** 3
    central = _uniform_ball(rng, n_central, r_central)
    m_c = rho * vc / n_central
    edges = r_central * (r_max / r_central) ** (np.arange(n_shells + 1) / n_shells)
    lo3 = np.repeat(edges[:-1] ** 3, per_shell)
    hi3 = np.repeat(edges[1:] ** 3, per_shell)
    r = np.cbrt(lo3 + rng.uniform(size=lo3.size) * (hi3 - lo3))
    shell = _unit_vectors(rng, lo3.size) * r[:, None]
    v_shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    m_shell = np.repeat(rho * v_shell / per_shell, per_shell)
    pos = np.concatenate([central, shell])
    mass = np.concatenate([np.full(n_central, m_c), m_shell])
    spacing = np.cbrt(mass / rho)
    psi = rng.standard_normal(pos.shape) * (disp_frac * spacing / math.sqrt(3.0))[:, None]
    pos = pos + psi
    vel = _growth_rate_hubble(a0, Om, OL) * psi
    h_min = h_min_frac * math.cbrt(m_c / rho)
    t0 = float(flat_lcdm_time(a0, Om, OL))
    return Particles(pos=pos, vel=vel, mass=mass, h_min=h_min, G=1.0, comoving=True, Om=Om,
                     OL=OL, a0=a0, t0=t0, n_central=n_central, r_central=r_central)


def lcdm_262k(seed: int = 2) -> Particles:
    """N = 262,144: 131,072 central in 50 Mpc/h + 64 shells x 2,048 to 4,000 Mpc/h."""
    return compactified(seed, 131072, 64, 2048)


def precision_1m(seed: int = 3) -> Particles:
    """N = 1,048,576: 524,288 central + 64 shells x 8,192 (the precision study)."""
    return compactified(seed, 524288, 64, 8192)


def precision_targets(n: int, count: int = 4096, seed: int = 3) -> np.ndarray:
    """Seeded subset of target rows at which the FP64 oracle is evaluated."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int64)


@dataclasses.dataclass
class Ensemble:
    sims: list               # list[Particles]
    sigma8: np.ndarray       # [nsims]


def ensemble(seed: int = 4, nsims: int = 64, n_lo: int = 8192, n_hi: int = 131072,
             n_shells: int = 64) -> Ensemble:
    """Independent compactified runs of uneven N and differing cosmology.

    N_s ~ U[n_lo, n_hi] rounded to a multiple of 2 n_shells, half central;
    Om ~ U[0.25, 0.35] (OL = 1 - Om), sigma8 ~ U[0.7, 0.9] scales the
    displacement amplitude (disp_frac = 0.01 sigma8 / 0.8)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = 2 * n_shells
    ns = (rng.integers(n_lo, n_hi + 1, size=nsims) // q) * q
    Oms = rng.uniform(0.25, 0.35, size=nsims)
    s8 = rng.uniform(0.7, 0.9, size=nsims)
    sims = []
    for s in range(nsims):
        n = int(ns[s])
        sims.append(compactified(seed * 1000 + s, n // 2, n_shells, n // 2 // n_shells,
                                 Om=float(Oms[s]), OL=1.0 - float(Oms[s]),
                                 disp_frac=0.01 * float(s8[s]) / 0.8))
    return Ensemble(sims=sims, sigma8=s8)


# ---------------------------------------------------------------------------
# Emulator training runs: Gaussian-random-field initial conditions
# ---------------------------------------------------------------------------
EMU_RANGES = {"Om": (0.25, 0.35), "sigma8": (0.7, 0.9), "h": (0.6, 0.8), "ns": (0.92, 1.0)}


def latin_hypercube(n: int, seed: int, ranges=EMU_RANGES) -> np.ndarray:
    """n points, one per stratum in every dimension, strata matched at random;
    columns in the order of ``ranges``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = []
    for lo, hi in ranges.values():
        u = (rng.permutation(n) + rng.uniform(size=n)) / n
        cols.append(lo + (hi - lo) * u)
    return np.stack(cols, axis=1)


def bbks_spectrum(k, Om: float, h: float, ns: float):
    """Un-normalised linear spectrum k^ns T^2(k), T the BBKS transfer function
    with shape parameter Gamma = Om h (k in h/Mpc)."""
    k = np.asarray(k, dtype=np.float64)
    q = np.maximum(k, 1e-30) / (Om * h)
    T = np.log1p(2.34 * q) / (2.34 * q) * (1 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3
                                          + (6.71 * q) ** 4) ** -0.25
    return k ** ns * T ** 2


def _sigma_r(Om, h, ns, R=8.0):
    lk = np.linspace(np.log(1e-5), np.log(1e3), 20001)
    k = np.exp(lk)
    x = k * R
    W = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    f = k ** 3 * bbks_spectrum(k, Om, h, ns) * W ** 2 / (2.0 * math.pi ** 2)
    return math.sqrt(np.trapezoid(f, lk))


def growth_factor(a: float, Om: float, OL: float) -> float:
    """Linear growth D(a) of flat LambdaCDM, D = (5 Om / 2) E(a) int_0^a da' / (a' E)^3,
    normalised to D ~ a early on."""
    x = np.linspace(0.0, 1.0, 4001)[1:] ** 2 * a  # dense near a' = 0
    E = np.sqrt(Om / x ** 3 + OL)
    integrand = 1.0 / (x * E) ** 3
    I = np.trapezoid(np.concatenate([[0.0], integrand]), np.concatenate([[0.0], x]))
    return 2.5 * Om * math.sqrt(Om / a ** 3 + OL) * I


def grf_displacement(seed: int, ngrid: int, box: float, Om: float, sigma8: float, h: float,
                     ns: float, a: float) -> np.ndarray:
    """Zel'dovich displacement field Psi [3][ngrid]^3 of a periodic box (side
    ``box`` Mpc/h) at scale factor a: a Gaussian random field with spectrum
    A k^ns T^2(k) normalised to sigma8 at a = 1 and scaled by D(a)/D(1);
    Psi(k) = i k / k^2 delta(k)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp2 = (sigma8 / _sigma_r(Om, h, ns)) ** 2 * (growth_factor(a, Om, 1 - Om) / growth_factor(1.0, Om, 1 - Om)) ** 2
    white = rng.standard_normal((ngrid, ngrid, ngrid))
    wk = np.fft.rfftn(white)
    kf = 2.0 * math.pi / box
    kx = np.fft.fftfreq(ngrid, d=1.0 / ngrid) * kf
    kz = np.fft.rfftfreq(ngrid, d=1.0 / ngrid) * kf
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    pk = amp2 * bbks_spectrum(np.sqrt(k2), Om, h, ns)
    delta = wk * np.sqrt(pk * ngrid ** 3 / box ** 3)
    delta[0, 0, 0] = 0.0
    psi = np.empty((3, ngrid, ngrid, ngrid))
    for c, K in enumerate((KX, KY, KZ)):
        psi[c] = np.fft.irfftn(1j * K / k2 * delta, s=(ngrid,) * 3, axes=(0, 1, 2))
    return psi


def _trilinear_periodic(field, pos, box):
    """Interpolate field [ngrid]^3 (cell-centred at i * box/ngrid) at pos [n][3]."""
    n = field.shape[0]
    u = np.mod(pos / box * n, n)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = np.zeros(pos.shape[0])
    for dx in (0, 1):
        wx = f[:, 0] if dx else 1 - f[:, 0]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1 - f[:, 1]
            for dz in (0, 1):
                wz = f[:, 2] if dz else 1 - f[:, 2]
                out += wx * wy * wz * field[(i0[:, 0] + dx) % n, (i0[:, 1] + dy) % n, (i0[:, 2] + dz) % n]
    return out


def _lattice_ball(rng, n, radius):
    """The n points of a randomly offset cubic lattice nearest the centre, the
    lattice spacing set by the ball's volume per point."""
    d = (4.0 / 3.0 * math.pi * radius ** 3 / n) ** (1.0 / 3.0)
    m = int(math.ceil(radius / d)) + 2
    g = (np.arange(-m, m + 1) * d)[:, None] + rng.uniform(0, d, size=3)[None, :]
    pts = np.stack(np.meshgrid(g[:, 0], g[:, 1], g[:, 2], indexing="ij"), axis=-1).reshape(-1, 3)
    r2 = np.einsum("ij,ij->i", pts, pts)
    return pts[np.argsort(r2, kind="stable")[:n]]


def _fibonacci_sphere(rng, n):
    """n nearly uniform unit vectors (golden-angle spiral), randomly rotated:
    its low multipoles are small, so a shell of them pulls almost nothing
    on the interior."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * k
    rxy = np.sqrt(1.0 - z * z)
    v = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return v @ (q * np.sign(np.diag(r))).T


def emulator_run(seed: int, Om: float, sigma8: float, h: float, ns: float, n_central: int = 16384,
                 n_shells: int = 32, per_shell: int = 512, r_central: float = 50.0,
                 r_max: float = 4000.0, a0: float = 0.02, ngrid: int = 128, box: float = 128.0,
                 h_min_frac: float = 1.0 / 50.0) -> Particles:
    """One training run of the correlation-function emulator (comoving).

    Central sphere: the n_central points of a cubic lattice nearest the
    centre, displaced by the Zel'dovich field of ``grf_displacement`` at a0
    (velocity f(a0) H(a0) Psi).  Shells: edges log-spaced from r_central to
    r_max, each shell's mass Om rho_crit V_shell on per_shell particles at the
    shell's volume-median radius, spread as a randomly rotated Fibonacci
    sphere and left unperturbed: random shell points would pull the central
    sphere with a dipole far larger than its own peculiar forces.  OL = 1 - Om."""
    rng = np.random.Generator(np.random.PCG64(seed))
    OL = 1.0 - Om
    rho = Om * RHO_CRIT
    central = _lattice_ball(rng, n_central, r_central)
    psi_grid = grf_displacement(seed + 7919, ngrid, box, Om, sigma8, h, ns, a0)
    psi_c = np.stack([_trilinear_periodic(psi_grid[c], central, box) for c in range(3)], axis=1)
    m_c = rho * 4.0 / 3.0 * math.pi * r_central ** 3 / n_central
    edges = r_central * (r_max / r_central) ** (np.arange(n_shells + 1) / n_shells)
    radii = np.cbrt(0.5 * (edges[:-1] ** 3 + edges[1:] ** 3))
    shell = np.concatenate([_fibonacci_sphere(rng, per_shell) * r for r in radii])
    v_shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    m_shell = np.repeat(rho * v_shell / per_shell, per_shell)
    pos = np.concatenate([central + psi_c, shell])
    psi = np.concatenate([psi_c, np.zeros_like(shell)])
    mass = np.concatenate([np.full(n_central, m_c), m_shell])
    vel = _growth_rate_hubble(a0, Om, OL) * psi
    return Particles(pos=pos, vel=vel, mass=mass, h_min=h_min_frac * math.cbrt(m_c / rho), G=1.0,
                     comoving=True, Om=Om, OL=OL, a0=a0, t0=float(flat_lcdm_time(a0, Om, OL)),
                     n_central=n_central, r_central=r_central)
