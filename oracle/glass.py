"""Oracle for the spherical-glass initial conditions (Sec. 3.1, Eq. 14-18).

TEST INFRASTRUCTURE ONLY: the plain numpy/scipy definition that the library's
glass layout and placement are checked against.  Only the test suite may
import it.  It shares no code with the CUDA path.

Compactification (Eq. 14-15): a real-space point at radius r maps to the
angle omega = 2 arctan(r / D_s) on the 3-sphere of diameter D_s, and back by
r = D_s tan(omega / 2).  The 3-sphere of radius R = D_s / 2 has volume element
R^3 sin^2(omega) sin(theta) d omega d theta d phi, so the compact volume inside
omega is V(omega) = (pi D_s^3 / 8)(2 omega - sin 2 omega), the form of Eq. 18.

Layouts (readings where the paper is silent are marked):
  * constant delta-omega (scheme 0): shells of equal width in omega between
    omega_c = 2 arctan(r_c / D_s) and omega_max = 2 arctan(R_sim / D_s)
    [reading: the shells start at omega_c]; the ball r < r_c is one united
    volume of N_inner = floor((4 pi / 3) r_c^3 rho_bar / m_inner) equal-mass
    particles (Eq. 17) [reading: m_inner is the particle mass of the first
    shell outside, so the mass is continuous at r_c], placed uniformly in real
    space [reading: equal masses represent a uniform density].
  * constant compact volume (scheme 1): edges omega_i from
    (8 V_bin / (pi D_s^3)) i = 2 omega_i - sin 2 omega_i (Eq. 18), with
    V_bin = V(omega_max) / n_radial, solved numerically.
Each shell holds n_shell particles placed uniformly in its compact volume:
omega from the density proportional to sin^2(omega) on the shell [reading of
"randomly"], direction uniform on the sphere; positions by Eq. 15.  Masses by
Eq. 16, m_j = rho_bar V_shell,j / N_shell with the real-space shell volume.
The random numbers are inputs: u[k] = (u_omega, u_cos, u_phi) in [0, 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def omega_of_r(r, D_s: float):
    """Eq. 14 (radial part): compact angle of a real-space radius."""
    return 2.0 * np.arctan(np.asarray(r, dtype=np.float64) / D_s)


def r_of_omega(omega, D_s: float):
    """Eq. 15 (radial part): real-space radius of a compact angle."""
    return D_s * np.tan(0.5 * np.asarray(omega, dtype=np.float64))


def compact_volume(omega, D_s: float):
    """Compact volume inside angle omega on the 3-sphere of diameter D_s."""
    w = np.asarray(omega, dtype=np.float64)
    return math.pi * D_s ** 3 / 8.0 * (2.0 * w - np.sin(2.0 * w))


def layout(scheme: int, D_s: float, R_sim: float, n_radial: int, n_shell: int, r_c: float,
           rho_bar: float):
    """Shell edges in omega ([n_radial + 1]), per-shell particle mass
    ([n_radial]), and the united inner ball (n_inner, m_inner; 0 for scheme 1)."""
    w_max = float(omega_of_r(R_sim, D_s))
    if scheme == 0:
        w_c = float(omega_of_r(r_c, D_s))
        edges = w_c + (w_max - w_c) * np.arange(n_radial + 1) / n_radial
    elif scheme == 1:
        v_bin = float(compact_volume(w_max, D_s)) / n_radial
        edges = np.empty(n_radial + 1)
        edges[0] = 0.0
        for i in range(1, n_radial + 1):
            target = 8.0 * v_bin / (math.pi * D_s ** 3) * i
            edges[i] = brentq(lambda w: 2.0 * w - math.sin(2.0 * w) - target, 0.0, math.pi,
                              xtol=1e-17, rtol=8.9e-16, maxiter=500)
        edges[-1] = w_max
    else:
        raise ValueError("scheme must be 0 or 1")
    r = r_of_omega(edges, D_s)
    v_shell = 4.0 * math.pi / 3.0 * (r[1:] ** 3 - r[:-1] ** 3)
    m_shell = rho_bar * v_shell / n_shell
    n_inner, m_inner = 0, 0.0
    if scheme == 0:
        m_inner = float(m_shell[0])
        n_inner = int(math.floor(4.0 * math.pi / 3.0 * r_c ** 3 * rho_bar / m_inner))
    return edges, m_shell, n_inner, m_inner


def place(scheme: int, D_s: float, R_sim: float, n_radial: int, n_shell: int, r_c: float,
          rho_bar: float, u):
    """Positions [n][3] and masses [n] from uniforms u [n][3]; the inner ball's
    particles come first, then shell 0, 1, ... (n_shell each)."""
    edges, m_shell, n_inner, m_inner = layout(scheme, D_s, R_sim, n_radial, n_shell, r_c, rho_bar)
    n = n_inner + n_radial * n_shell
    u = np.asarray(u, dtype=np.float64).reshape(n, 3)
    radius = np.empty(n)
    mass = np.empty(n)
    if n_inner:
        radius[:n_inner] = r_c * np.cbrt(u[:n_inner, 0])
        mass[:n_inner] = m_inner
    shell = np.repeat(np.arange(n_radial), n_shell)
    lo, hi = edges[shell], edges[shell + 1]
    F = lambda w: 2.0 * w - np.sin(2.0 * w)
    target = F(lo) + u[n_inner:, 0] * (F(hi) - F(lo))
    a, b = lo.copy(), hi.copy()
    for _ in range(200):                       # plain bisection on F(w) = target
        mid = 0.5 * (a + b)
        below = F(mid) < target
        a = np.where(below, mid, a)
        b = np.where(below, b, mid)
    radius[n_inner:] = r_of_omega(0.5 * (a + b), D_s)
    mass[n_inner:] = m_shell[shell]
    cos_t = 1.0 - 2.0 * u[:, 1]
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * u[:, 2]
    pos = np.stack([radius * sin_t * np.cos(phi), radius * sin_t * np.sin(phi), radius * cos_t], axis=1)
    return pos, mass
