"""FP64 CPU oracle for the StePS direct-summation path.

TEST INFRASTRUCTURE ONLY.  The plain, slow, obviously-correct definition of
what the GPU library computes: the spline-softened pair sum (Eq. 3, 4, 8), the
mass-tied softening (Eq. 7), the kick-drift-kick step (Eq. 9-11) with an RK4
scale factor (Eq. 1), the adaptive step length (Eq. 12), the periodic image sum
(Eq. 2, Eq. 5) and its KDK step, the pair potential,
pair counts and the emulator MLP.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

The C part (``steps_oracle.c``) is compiled with gcc on first use; ``build()``
does it explicitly.  The MLP oracle is plain numpy in ``mlp.py``; the
spherical-glass layout and placement (Eq. 14-18) are plain numpy in
``glass.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "steps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-D_GNU_SOURCE"]


def build(force: bool = False) -> str:
    """Compile ``steps_oracle.c`` into ``liboracle.so`` (gcc, no SIMD flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cosmo(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("H0", ctypes.c_double), ("Om", ctypes.c_double),
                ("OL", ctypes.c_double), ("Or", ctypes.c_double), ("Ok", ctypes.c_double),
                ("comoving", ctypes.c_int), ("reversed", ctypes.c_int)]


def cosmo(G=1.0, H0=1.0, Om=0.3, OL=0.7, Or=0.0, Ok=0.0, comoving=True, reversed=False) -> Cosmo:
    """reversed: Eq. 8 with gravity reversed (pair and background terms change
    sign; comoving only), as in the glass relaxation of Sec. 3.1."""
    return Cosmo(G, H0, Om, OL, Or, Ok, 1 if (comoving or reversed) else 0, 1 if reversed else 0)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D, P, I64 = ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
        lib.oracle_spline_F.restype = D
        lib.oracle_spline_F.argtypes = [D, D]
        lib.oracle_pair_W.restype = D
        lib.oracle_pair_W.argtypes = [D, D]
        lib.oracle_softening.argtypes = [I64, P, D, P]
        lib.oracle_pair_acc.argtypes = [I64, P, P, P, D, I64, P, P]
        lib.oracle_pair_potential.restype = D
        lib.oracle_pair_potential.argtypes = [I64, P, P, P, D]
        lib.oracle_hubble.restype = D
        lib.oracle_hubble.argtypes = [D, ctypes.POINTER(Cosmo)]
        lib.oracle_rk4_a.restype = D
        lib.oracle_rk4_a.argtypes = [D, D, ctypes.POINTER(Cosmo)]
        lib.oracle_kdk_step.argtypes = [I64, P, P, P, P, P, D, P, P, ctypes.POINTER(Cosmo)]
        lib.oracle_kinetic.argtypes = [I64, P, P, P, P]
        lib.oracle_pair_acc_periodic.argtypes = [I64, P, P, P, D, D, ctypes.c_int, I64, P, P]
        lib.oracle_kdk_step_periodic.argtypes = [I64, P, P, P, P, P, D, P, P, D, D, D, D, D, D, D, ctypes.c_int]
        lib.oracle_timestep.restype = D
        lib.oracle_timestep.argtypes = [I64, P, P, P, P, D, D, D, D, ctypes.POINTER(Cosmo)]
        lib.oracle_paircount.argtypes = [I64, P, ctypes.c_int, P, P]
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def spline_F(r: float, h: float) -> float:
    """Eq. 4, the scalar kernel magnitude (per unit G m)."""
    return _load().oracle_spline_F(float(r), float(h))


def pair_W(r: float, H: float) -> float:
    """Pair potential per unit G m_i m_j (antiderivative of Eq. 4)."""
    return _load().oracle_pair_W(float(r), float(H))


def softening(m, h_min: float) -> np.ndarray:
    """Eq. 7, h_i = (m_i / m_min)^(1/3) h_min."""
    m = _f64(m)
    out = np.empty_like(m)
    _load().oracle_softening(m.size, _ptr(m), float(h_min), _ptr(out))
    return out


def pair_acc(pos, m, h, G: float = 1.0, targets=None) -> np.ndarray:
    """Pair term of Eq. 8 (G included, no 1/a^3) for the selected target rows."""
    pos = _f64(pos, (-1, 3))
    m, h = _f64(m), _f64(h)
    n = pos.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = targets.size, _ptr(targets)
    out = np.empty((nt, 3), dtype=np.float64)
    _load().oracle_pair_acc(n, _ptr(pos), _ptr(m), _ptr(h), float(G), nt, tp, _ptr(out))
    return out


def pair_acc_periodic(pos, m, h, G: float, L: float, images: int = 0, targets=None) -> np.ndarray:
    """Periodic pair term (Eq. 2 with Eq. 5): images = 0 sums every image with
    |x_i - x_j - nL| < 2.6 L, images = 1 keeps the leading (nearest) one."""
    pos = _f64(pos, (-1, 3))
    m, h = _f64(m), _f64(h)
    n = pos.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = targets.size, _ptr(targets)
    out = np.empty((nt, 3), dtype=np.float64)
    _load().oracle_pair_acc_periodic(n, _ptr(pos), _ptr(m), _ptr(h), float(G), float(L), int(images), nt, tp,
                                     _ptr(out))
    return out


class KDKPeriodic:
    """Literal KDK (Eq. 9-11) of the periodic comoving equation of motion (Eq. 2):
    no background term, positions wrapped into [0, L)^3 after each drift."""

    def __init__(self, pos, vel, m, h, L: float, images: int = 0, G=1.0, H0=1.0, Om=1.0, OL=0.0, Or=0.0,
                 Ok=0.0, a0: float = 1.0, t0: float = 0.0):
        self.pos = _f64(pos, (-1, 3)).copy()
        self.vel = _f64(vel, (-1, 3)).copy()
        self.m = _f64(m).copy()
        self.h = _f64(h).copy()
        self.L, self.images = float(L), int(images)
        self.par = (float(G), float(H0), float(Om), float(OL), float(Or), float(Ok))
        self.a = ctypes.c_double(a0)
        self.t = ctypes.c_double(t0)
        self.acc = pair_acc_periodic(self.pos, self.m, self.h, G, L, images)

    def step(self, dt: float):
        _load().oracle_kdk_step_periodic(self.m.size, _ptr(self.pos), _ptr(self.vel), _ptr(self.acc),
                                         _ptr(self.m), _ptr(self.h), float(dt), ctypes.byref(self.a),
                                         ctypes.byref(self.t), *self.par, self.L, self.images)


def pair_potential(pos, m, h, G: float = 1.0) -> float:
    pos = _f64(pos, (-1, 3))
    m, h = _f64(m), _f64(h)
    return _load().oracle_pair_potential(pos.shape[0], _ptr(pos), _ptr(m), _ptr(h), float(G))


def hubble(a: float, c: Cosmo) -> float:
    """Eq. 1, H(a) = adot/a."""
    return _load().oracle_hubble(float(a), ctypes.byref(c))


def rk4_a(a: float, dt: float, c: Cosmo) -> float:
    return _load().oracle_rk4_a(float(a), float(dt), ctypes.byref(c))


def timestep(pos, vel, acc, h, eps: float, dt_max: float, a: float, c: Cosmo,
             t_left: float = float("inf")) -> float:
    """Eq. 12: min(dt_max, min_i sqrt(2 * 2.8 h_i * eps / |A_i|)), A_i the kick's
    acceleration at the current state (acc = pair term, G included)."""
    pos, vel, acc = _f64(pos, (-1, 3)), _f64(vel, (-1, 3)), _f64(acc, (-1, 3))
    h = _f64(h)
    return _load().oracle_timestep(h.size, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(h), float(eps),
                                   float(dt_max), float(t_left), float(a), ctypes.byref(c))


def kinetic(vel, m):
    vel, m = _f64(vel, (-1, 3)), _f64(m)
    e = ctypes.c_double()
    p = np.zeros(3)
    _load().oracle_kinetic(m.size, _ptr(vel), _ptr(m), ctypes.byref(e), _ptr(p))
    return e.value, p


class KDK:
    """Literal KDK integrator state (Eq. 9-11) in FP64, caller-owned arrays."""

    def __init__(self, pos, vel, m, h, c: Cosmo, a0: float = 1.0, t0: float = 0.0):
        self.pos = _f64(pos, (-1, 3)).copy()
        self.vel = _f64(vel, (-1, 3)).copy()
        self.m = _f64(m).copy()
        self.h = _f64(h).copy()
        self.c = c
        self.a = ctypes.c_double(a0)
        self.t = ctypes.c_double(t0)
        self.acc = pair_acc(self.pos, self.m, self.h, -c.G if c.reversed else c.G)

    def step(self, dt: float):
        _load().oracle_kdk_step(self.m.size, _ptr(self.pos), _ptr(self.vel), _ptr(self.acc),
                                _ptr(self.m), _ptr(self.h), float(dt), ctypes.byref(self.a),
                                ctypes.byref(self.t), ctypes.byref(self.c))

    def timestep(self, eps: float, dt_max: float, t_end: float = float("inf")) -> float:
        """Eq. 12 at the current state, limited to t_end - t."""
        return timestep(self.pos, self.vel, self.acc, self.h, eps, dt_max, self.a.value, self.c,
                        t_left=t_end - self.t.value)

    def adaptive_step(self, eps: float, dt_max: float, t_end: float = float("inf")) -> float:
        """One KDK step (Eq. 9-11) whose length is Eq. 12 at the step's start."""
        dt = self.timestep(eps, dt_max, t_end)
        self.step(dt)
        return dt

    def energy(self):
        ek, _ = kinetic(self.vel, self.m)
        return ek + pair_potential(self.pos, self.m, self.h, self.c.G)


def paircount(q, edge2) -> np.ndarray:
    """Integer pair counts of fixed-point positions q[n][3] (int32) in squared-edge bins."""
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1, 3)
    edge2 = np.ascontiguousarray(edge2, dtype=np.int64)
    nb = edge2.size - 1
    dd = np.zeros(nb, dtype=np.uint64)
    _load().oracle_paircount(q.shape[0], _ptr(q), nb, _ptr(edge2), _ptr(dd))
    return dd


def ball_pair_cdf(s, R: float):
    """Fraction of pairs of independent uniform points in a ball of radius R
    that lie closer than s: the integral of the pair-distance density
    p(s) = (3 s^2 / R^3)(1 - 3s/(4R) + s^3/(16 R^3)) on [0, 2R]."""
    x = np.clip(np.asarray(s, dtype=np.float64) / R, 0.0, 2.0)
    return x ** 3 - 9.0 / 16.0 * x ** 4 + x ** 6 / 32.0


def rr_ball(n: int, R: float, edges) -> np.ndarray:
    """Expected pair counts RR per bin for n uniform points in a ball."""
    return 0.5 * n * (n - 1) * np.diff(ball_pair_cdf(edges, R))


def xi_natural(dd, n: int, R: float, edges) -> np.ndarray:
    """Natural estimator xi = DD/RR - 1 of the central sphere's correlation function."""
    return np.asarray(dd, dtype=np.float64) / rr_ball(n, R, edges) - 1.0
