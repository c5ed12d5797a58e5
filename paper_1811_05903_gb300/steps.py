"""Thin ctypes binding of libsteps (include/steps.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The functions keep the C names.  Array arguments may be numpy arrays (host) or
torch CUDA tensors (device); both must be C-contiguous float64.  Importing this
module does not load the library; the first call does, and raises if the CUDA
library is missing or cannot be loaded -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

STEPS_OK, STEPS_EINVAL, STEPS_ENOMEM, STEPS_ECUDA, STEPS_ETIMEOUT, STEPS_ENONFINITE, STEPS_EUNSUPPORTED = range(7)
STEPS_STATIC, STEPS_COMOVING, STEPS_COMOVING_REVERSED, STEPS_PERIODIC = 0, 1, 2, 3
STEPS_GLASS_CONST_DOMEGA, STEPS_GLASS_CONST_VOLUME = 0, 1
STEPS_F32_COMP, STEPS_F32_NAIVE, STEPS_F64 = 0, 1, 2

HEADER_SYMBOLS = [
    "steps_default_config", "steps_init", "steps_forces", "steps_kdk_step", "steps_kdk_run",
    "steps_get_state", "steps_set_state", "steps_checkpoint_size", "steps_checkpoint_save",
    "steps_checkpoint_load", "steps_diagnostics", "steps_size", "steps_free", "steps_strerror",
    "steps_last_error", "steps_set_wait_limit", "steps_set_memory_limit", "steps_num_variants",
    "steps_variant_name", "steps_forces_subset", "steps_profile_enable", "steps_profile_read",
    "steps_profile_read_far", "steps_timestep", "steps_kdk_run_adaptive", "steps_glass_layout",
    "steps_glass_place",
    "steps_force_stats", "steps_get_variant", "steps_forces_noalloc", "steps_set_near_alpha",
    "steps_ensemble_init", "steps_ensemble_run", "steps_ensemble_get_state", "steps_ensemble_stats",
    "steps_ensemble_variant",
    "steps_ensemble_free", "steps_paircount",
    # steps_emu.h
    "steps_emu_create", "steps_emu_set_data", "steps_emu_train", "steps_emu_predict",
    "steps_emu_gradients", "steps_emu_get_params", "steps_emu_free",
]


class StepsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


_STATUS_NAMES = {0: "STEPS_OK", 1: "STEPS_EINVAL", 2: "STEPS_ENOMEM", 3: "STEPS_ECUDA",
                 4: "STEPS_ETIMEOUT", 5: "STEPS_ENONFINITE", 6: "STEPS_EUNSUPPORTED"}


class steps_glass_spec(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("D_s", ctypes.c_double), ("R_sim", ctypes.c_double),
                ("n_radial", ctypes.c_int), ("n_shell", ctypes.c_int64), ("r_c", ctypes.c_double),
                ("rho_bar", ctypes.c_double)]


class steps_config(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("H0", ctypes.c_double), ("Om", ctypes.c_double),
                ("OL", ctypes.c_double), ("Or", ctypes.c_double), ("Ok", ctypes.c_double),
                ("mode", ctypes.c_int), ("prec", ctypes.c_int), ("resort_every", ctypes.c_int),
                ("tile_override", ctypes.c_int), ("box", ctypes.c_double), ("images", ctypes.c_int)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsteps.so.  Raises OSError if it is absent (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise OSError("libsteps.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, I64, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    lib.steps_default_config.restype = steps_config
    lib.steps_init.argtypes = [ctypes.POINTER(P), I64, P, P, P, P, D, D, D, ctypes.POINTER(steps_config), P]
    lib.steps_forces.argtypes = [P, P]
    lib.steps_kdk_step.argtypes = [P, D, P]
    lib.steps_kdk_run.argtypes = [P, I, P]
    lib.steps_timestep.argtypes = [P, D, D, D, P]
    lib.steps_glass_layout.argtypes = [ctypes.POINTER(steps_glass_spec), P, P, P, P, P]
    lib.steps_glass_place.argtypes = [ctypes.POINTER(steps_glass_spec), I64, P, P, P, P]
    lib.steps_kdk_run_adaptive.argtypes = [P, I, D, D, D, P]
    lib.steps_get_state.argtypes = [P, P, P, P, P, P]
    lib.steps_set_state.argtypes = [P, P, P, D, D]
    lib.steps_checkpoint_size.argtypes = [P, ctypes.POINTER(S)]
    lib.steps_checkpoint_save.argtypes = [P, P]
    lib.steps_checkpoint_load.argtypes = [P, P]
    lib.steps_diagnostics.argtypes = [P, P, P, P]
    lib.steps_size.argtypes = [P]
    lib.steps_size.restype = I64
    lib.steps_free.argtypes = [P]
    lib.steps_free.restype = None
    lib.steps_strerror.argtypes = [I]
    lib.steps_strerror.restype = ctypes.c_char_p
    lib.steps_last_error.restype = ctypes.c_char_p
    lib.steps_set_wait_limit.argtypes = [P, I64]
    lib.steps_set_memory_limit.argtypes = [S]
    lib.steps_forces_subset.argtypes = [P, I64, P, P]
    lib.steps_profile_enable.argtypes = [P, I]
    lib.steps_profile_read.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(I64), I]
    lib.steps_profile_read_far.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(I64)]
    lib.steps_force_stats.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.steps_get_variant.argtypes = [P, ctypes.POINTER(I)]
    lib.steps_set_near_alpha.argtypes = [P, D]
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.steps_ensemble_init.argtypes = [ctypes.POINTER(P), I, P, PP, PP, PP, PP, P, P, P,
                                        ctypes.POINTER(steps_config), P]
    lib.steps_ensemble_run.argtypes = [P, I, P]
    lib.steps_ensemble_get_state.argtypes = [P, I, P, P, P, P, P]
    lib.steps_ensemble_variant.argtypes = [P, ctypes.POINTER(I)]
    lib.steps_ensemble_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64)]
    lib.steps_paircount.argtypes = [I, P, P, P, D, I, P, P, P]
    lib.steps_ensemble_free.argtypes = [P]
    lib.steps_ensemble_free.restype = None
    lib.steps_forces_noalloc.argtypes = [I64, P, P, P, D, D, P, P]
    lib.steps_emu_create.argtypes = [ctypes.POINTER(P), P, I, P]
    lib.steps_emu_set_data.argtypes = [P, I64, P, P]
    lib.steps_emu_train.argtypes = [P, I, P, P, P]
    lib.steps_emu_predict.argtypes = [P, I64, P, P]
    lib.steps_emu_gradients.argtypes = [P, P, P, P, P]
    lib.steps_emu_get_params.argtypes = [P, P, P, P, P]
    lib.steps_emu_free.argtypes = [P]
    lib.steps_emu_free.restype = None
    lib.steps_num_variants.restype = I
    lib.steps_variant_name.argtypes = [I]
    lib.steps_variant_name.restype = ctypes.c_char_p
    for name in ["steps_init", "steps_forces", "steps_kdk_step", "steps_kdk_run", "steps_timestep",
                 "steps_kdk_run_adaptive", "steps_glass_layout", "steps_glass_place", "steps_get_state",
                 "steps_set_state", "steps_checkpoint_size", "steps_checkpoint_save",
                 "steps_checkpoint_load", "steps_diagnostics", "steps_set_wait_limit",
                 "steps_set_memory_limit", "steps_forces_subset", "steps_profile_enable",
                 "steps_profile_read", "steps_profile_read_far", "steps_force_stats", "steps_get_variant",
                 "steps_forces_noalloc", "steps_set_near_alpha", "steps_ensemble_init",
                 "steps_ensemble_run", "steps_ensemble_get_state", "steps_ensemble_stats", "steps_ensemble_variant",
                 "steps_paircount", "steps_emu_create", "steps_emu_set_data", "steps_emu_train",
                 "steps_emu_predict", "steps_emu_gradients", "steps_emu_get_params"]:
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(status: int):
    if status != STEPS_OK:
        raise StepsError(status, _lib.steps_last_error().decode(errors="replace"))


def ptr(a):
    """Raw pointer of a numpy array, a torch tensor, None or an int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def _f64(a, shape):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a.reshape(shape)
    return a  # torch tensor: caller guarantees float64, contiguous


def steps_default_config() -> steps_config:
    return load().steps_default_config()


def steps_init(pos, vel, mass, soft=None, h_min=0.0, t0=0.0, a0=1.0, cfg=None, stream=None):
    """Returns an opaque context handle (int)."""
    lib = load()
    n = int(mass.shape[0])
    pos, vel, mass, soft = _f64(pos, (n, 3)), _f64(vel, (n, 3)), _f64(mass, (n,)), _f64(soft, (n,))
    h = ctypes.c_void_p()
    c = cfg if cfg is not None else lib.steps_default_config()
    _check(lib.steps_init(ctypes.byref(h), n, ptr(pos), ptr(vel), ptr(mass), ptr(soft), float(h_min),
                          float(t0), float(a0), ctypes.byref(c), stream))
    return h.value


def steps_forces(ctx, acc_out=None):
    _check(load().steps_forces(ctx, ptr(acc_out)))
    return acc_out


def steps_forces_subset(ctx, targets, acc_out=None):
    """FP64-on-GPU pair term for the caller-order rows in ``targets``."""
    if isinstance(targets, np.ndarray):
        targets = np.ascontiguousarray(targets, dtype=np.int64)
    nt = int(targets.shape[0])
    if acc_out is None:
        acc_out = np.empty((nt, 3))
    _check(load().steps_forces_subset(ctx, nt, ptr(targets), ptr(acc_out)))
    return acc_out


def steps_profile_enable(ctx, on: bool = True):
    _check(load().steps_profile_enable(ctx, 1 if on else 0))


def steps_profile_read(ctx, reset: bool = True):
    """(summed pair-force kernel ms, force launches, all kernel launches)."""
    ms, fl, kl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().steps_profile_read(ctx, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(kl),
                                     1 if reset else 0))
    return ms.value, fl.value, kl.value


def steps_profile_read_far(ctx):
    """(summed far-field kernel ms, far-field launches) since the last profile reset."""
    ms, fl = ctypes.c_double(), ctypes.c_int64()
    _check(load().steps_profile_read_far(ctx, ctypes.byref(ms), ctypes.byref(fl)))
    return ms.value, fl.value


def steps_force_stats(ctx):
    """(near tile pairs, all tile pairs) since the last call."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().steps_force_stats(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def steps_kdk_step(ctx, dt: float, want_a: bool = False):
    a = ctypes.c_double()
    _check(load().steps_kdk_step(ctx, float(dt), ctypes.byref(a) if want_a else None))
    return a.value if want_a else None


def steps_timestep(ctx, eps: float, dt_max: float, t_end: float = float("inf")) -> float:
    """Eq. 12 at the current state (device reduction); returns dt."""
    dt = ctypes.c_double()
    _check(load().steps_timestep(ctx, float(eps), float(dt_max), float(t_end), ctypes.byref(dt)))
    return dt.value


def steps_kdk_run_adaptive(ctx, nsteps: int, eps: float, dt_max: float, t_end: float = float("inf")) -> float:
    """nsteps KDK steps of Eq. 12 length, chosen on the device; returns the final t."""
    t = ctypes.c_double()
    _check(load().steps_kdk_run_adaptive(ctx, int(nsteps), float(eps), float(dt_max), float(t_end),
                                         ctypes.byref(t)))
    return t.value


def glass_spec(scheme, D_s, R_sim, n_radial, n_shell, r_c=0.0, rho_bar=1.0) -> steps_glass_spec:
    return steps_glass_spec(int(scheme), float(D_s), float(R_sim), int(n_radial), int(n_shell), float(r_c),
                            float(rho_bar))


def steps_glass_layout(spec: steps_glass_spec):
    """(n_total, n_inner, m_inner, omega edges [n_radial + 1], shell masses [n_radial])."""
    n, ni, mi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    edges = np.empty(spec.n_radial + 1)
    masses = np.empty(spec.n_radial)
    _check(load().steps_glass_layout(ctypes.byref(spec), ctypes.byref(n), ctypes.byref(ni), ctypes.byref(mi),
                                     ptr(edges), ptr(masses)))
    return n.value, ni.value, mi.value, edges, masses


def steps_glass_place(spec: steps_glass_spec, u, pos=None, mass=None, stream=None):
    """Positions [n][3] and masses [n] from uniforms u [n][3] (numpy or CUDA tensors)."""
    if isinstance(u, np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
    n = int(u.shape[0])
    if pos is None:
        pos = np.empty((n, 3))
    if mass is None:
        mass = np.empty(n)
    _check(load().steps_glass_place(ctypes.byref(spec), n, ptr(u), ptr(pos), ptr(mass), stream))
    return pos, mass


def steps_kdk_run(ctx, dts):
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    _check(load().steps_kdk_run(ctx, int(dts.size), dts.ctypes.data))


def steps_get_state(ctx, pos=None, vel=None, acc=None):
    t, a = ctypes.c_double(), ctypes.c_double()
    _check(load().steps_get_state(ctx, ptr(pos), ptr(vel), ptr(acc), ctypes.byref(t), ctypes.byref(a)))
    return t.value, a.value


def steps_set_state(ctx, pos, vel, t: float, a: float):
    _check(load().steps_set_state(ctx, ptr(pos), ptr(vel), float(t), float(a)))


def steps_checkpoint_save(ctx) -> bytes:
    lib = load()
    size = ctypes.c_size_t()
    _check(lib.steps_checkpoint_size(ctx, ctypes.byref(size)))
    buf = ctypes.create_string_buffer(size.value)
    _check(lib.steps_checkpoint_save(ctx, buf))
    return buf.raw


def steps_checkpoint_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().steps_checkpoint_load(ctx, buf))


def steps_diagnostics(ctx, potential: bool = True):
    ek, ep = ctypes.c_double(), ctypes.c_double()
    p = (ctypes.c_double * 3)()
    _check(load().steps_diagnostics(ctx, ctypes.byref(ek), ctypes.byref(ep) if potential else None, p))
    return ek.value, (ep.value if potential else None), np.array(list(p))


def steps_size(ctx) -> int:
    return int(load().steps_size(ctx))


def steps_free(ctx):
    if ctx:
        load().steps_free(ctx)


def steps_set_wait_limit(ctx, ns: int):
    _check(load().steps_set_wait_limit(ctx, int(ns)))


def steps_set_memory_limit(nbytes: int):
    _check(load().steps_set_memory_limit(int(nbytes)))


STEPS_NOALLOC_MAX_N = 8192


def steps_forces_noalloc(pos, mass, acc_out, soft=None, h_min=0.0, G=1.0, stream=None):
    """Pair term for <= STEPS_NOALLOC_MAX_N particles with no device allocation.
    pos/mass/soft/acc_out are device tensors (float64, contiguous)."""
    n = int(mass.shape[0])
    _check(load().steps_forces_noalloc(n, ptr(pos), ptr(mass), ptr(soft), float(h_min), float(G),
                                       ptr(acc_out), stream))
    return acc_out


def steps_set_near_alpha(ctx, alpha: float):
    _check(load().steps_set_near_alpha(ctx, float(alpha)))


def steps_get_variant(ctx) -> int:
    k = ctypes.c_int()
    _check(load().steps_get_variant(ctx, ctypes.byref(k)))
    return k.value


def steps_variants():
    lib = load()
    return [lib.steps_variant_name(k).decode() for k in range(lib.steps_num_variants())]


def make_config(mode=STEPS_STATIC, prec=STEPS_F32_COMP, G=1.0, H0=1.0, Om=0.3, OL=0.7, Or=0.0,
                Ok=0.0, resort_every=8, tile_override=0, box=0.0, images=0) -> steps_config:
    return steps_config(G, H0, Om, OL, Or, Ok, mode, prec, resort_every, tile_override, box, images)


def steps_paircount(offsets, pos, centres, step, edge2, stream=None):
    """Exact DD counts of point sets; returns uint64 [nsets][nbins]."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    edge2 = np.ascontiguousarray(edge2, dtype=np.int64)
    pos = _f64(pos, (-1, 3)) if isinstance(pos, np.ndarray) else pos
    centres = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    nsets, nbins = offsets.size - 1, edge2.size - 1
    dd = np.zeros((nsets, nbins), dtype=np.uint64)
    _check(load().steps_paircount(nsets, ptr(offsets), ptr(pos), ptr(centres), float(step), nbins,
                                  ptr(edge2), ptr(dd), stream))
    return dd


STEPS_EMU_IN, STEPS_EMU_WIDTH, STEPS_EMU_NPARAMS = 5, 256, 133377


def _f32(a, shape):
    if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
        return np.ascontiguousarray(a, dtype=np.float32).reshape(shape)
    return a  # torch tensor: caller guarantees float32, contiguous


class Emulator:
    """Owner of one emulator context (include/steps_emu.h)."""

    def __init__(self, params, batch=1024, stream=None):
        params = _f32(params, (STEPS_EMU_NPARAMS,))
        h = ctypes.c_void_p()
        _check(load().steps_emu_create(ctypes.byref(h), ptr(params), int(batch), stream))
        self.ctx, self.batch = h.value, int(batch)

    def set_data(self, x, t):
        x, t = _f32(x, (-1, STEPS_EMU_IN)), _f32(t, (-1,))
        _check(load().steps_emu_set_data(self.ctx, int(x.shape[0]), ptr(x), ptr(t)))

    def train(self, rows, lr):
        """rows [nsteps][batch] int32, lr [nsteps]; returns the per-step losses."""
        rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, self.batch)
        lr = np.ascontiguousarray(lr, dtype=np.float32).reshape(-1)
        losses = np.empty(rows.shape[0], dtype=np.float32)
        _check(load().steps_emu_train(self.ctx, int(rows.shape[0]), ptr(rows), ptr(lr), ptr(losses)))
        return losses

    def predict(self, x):
        x = _f32(x, (-1, STEPS_EMU_IN))
        y = np.empty(x.shape[0], dtype=np.float32)
        _check(load().steps_emu_predict(self.ctx, int(x.shape[0]), ptr(x), ptr(y)))
        return y

    def gradients(self, x, t):
        x, t = _f32(x, (self.batch, STEPS_EMU_IN)), _f32(t, (self.batch,))
        g = np.empty(STEPS_EMU_NPARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().steps_emu_gradients(self.ctx, ptr(x), ptr(t), ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def params(self):
        p, m, v = (np.empty(STEPS_EMU_NPARAMS, dtype=np.float32) for _ in range(3))
        n = ctypes.c_int64()
        _check(load().steps_emu_get_params(self.ctx, ptr(p), ptr(m), ptr(v), ctypes.byref(n)))
        return p, m, v, n.value

    def close(self):
        if self.ctx:
            load().steps_emu_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Owner of one ensemble context (many independent simulations)."""

    def __init__(self, members, cfgs, stream=None):
        """members: list of workloads.Particles-like objects (pos, vel, mass, h_min, t0, a0)."""
        lib = load()
        ns = len(members)
        self.n = [int(p.mass.shape[0]) for p in members]
        self._keep = []
        def arr(xs, shape):
            out = (ctypes.c_void_p * ns)()
            for k, x in enumerate(xs):
                if x is None:
                    out[k] = None
                    continue
                a = _f64(x, shape(k))
                self._keep.append(a)
                out[k] = ptr(a)
            return out
        pos = arr([p.pos for p in members], lambda k: (self.n[k], 3))
        vel = arr([p.vel for p in members], lambda k: (self.n[k], 3))
        mass = arr([p.mass for p in members], lambda k: (self.n[k],))
        n = np.array(self.n, dtype=np.int64)
        hmin = np.array([p.h_min for p in members], dtype=np.float64)
        t0 = np.array([p.t0 for p in members], dtype=np.float64)
        a0 = np.array([p.a0 for p in members], dtype=np.float64)
        cfg_arr = (steps_config * ns)(*cfgs)
        h = ctypes.c_void_p()
        _check(lib.steps_ensemble_init(ctypes.byref(h), ns, ptr(n), pos, vel, mass, None, ptr(hmin),
                                       ptr(t0), ptr(a0), cfg_arr, stream))
        self.ctx = h.value
        self.nsims = ns

    def run(self, dts):
        """dts: [nsims][nsteps] step lengths."""
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        _check(load().steps_ensemble_run(self.ctx, int(dts.shape[1]), dts.ctypes.data))

    def state(self, s):
        n = self.n[s]
        pos, vel, acc = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
        t, a = ctypes.c_double(), ctypes.c_double()
        _check(load().steps_ensemble_get_state(self.ctx, s, ptr(pos), ptr(vel), ptr(acc),
                                               ctypes.byref(t), ctypes.byref(a)))
        return pos, vel, acc, t.value, a.value

    def stats(self):
        tp, nn, na = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().steps_ensemble_stats(self.ctx, ctypes.byref(tp), ctypes.byref(nn), ctypes.byref(na)))
        return tp.value, nn.value, na.value

    def variant(self) -> int:
        k = ctypes.c_int()
        _check(load().steps_ensemble_variant(self.ctx, ctypes.byref(k)))
        return k.value

    def close(self):
        if self.ctx:
            load().steps_ensemble_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Convenience owner of one context (frees it on close/GC)."""

    def __init__(self, pos, vel, mass, soft=None, h_min=0.0, t0=0.0, a0=1.0, cfg=None, stream=None):
        self.n = int(mass.shape[0])
        self.ctx = steps_init(pos, vel, mass, soft, h_min, t0, a0, cfg, stream)

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.n, 3))
        steps_forces(self.ctx, out)
        return out

    def step(self, dt, want_a=False):
        return steps_kdk_step(self.ctx, dt, want_a)

    def run(self, dts):
        steps_kdk_run(self.ctx, dts)

    def timestep(self, eps, dt_max, t_end=float("inf")):
        return steps_timestep(self.ctx, eps, dt_max, t_end)

    def run_adaptive(self, nsteps, eps, dt_max, t_end=float("inf")):
        return steps_kdk_run_adaptive(self.ctx, nsteps, eps, dt_max, t_end)

    def state(self):
        pos, vel, acc = np.empty((self.n, 3)), np.empty((self.n, 3)), np.empty((self.n, 3))
        t, a = steps_get_state(self.ctx, pos, vel, acc)
        return pos, vel, acc, t, a

    def close(self):
        if self.ctx:
            steps_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
