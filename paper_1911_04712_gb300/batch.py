"""Binding of the multi-box batch (dpd_batch_*) and the kernel tuning table:
argument marshalling only, like ``dpd``."""

from __future__ import annotations

import ctypes
import json
import os

import numpy as np

BATCH_GRAPH_CHUNK = 100
NUM_FORCE_VARIANTS = 14
TUNING_PACKED = 2
# tuning tables: single box (full, half stencil) and packed sets of boxes
TABLES = (("full", 0), ("half", 1), ("full_packed", 2), ("half_packed", 3))
MAX_DENSITY_BANDS = 8
TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


class BoxDesc(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("a", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kT", ctypes.c_double), ("rc", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("n", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("kexp", ctypes.c_double), ("mass", ctypes.c_double),
                ("body_force", ctypes.c_double), ("body_mode", ctypes.c_int),
                ("flow_axis", ctypes.c_int), ("grad_axis", ctypes.c_int), ("noise", ctypes.c_int),
                ("nspecies", ctypes.c_int), ("species_a", ctypes.c_double * 16),
                ("species_gamma", ctypes.c_double * 16), ("species_rc", ctypes.c_double * 16)]


def declare(L):
    """Argument types of the batch and tuning entry points (called by dpd.lib())."""
    c = ctypes
    vp, i64, dbl, i32 = c.c_void_p, c.c_int64, c.c_double, c.c_int
    from .dpd import Stats
    L.dpd_force_variant_info.argtypes = [i32, c.POINTER(i32), c.POINTER(i32)]
    L.dpd_tuning_set.argtypes = [i32, i32, c.POINTER(dbl), c.POINTER(i32)]
    L.dpd_tuning_get.argtypes = [i32, i32, c.POINTER(dbl), c.POINTER(i32), c.POINTER(i32)]
    L.dpd_batch_create.argtypes = [c.POINTER(vp), i32, c.POINTER(BoxDesc)]
    L.dpd_batch_destroy.argtypes = [vp]
    L.dpd_batch_set_stream.argtypes = [vp, vp]
    L.dpd_batch_set_option.argtypes = [vp, i32, dbl]
    L.dpd_batch_set_state.argtypes = [vp, i32, vp, vp, i32]
    L.dpd_batch_set_state_species.argtypes = [vp, i32, vp, vp, vp, i32]
    L.dpd_batch_step.argtypes = [vp, i64]
    L.dpd_batch_get_state.argtypes = [vp, i32, vp, vp, i32]
    L.dpd_batch_get_forces.argtypes = [vp, i32, vp, i32]
    L.dpd_batch_get_stats.argtypes = [vp, c.POINTER(Stats)]
    L.dpd_batch_profile_steps.argtypes = [vp, i64, c.POINTER(dbl)]
    L.dpd_batch_num_boxes.argtypes = [vp]
    for name in ("dpd_force_variant_info", "dpd_tuning_set", "dpd_tuning_get", "dpd_batch_create",
                 "dpd_batch_destroy", "dpd_batch_set_stream", "dpd_batch_set_option",
                 "dpd_batch_set_state", "dpd_batch_set_state_species", "dpd_batch_step",
                 "dpd_batch_get_state",
                 "dpd_batch_get_forces", "dpd_batch_get_stats", "dpd_batch_profile_steps",
                 "dpd_batch_num_boxes"):
        getattr(L, name).restype = i32
    _load_tuning_file(L)
    return L


def _load_tuning_file(L):
    """Install the committed per-density-band table, if present."""
    if not os.path.exists(TUNING_FILE):
        return
    with open(TUNING_FILE) as f:
        table = json.load(f)
    for stencil_name, stencil in TABLES:
        bands = table.get(stencil_name)
        if not bands:
            continue
        up = (ctypes.c_double * len(bands))(*[b["rho_upper"] for b in bands])
        var = (ctypes.c_int * len(bands))(*[b["variant"] for b in bands])
        L.dpd_tuning_set(stencil, len(bands), up, var)


def _lib():
    from . import dpd
    return dpd.lib()


def _check(rc):
    from . import dpd
    return dpd.check(rc)


def variant_info(v: int) -> tuple:
    t, c = ctypes.c_int(), ctypes.c_int()
    _check(_lib().dpd_force_variant_info(v, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def tuning_set(table: int, rho_upper, variants):
    """Set tuning table `table`: stencil (0 full, 1 half) + TUNING_PACKED for packed sets."""
    up = (ctypes.c_double * len(rho_upper))(*rho_upper)
    var = (ctypes.c_int * len(variants))(*variants)
    _check(_lib().dpd_tuning_set(table, len(rho_upper), up, var))


def tuning_get(table: int):
    n = ctypes.c_int()
    up = (ctypes.c_double * MAX_DENSITY_BANDS)()
    var = (ctypes.c_int * MAX_DENSITY_BANDS)()
    _check(_lib().dpd_tuning_get(table, MAX_DENSITY_BANDS, up, var, ctypes.byref(n)))
    return list(up[:n.value]), list(var[:n.value])


def make_desc(L, n, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=0, steps=0, kexp=1.0,
              mass=1.0, body_force=0.0, body_mode=0, flow_axis=2, grad_axis=0,
              noise=0, species=None) -> BoxDesc:
    """species: None, or (a, gamma, rc) S x S tables of several species."""
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    nsp, tabs = 1, [[0.0] * 16 for _ in range(3)]
    if species is not None:
        t = [np.asarray(x, dtype=np.float64) for x in species]
        nsp = t[0].shape[0]
        tabs = [[float(x[s, u]) if s < nsp and u < nsp else 0.0 for s in range(4)
                 for u in range(4)] for x in t]
    return BoxDesc((ctypes.c_double * 3)(*L3), a, gamma, kT, rc, dt, int(seed), int(n),
                   int(steps), kexp, mass, body_force, body_mode, flow_axis, grad_axis, noise,
                   nsp, *[(ctypes.c_double * 16)(*x) for x in tabs])


class Batch:
    """Many independent periodic boxes stepped together (dpd_batch_*)."""

    def __init__(self, descs, stream=None, stencil=None, variant=None, graph_chunk=None):
        from .dpd import _stream_ptr
        arr = (BoxDesc * len(descs))(*descs)
        self._b = ctypes.c_void_p()
        _check(_lib().dpd_batch_create(ctypes.byref(self._b), len(descs), arr))
        self.n = [int(d.n) for d in descs]
        self.nbox = len(descs)
        self._stream_ref = stream
        if stream is not None:
            _check(_lib().dpd_batch_set_stream(self._b, _stream_ptr(stream)))
        if stencil is not None:
            self.set_option(7, stencil)
        if variant is not None:
            self.set_option(11, variant)
        if graph_chunk is not None:
            self.set_option(BATCH_GRAPH_CHUNK, graph_chunk)

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            _lib().dpd_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value):
        _check(_lib().dpd_batch_set_option(self._b, int(key), float(value)))

    def set_state(self, box: int, pos, vel, species=None):
        """Load box `box`; species: one int per particle (host, same memory as pos), or None."""
        from .dpd import WHERE_HOST, _vec3_arg
        pp, wp, kp = _vec3_arg(pos, self.n[box])
        vv, wv, kv = _vec3_arg(vel, self.n[box])
        if wp != wv:
            raise ValueError("pos and vel must both be host arrays or both CUDA tensors")
        if species is None:
            _check(_lib().dpd_batch_set_state(self._b, box, pp, vv, wp))
        else:
            if wp != WHERE_HOST:
                raise ValueError("species with host positions and velocities")
            sp = np.ascontiguousarray(species, dtype=np.int32).reshape(-1)
            if sp.size != self.n[box]:
                raise ValueError("species must have one entry per particle")
            _check(_lib().dpd_batch_set_state_species(self._b, box, pp, vv,
                                                      sp.ctypes.data_as(ctypes.c_void_p), wp))

    def step(self, nsteps: int = 1):
        _check(_lib().dpd_batch_step(self._b, int(nsteps)))

    def profile(self, nsteps: int) -> list:
        ms = (ctypes.c_double * 5)()
        _check(_lib().dpd_batch_profile_steps(self._b, int(nsteps), ms))
        return list(ms)

    def get_state(self, box: int):
        n = self.n[box]
        pos = np.empty((n, 3), dtype=np.float32)
        vel = np.empty_like(pos)
        _check(_lib().dpd_batch_get_state(self._b, box, pos.ctypes.data_as(ctypes.c_void_p),
                                          vel.ctypes.data_as(ctypes.c_void_p), 0))
        return pos, vel

    def get_forces(self, box: int):
        f = np.empty((self.n[box], 3), dtype=np.float32)
        _check(_lib().dpd_batch_get_forces(self._b, box, f.ctypes.data_as(ctypes.c_void_p), 0))
        return f

    def stats(self) -> list:
        from .dpd import Stats
        out = (Stats * self.nbox)()
        _check(_lib().dpd_batch_get_stats(self._b, out))
        return [s.as_dict() for s in out]
