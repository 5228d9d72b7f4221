"""FP64 CPU oracle for the DPD fluid step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it.
It is a plain restatement of the paper's method (Sec. 2.1 Eqs. 1-5, the
Sec. 3.2 cell list, the Sec. 3.1 fused velocity-Verlet, the Sec. 4.2 periodic
Poiseuille force) in double precision; see ``dpd_oracle.c`` for the per-
function citations.

The C source is compiled on first use with gcc (``-O2 -fopenmp
-ffp-contract=off``, so x86-64 and aarch64 hosts round identically) into
``oracle/_build/``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_BRUTE = 0
MODE_CELLS = 1
FB_NONE, FB_CONST, FB_POISEUILLE = 0, 1, 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double * 3),
        ("a", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("kexp", ctypes.c_double),
        ("fb", ctypes.c_double),
        ("fb_mode", ctypes.c_int),
        ("fb_flow", ctypes.c_int),
        ("fb_grad", ctypes.c_int),
        ("rounds", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("noise", ctypes.c_int),
        ("nspec", ctypes.c_int),
        ("species", ctypes.POINTER(ctypes.c_int32)),
        ("sa", ctypes.c_double * 16),
        ("sg", ctypes.c_double * 16),
        ("src", ctypes.c_double * 16),
    ]


@dataclass
class Params:
    """DPD parameters as the oracle reads them (names follow Sec. 2.1)."""
    L: tuple = (8.0, 8.0, 8.0)
    a: float = 25.0
    gamma: float = 4.5
    kT: float = 1.0
    rc: float = 1.0
    dt: float = 0.005
    mass: float = 1.0
    kexp: float = 1.0
    fb: float = 0.0
    fb_mode: int = FB_NONE
    fb_flow: int = 2
    fb_grad: int = 0
    rounds: int = 10
    seed: int = 0
    noise: int = 0   # 0 uniform, 1 Gaussian
    # several species: per-pair tables (S x S, symmetric) and the species of
    # each particle by id; nspec = 1 uses a, gamma, rc
    nspec: int = 1
    species: object = None
    sa: object = None
    sg: object = None
    src: object = None

    def set_species(self, species, a, gamma, rc):
        """Species of each particle (by id) and the S x S interaction tables."""
        a, gamma, rc = (np.asarray(t, dtype=np.float64) for t in (a, gamma, rc))
        S = a.shape[0]
        assert 1 <= S <= 4 and a.shape == gamma.shape == rc.shape == (S, S)
        self.nspec = S
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        pad = lambda t: [float(t[s, u]) if s < S and u < S else 0.0
                         for s in range(4) for u in range(4)]
        self.sa, self.sg, self.src = pad(a), pad(gamma), pad(rc)
        return self

    def c(self) -> _Params:
        L = np.broadcast_to(np.asarray(self.L, dtype=np.float64), (3,))
        zeros = [0.0] * 16
        sp = None
        if self.species is not None:
            self._species_c = np.ascontiguousarray(self.species, dtype=np.int32)
            sp = self._species_c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        return _Params((ctypes.c_double * 3)(*L), self.a, self.gamma, self.kT, self.rc,
                       self.dt, self.mass, self.kexp, self.fb, self.fb_mode, self.fb_flow,
                       self.fb_grad, self.rounds, self.seed, self.noise, self.nspec, sp,
                       (ctypes.c_double * 16)(*(self.sa or zeros)),
                       (ctypes.c_double * 16)(*(self.sg or zeros)),
                       (ctypes.c_double * 16)(*(self.src or zeros)))


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    dp, u32p, i64p = P(ctypes.c_double), P(ctypes.c_uint32), P(ctypes.c_int64)
    pp = P(_Params)
    lib.orc_philox4x32.argtypes = [u32p, u32p, ctypes.c_int, u32p]
    lib.orc_pair_word.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_int]
    lib.orc_pair_word.restype = ctypes.c_uint32
    lib.orc_xi_from_word.argtypes = [ctypes.c_uint32]
    lib.orc_xi_from_word.restype = ctypes.c_double
    lib.orc_rng.argtypes = [ctypes.c_int64, u32p, u32p, ctypes.c_uint64, ctypes.c_uint64,
                            ctypes.c_int, u32p, dp]
    lib.orc_rng_gauss.argtypes = [ctypes.c_int64, u32p, u32p, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_int, u32p, u32p, dp]
    lib.orc_xi_gauss.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    lib.orc_xi_gauss.restype = ctypes.c_double
    lib.orc_pair_force.argtypes = [pp, dp, dp, dp, dp, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint64, dp, dp]
    lib.orc_forces.argtypes = [pp, ctypes.c_int64, dp, dp, u32p, ctypes.c_uint64, ctypes.c_int,
                               dp, dp]
    lib.orc_forces.restype = ctypes.c_int
    lib.orc_forces_subset.argtypes = [pp, ctypes.c_int64, dp, dp, u32p, ctypes.c_uint64,
                                      ctypes.c_int64, i64p, dp]
    lib.orc_forces_subset.restype = ctypes.c_int
    lib.orc_run.argtypes = [pp, ctypes.c_int64, dp, dp, u32p, dp, ctypes.c_uint64,
                            ctypes.c_int64, ctypes.c_int, dp]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_stats.argtypes = [pp, ctypes.c_int64, dp, ctypes.c_double, dp]
    lib.orc_profile.argtypes = [pp, ctypes.c_int64, dp, dp, ctypes.c_int, dp, i64p]
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ids(n, ids=None):
    if ids is None:
        return np.arange(n, dtype=np.uint32)
    return np.ascontiguousarray(ids, dtype=np.uint32)


# ---------------------------------------------------------------- RNG

def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    """Philox-4x32-R block function on one counter (4 words) and key (2 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), rounds,
                       _ptr(out, ctypes.c_uint32))
    return out


def pair_rng(ida, idb, step: int, seed: int, rounds: int = 10):
    """Words u and noise values xi for the pairs (ida[k], idb[k]) at ``step``."""
    lib = _load()
    a = np.ascontiguousarray(ida, dtype=np.uint32)
    b = np.ascontiguousarray(idb, dtype=np.uint32)
    n = a.size
    words = np.zeros(n, dtype=np.uint32)
    xi = np.zeros(n, dtype=np.float64)
    lib.orc_rng(n, _ptr(a, ctypes.c_uint32), _ptr(b, ctypes.c_uint32), step, seed, rounds,
                _ptr(words, ctypes.c_uint32), _ptr(xi, ctypes.c_double))
    return words, xi


def pair_rng_gauss(ida, idb, step: int, seed: int, rounds: int = 10):
    """Words 0, 1 and the Gaussian noise values for the pairs (ida[k], idb[k])."""
    lib = _load()
    a = np.ascontiguousarray(ida, dtype=np.uint32)
    b = np.ascontiguousarray(idb, dtype=np.uint32)
    n = a.size
    w0 = np.zeros(n, dtype=np.uint32)
    w1 = np.zeros(n, dtype=np.uint32)
    xi = np.zeros(n, dtype=np.float64)
    lib.orc_rng_gauss(n, _ptr(a, ctypes.c_uint32), _ptr(b, ctypes.c_uint32), step, seed, rounds,
                      _ptr(w0, ctypes.c_uint32), _ptr(w1, ctypes.c_uint32),
                      _ptr(xi, ctypes.c_double))
    return w0, w1, xi


def xi_gauss(u0: int, u1: int) -> float:
    return _load().orc_xi_gauss(int(u0), int(u1))


def xi_from_word(u: int) -> float:
    return _load().orc_xi_from_word(int(u))


# ---------------------------------------------------------------- forces

def pair_force(p: Params, xi, xj, vi, vj, idi: int, idj: int, step: int):
    """F_ij and r_ij . F^C_ij for one pair."""
    lib = _load()
    xi, xj, vi, vj = (_f64(t, (3,)) for t in (xi, xj, vi, vj))
    f = np.zeros(3)
    rfc = np.zeros(1)
    lib.orc_pair_force(ctypes.byref(p.c()), _ptr(xi, ctypes.c_double), _ptr(xj, ctypes.c_double),
                       _ptr(vi, ctypes.c_double), _ptr(vj, ctypes.c_double), idi, idj, step,
                       _ptr(f, ctypes.c_double), _ptr(rfc, ctypes.c_double))
    return f, float(rfc[0])


def forces(p: Params, x, v, step: int = 0, ids=None, mode: int = MODE_BRUTE):
    """Total force on every particle (pair sum + body force) and the virial."""
    lib = _load()
    x = _f64(x)
    v = _f64(v)
    n = x.shape[0]
    ids = _ids(n, ids)
    f = np.zeros((n, 3))
    vir = np.zeros(1)
    rc = lib.orc_forces(ctypes.byref(p.c()), n, _ptr(x, ctypes.c_double), _ptr(v, ctypes.c_double),
                        _ptr(ids, ctypes.c_uint32), step, mode, _ptr(f, ctypes.c_double),
                        _ptr(vir, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle forces failed ({rc})")
    return f, float(vir[0])


def forces_subset(p: Params, x, v, which, step: int = 0, ids=None):
    """Forces on particles ``which`` only, from the cell list over all of x."""
    lib = _load()
    x = _f64(x)
    v = _f64(v)
    n = x.shape[0]
    ids = _ids(n, ids)
    w = np.ascontiguousarray(which, dtype=np.int64)
    f = np.zeros((w.size, 3))
    rc = lib.orc_forces_subset(ctypes.byref(p.c()), n, _ptr(x, ctypes.c_double),
                               _ptr(v, ctypes.c_double), _ptr(ids, ctypes.c_uint32), step, w.size,
                               _ptr(w, ctypes.c_int64), _ptr(f, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle forces_subset failed ({rc})")
    return f


class State:
    """Oracle state (x, v at the full step, f) advanced by ``run``."""

    def __init__(self, p: Params, x, v, ids=None, step: int = 0, mode: int = MODE_BRUTE):
        self.p = p
        self.x = _f64(x).copy()
        self.v = _f64(v).copy()
        self.n = self.x.shape[0]
        self.ids = _ids(self.n, ids).copy()
        self.step = step
        self.mode = mode
        self.f, self.virial = forces(p, self.x, self.v, step, self.ids, mode)

    def run(self, nsteps: int):
        lib = _load()
        vir = np.zeros(1)
        rc = lib.orc_run(ctypes.byref(self.p.c()), self.n, _ptr(self.x, ctypes.c_double),
                         _ptr(self.v, ctypes.c_double), _ptr(self.ids, ctypes.c_uint32),
                         _ptr(self.f, ctypes.c_double), self.step, nsteps, self.mode,
                         _ptr(vir, ctypes.c_double))
        if rc:
            raise ValueError(f"oracle run failed ({rc})")
        if nsteps > 0:
            self.virial = float(vir[0])
        self.step += nsteps
        return self

    def stats(self) -> dict:
        lib = _load()
        out = np.zeros(6)
        lib.orc_stats(ctypes.byref(self.p.c()), self.n, _ptr(self.v, ctypes.c_double),
                      self.virial, _ptr(out, ctypes.c_double))
        return {"P": out[0:3].copy(), "KE": out[3], "kT": out[4], "pressure": out[5]}

    def profile(self, nbins: int):
        lib = _load()
        prof = np.zeros(nbins)
        cnt = np.zeros(nbins, dtype=np.int64)
        lib.orc_profile(ctypes.byref(self.p.c()), self.n, _ptr(self.x, ctypes.c_double),
                        _ptr(self.v, ctypes.c_double), nbins, _ptr(prof, ctypes.c_double),
                        _ptr(cnt, ctypes.c_int64))
        return prof, cnt


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(t: int):
    _load().orc_set_num_threads(int(t))
