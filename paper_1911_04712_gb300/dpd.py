"""Python binding of libdpd.so: argument marshalling only.

Every step of the DPD fluid update runs in the library's CUDA kernels.  This
module converts arrays to pointers (NumPy arrays become host pointers, CUDA
torch tensors become device pointers), checks status codes and raises
``DPDError`` with the library's message.  There is no CPU fallback: if the
shared library is missing, importing the binding's entry points raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DPD_LIBRARY selects another build of the same library (e.g. another
# Philox round count); the default is the in-tree libdpd.so.
LIB_PATH = os.environ.get("DPD_LIBRARY") or os.path.join(HERE, "libdpd.so")

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_STATE, ERR_NUMERIC, ERR_TIMEOUT, ERR_BUSY = (
    0, -1, -2, -3, -4, -5, -6, -7)
ERR_INTERNAL = -8  # checked build only: a kernel's index check failed
WHERE_HOST, WHERE_DEVICE = 0, 1
PARAM_KEXP, PARAM_MASS, PARAM_BODYFORCE, PARAM_POISEUILLE_F = 1, 2, 3, 4
PARAM_FLOW_AXIS, PARAM_GRAD_AXIS, PARAM_STENCIL = 5, 6, 7
PARAM_FORCE_TILES, PARAM_TILE_CELLS, PARAM_STAGE_CAP, PARAM_FORCE_VARIANT = 8, 9, 10, 11
PARAM_NOISE = 12
PARAM_FUSE = 13
NOISE_UNIFORM, NOISE_GAUSSIAN = 0, 1
STENCIL_FULL, STENCIL_HALF = 0, 1
NUM_STAGES, KERNELS_PER_STEP = 5, 7


def kernels_per_step(half: bool, force_bands: int = 1) -> int:
    """Kernel launches of one step: the full stencil's sequence has a key pass
    the half stencil skips, and the force kernel launches once per band."""
    return KERNELS_PER_STEP - (1 if half else 0) + (force_bands - 1)


STAGE_NAMES = ("integrate_bin", "scan", "bin_keys", "bin_scatter", "force")

_NAMES = {ERR_ARG: "DPD_ERR_ARG", ERR_NOMEM: "DPD_ERR_NOMEM", ERR_CUDA: "DPD_ERR_CUDA",
          ERR_STATE: "DPD_ERR_STATE", ERR_NUMERIC: "DPD_ERR_NUMERIC",
          ERR_TIMEOUT: "DPD_ERR_TIMEOUT", ERR_BUSY: "DPD_ERR_BUSY",
          ERR_INTERNAL: "DPD_ERR_INTERNAL"}


class DPDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("momentum", ctypes.c_double * 3), ("kinetic", ctypes.c_double),
                ("kT", ctypes.c_double), ("virial", ctypes.c_double),
                ("pressure", ctypes.c_double), ("step", ctypes.c_int64), ("n", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {"momentum": np.array(self.momentum[:]), "kinetic": self.kinetic, "kT": self.kT,
                "virial": self.virial, "pressure": self.pressure, "step": self.step, "n": self.n}


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1911_04712_gb300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    c = ctypes
    vp, i64, u64, dbl, i32 = c.c_void_p, c.c_int64, c.c_uint64, c.c_double, c.c_int
    L.dpd_last_error.restype = c.c_char_p
    L.dpd_version.restype = c.c_char_p
    L.dpd_create.argtypes = [c.POINTER(vp), c.POINTER(dbl), dbl, dbl, dbl, dbl, dbl, u64]
    L.dpd_destroy.argtypes = [vp]
    L.dpd_set_param.argtypes = [vp, i32, dbl]
    L.dpd_set_stream.argtypes = [vp, vp]
    L.dpd_get_param.argtypes = [vp, i32, c.POINTER(dbl)]
    L.dpd_get_param.restype = i32
    L.dpd_set_state.argtypes = [vp, i64, vp, vp, i32]
    L.dpd_set_state_species.argtypes = [vp, i64, vp, vp, vp, i32]
    L.dpd_set_species.argtypes = [vp, i32, c.POINTER(dbl), c.POINTER(dbl), c.POINTER(dbl)]
    L.dpd_get_species.argtypes = [vp, c.POINTER(i32), c.POINTER(dbl), c.POINTER(dbl),
                                  c.POINTER(dbl)]
    L.dpd_step.argtypes = [vp, i64]
    L.dpd_get_state.argtypes = [vp, vp, vp, i32]
    L.dpd_get_forces.argtypes = [vp, vp, i32]
    L.dpd_get_stats.argtypes = [vp, c.POINTER(Stats)]
    L.dpd_num_particles.argtypes = [vp]
    L.dpd_num_particles.restype = i64
    L.dpd_profile_steps.argtypes = [vp, i64, c.POINTER(dbl)]
    L.dpd_profile_steps.restype = i32
    L.dpd_checkpoint_size.argtypes = [vp]
    L.dpd_checkpoint_size.restype = i64
    L.dpd_checkpoint_save.argtypes = [vp, vp, i64]
    L.dpd_checkpoint_save.restype = i32
    L.dpd_checkpoint_load.argtypes = [vp, vp, i64]
    L.dpd_checkpoint_load.restype = i32
    L.dpd_debug_rng.argtypes = [vp, vp, i64, u64, u64, i32, vp, vp, vp, vp]
    L.dpd_forces_noalloc.argtypes = [i64, vp, vp, c.POINTER(dbl), dbl, dbl, dbl, dbl, dbl, u64,
                                     u64, vp, vp]
    L.dpd_forces_noalloc.restype = i32
    for name in ("dpd_set_state_species", "dpd_set_species", "dpd_get_species"):
        getattr(L, name).restype = i32
    for name in ("dpd_create", "dpd_destroy", "dpd_set_param", "dpd_set_stream", "dpd_set_state",
                 "dpd_step", "dpd_get_state", "dpd_get_forces", "dpd_get_stats",
                 "dpd_debug_rng"):
        getattr(L, name).restype = i32
    _register_batch(L)
    _lib = L
    return L


def _register_batch(L):
    """Declare the multi-box and queue entry points when the library has them."""
    try:
        from . import batch as _b
    except ImportError:  # pragma: no cover
        return
    _b.declare(L)


def check(rc: int):
    if rc != OK:
        raise DPDError(rc, lib().dpd_last_error().decode(errors="replace"))
    return rc


def _torch_int32():
    import torch
    return torch.int32


def version() -> str:
    return lib().dpd_version().decode()


def issue_rates(stream=None) -> dict:
    """Measured FP32 FMA lane-ops/s and Philox words/s of the current device
    (register-only loops timed with CUDA events; dpd_issue_rates)."""
    L = lib()
    L.dpd_issue_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    L.dpd_issue_rates.restype = ctypes.c_int
    r = (ctypes.c_double * 2)()
    check(L.dpd_issue_rates(r, _stream_ptr(stream)))
    return {"fma_lane_ops_per_s": r[0], "philox_words_per_s": r[1]}


def philox_rounds() -> int:
    """Rounds of the loaded library's Philox-4x32-R noise generator."""
    L = lib()
    L.dpd_philox_rounds.restype = ctypes.c_int
    return L.dpd_philox_rounds()


# ----------------------------------------------------------------- helpers
def _is_cuda_tensor(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _vec3_arg(x, n=None):
    """(pointer, where, keepalive) for an n x 3 float32 array or CUDA tensor."""
    if _is_cuda_tensor(x):
        import torch
        t = x.detach()
        if t.dtype != torch.float32 or not t.is_contiguous():
            t = t.to(torch.float32).contiguous()
        if t.dim() != 2 or t.shape[1] != 3 or (n is not None and t.shape[0] != n):
            raise ValueError("expected an n x 3 tensor")
        return ctypes.c_void_p(t.data_ptr()), WHERE_DEVICE, t
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3 or (n is not None and a.shape[0] != n):
        raise ValueError("expected an n x 3 array")
    return a.ctypes.data_as(ctypes.c_void_p), WHERE_HOST, a


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# --------------------------------------------------------------------- box
class Box:
    """One periodic DPD box behind the dpd_* C ABI."""

    def __init__(self, L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=0, *,
                 stencil=None, kexp=None, mass=None, body_force=None, poiseuille_f=None,
                 flow_axis=None, grad_axis=None, stream=None, tiles=None, tile_cells=None,
                 stage_cap=None, variant=None, noise=None):
        L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        self.L = tuple(float(v) for v in L3)
        self._ctx = ctypes.c_void_p()
        box = (ctypes.c_double * 3)(*self.L)
        check(lib().dpd_create(ctypes.byref(self._ctx), box, a, gamma, kT, rc, dt, int(seed)))
        self.n = 0
        for key, val in ((PARAM_FLOW_AXIS, flow_axis), (PARAM_GRAD_AXIS, grad_axis),
                         (PARAM_KEXP, kexp), (PARAM_MASS, mass), (PARAM_BODYFORCE, body_force),
                         (PARAM_POISEUILLE_F, poiseuille_f), (PARAM_STENCIL, stencil),
                         (PARAM_FORCE_TILES, tiles), (PARAM_TILE_CELLS, tile_cells),
                         (PARAM_STAGE_CAP, stage_cap), (PARAM_FORCE_VARIANT, variant),
                         (PARAM_NOISE, noise)):
            if val is not None:
                self.set_param(key, val)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().dpd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_param(self, key: int, value: float):
        check(lib().dpd_set_param(self._ctx, int(key), float(value)))

    def get_param(self, key: int) -> float:
        v = ctypes.c_double()
        check(lib().dpd_get_param(self._ctx, int(key), ctypes.byref(v)))
        return v.value

    def tiling(self) -> dict:
        """Force-kernel tiling in use: staged tiles on/off, cells per tile, staging capacity."""
        return {"tiles": int(self.get_param(PARAM_FORCE_TILES)),
                "tile_cells": int(self.get_param(PARAM_TILE_CELLS)),
                "stage_cap": int(self.get_param(PARAM_STAGE_CAP))}

    def set_stream(self, stream):
        check(lib().dpd_set_stream(self._ctx, _stream_ptr(stream)))
        self._stream_ref = stream   # the stream must outlive the work enqueued on it

    def set_state(self, pos, vel, species=None):
        """Load n particles (ids 0..n-1); species: n ints 0..nspecies-1, in the same
        memory as pos and vel (NumPy, or a CUDA int32 tensor), or None for all 0."""
        n = int(pos.shape[0])
        pp, wp, kp = _vec3_arg(pos, n)
        vv, wv, kv = _vec3_arg(vel, n)
        if wp != wv:
            raise ValueError("pos and vel must both be host arrays or both CUDA tensors")
        if species is None:
            check(lib().dpd_set_state(self._ctx, n, pp, vv, wp))
        else:
            if _is_cuda_tensor(species):
                if wp != WHERE_DEVICE or species.dtype != _torch_int32() or species.numel() != n:
                    raise ValueError("species must be a CUDA int32 tensor of n entries")
                keep = species.contiguous()
                sp = ctypes.c_void_p(keep.data_ptr())
            else:
                if wp != WHERE_HOST:
                    raise ValueError("species must be in the same memory as pos and vel")
                keep = np.ascontiguousarray(species, dtype=np.int32).reshape(-1)
                if keep.size != n:
                    raise ValueError("species must have one entry per particle")
                sp = keep.ctypes.data_as(ctypes.c_void_p)
            check(lib().dpd_set_state_species(self._ctx, n, pp, vv, sp, wp))
        self.n = n

    def set_species(self, a=None, gamma=None, rc=None):
        """Interaction tables of several species (S x S, symmetric), or no
        argument to return to one species."""
        if a is None:
            check(lib().dpd_set_species(self._ctx, 1, None, None, None))
            return
        t = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, gamma, rc)]
        S = t[0].shape[0]
        if any(x.shape != (S, S) for x in t):
            raise ValueError("a, gamma and rc must be S x S")
        ptr = [x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in t]
        check(lib().dpd_set_species(self._ctx, S, *ptr))

    def get_species(self):
        """(S, a, gamma, rc) with S x S tables (None when S is 1)."""
        S = ctypes.c_int()
        check(lib().dpd_get_species(self._ctx, ctypes.byref(S), None, None, None))
        if S.value == 1:
            return 1, None, None, None
        t = [np.zeros((S.value, S.value)) for _ in range(3)]
        ptr = [x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in t]
        check(lib().dpd_get_species(self._ctx, ctypes.byref(S), *ptr))
        return (S.value, *t)

    def step(self, nsteps: int = 1):
        check(lib().dpd_step(self._ctx, int(nsteps)))

    def get_state(self, device: bool = False):
        """(positions, full-step velocities) in id order: NumPy, or CUDA tensors if device."""
        if device:
            import torch
            pos = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
            vel = torch.empty_like(pos)
            check(lib().dpd_get_state(self._ctx, ctypes.c_void_p(pos.data_ptr()),
                                      ctypes.c_void_p(vel.data_ptr()), WHERE_DEVICE))
            return pos, vel
        pos = np.empty((self.n, 3), dtype=np.float32)
        vel = np.empty_like(pos)
        check(lib().dpd_get_state(self._ctx, pos.ctypes.data_as(ctypes.c_void_p),
                                  vel.ctypes.data_as(ctypes.c_void_p), WHERE_HOST))
        return pos, vel

    def get_state_into(self, pos, vel):
        """Fill caller-provided n x 3 buffers (pinned host tensors/arrays or CUDA tensors)."""
        pp, wp, _ = _vec3_arg(pos, self.n) if not _is_cuda_tensor(pos) else (
            ctypes.c_void_p(pos.data_ptr()), WHERE_DEVICE, pos)
        vv, _, _ = _vec3_arg(vel, self.n) if not _is_cuda_tensor(vel) else (
            ctypes.c_void_p(vel.data_ptr()), WHERE_DEVICE, vel)
        check(lib().dpd_get_state(self._ctx, pp, vv, wp))

    def get_forces(self, device: bool = False):
        if device:
            import torch
            f = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
            check(lib().dpd_get_forces(self._ctx, ctypes.c_void_p(f.data_ptr()), WHERE_DEVICE))
            return f
        f = np.empty((self.n, 3), dtype=np.float32)
        check(lib().dpd_get_forces(self._ctx, f.ctypes.data_as(ctypes.c_void_p), WHERE_HOST))
        return f

    def profile(self, nsteps: int) -> list:
        """Mean device ms per stage over nsteps steps: [integrate+count, scan,
        key pass, reorder, force]."""
        ms = (ctypes.c_double * NUM_STAGES)()
        check(lib().dpd_profile_steps(self._ctx, int(nsteps), ms))
        return list(ms)

    def checkpoint(self) -> bytes:
        """Internal state (cell order, step counter) as bytes."""
        n = lib().dpd_checkpoint_size(self._ctx)
        buf = ctypes.create_string_buffer(n)
        check(lib().dpd_checkpoint_save(self._ctx, buf, n))
        return buf.raw

    def restore(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        check(lib().dpd_checkpoint_load(self._ctx, buf, len(data)))
        self.n = self._n_from_header(data)

    @staticmethod
    def _n_from_header(data: bytes) -> int:
        return int(np.frombuffer(data[8:16], dtype=np.int64)[0])

    def stats(self) -> dict:
        s = Stats()
        check(lib().dpd_get_stats(self._ctx, ctypes.byref(s)))
        return s.as_dict()


def debug_rng(lo, hi, step: int, seed: int, stream=None, noise: int = NOISE_UNIFORM,
              word1: bool = False):
    """Noise words (uint32) and FP32 xi for pairs (lo[k], hi[k]) computed on the GPU;
    with word1=True also Philox word 1."""
    import torch
    lo = np.ascontiguousarray(lo, dtype=np.uint32)
    hi = np.ascontiguousarray(hi, dtype=np.uint32)
    n = lo.size
    d_lo = torch.from_numpy(lo.view(np.int32)).cuda()
    d_hi = torch.from_numpy(hi.view(np.int32)).cuda()
    d_out = torch.empty(n, dtype=torch.int32, device="cuda")
    d_out1 = torch.empty(n, dtype=torch.int32, device="cuda")
    d_xi = torch.empty(n, dtype=torch.float32, device="cuda")
    check(lib().dpd_debug_rng(ctypes.c_void_p(d_lo.data_ptr()), ctypes.c_void_p(d_hi.data_ptr()),
                              n, int(step), int(seed), int(noise),
                              ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(d_out1.data_ptr()),
                              ctypes.c_void_p(d_xi.data_ptr()), _stream_ptr(stream)))
    w0 = d_out.cpu().numpy().view(np.uint32)
    if word1:
        return w0, d_out1.cpu().numpy().view(np.uint32), d_xi.cpu().numpy()
    return w0, d_xi.cpu().numpy()


NOALLOC_MAX_PARTICLES = 32768
NOALLOC_MAX_CELLS = 32767


def forces_noalloc(pos, vel, L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=0, step=0,
                   out=None, stream=None):
    """Pair forces from a caller-held CUDA state through dpd_forces_noalloc,
    which allocates no device memory (its scratch is a static device array).

    pos, vel: n x 3 CUDA tensors on one device (copied to contiguous float32
    if they are not); ``out``, if given, must be a contiguous float32 n x 3
    tensor on the same device.  The work is enqueued on ``stream`` (default:
    torch's current stream of that device) without synchronising; the call
    runs with that device current, whose scratch array it uses."""
    import torch
    if not (_is_cuda_tensor(pos) and _is_cuda_tensor(vel)):
        raise ValueError("pos and vel must be CUDA tensors")
    dev = pos.device
    if vel.device != dev:
        raise ValueError("pos and vel must be on the same device")
    n = int(pos.shape[0])
    if out is not None:
        if not (_is_cuda_tensor(out) and out.device == dev and out.dtype == torch.float32
                and out.is_contiguous() and tuple(out.shape) == (n, 3)):
            raise ValueError("out must be a contiguous float32 (n, 3) tensor on pos.device")
    with torch.cuda.device(dev):
        pp, _, kp = _vec3_arg(pos, n)
        vv, _, kv = _vec3_arg(vel, n)
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        box = (ctypes.c_double * 3)(*L3)
        check(lib().dpd_forces_noalloc(n, pp, vv, box, a, gamma, kT, rc, dt, int(seed),
                                       int(step), ctypes.c_void_p(out.data_ptr()),
                                       _stream_ptr(st)))
        if isinstance(st, torch.cuda.Stream):
            # converted copies stay allocated until the enqueued work has read them
            for t in (kp, kv):
                if t is not pos and t is not vel:
                    t.record_stream(st)
    return out
