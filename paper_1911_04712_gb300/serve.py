"""Binding of the served form (dpd_queue_*): argument marshalling only."""

from __future__ import annotations

import ctypes

import numpy as np

POLICY_FIFO, POLICY_SJF = 0, 1


class QueueOpts(ctypes.Structure):
    _fields_ = [("max_boxes", ctypes.c_int64), ("chunk_steps", ctypes.c_int64),
                ("sample_every", ctypes.c_int64), ("nbins", ctypes.c_int),
                ("policy", ctypes.c_int), ("stencil", ctypes.c_int), ("pad_", ctypes.c_int),
                ("chunk_timeout_s", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("rho", ctypes.c_double), ("n", ctypes.c_int64),
                ("a", ctypes.c_double), ("gamma", ctypes.c_double), ("kT", ctypes.c_double),
                ("rc", ctypes.c_double), ("dt", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("steps", ctypes.c_int64), ("body_force", ctypes.c_double),
                ("body_mode", ctypes.c_int), ("flow_axis", ctypes.c_int),
                ("grad_axis", ctypes.c_int), ("noise", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nbins", ctypes.c_int), ("n", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("kT_mean", ctypes.c_double), ("pressure_mean", ctypes.c_double),
                ("profile", ctypes.c_double * 64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"status": self.status, "n": self.n, "steps": self.steps, "samples": self.samples,
                "kT_mean": self.kT_mean, "pressure_mean": self.pressure_mean,
                "profile": np.array(self.profile[:self.nbins]), "t_submit": self.t_submit,
                "t_admit": self.t_admit, "t_done": self.t_done,
                "latency": self.t_done - self.t_submit}


class QueueStats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_uint64), ("particle_steps", ctypes.c_double),
                ("busy_seconds", ctypes.c_double), ("clock_seconds", ctypes.c_double)]


def _declare(L):
    c = ctypes
    vp = c.c_void_p
    L.dpd_queue_create.argtypes = [c.POINTER(vp), c.c_size_t, c.POINTER(QueueOpts)]
    L.dpd_queue_destroy.argtypes = [vp]
    L.dpd_queue_submit.argtypes = [vp, c.POINTER(Request), c.POINTER(c.c_uint64)]
    L.dpd_queue_submit_state.argtypes = [vp, c.POINTER(Request), vp, vp, c.c_int,
                                         c.POINTER(c.c_uint64)]
    L.dpd_queue_final_state.argtypes = [vp, c.c_uint64, vp, vp]
    L.dpd_queue_poll.argtypes = [vp, c.c_uint64, c.POINTER(c.c_int)]
    L.dpd_queue_result.argtypes = [vp, c.c_uint64, c.POINTER(Result)]
    L.dpd_queue_cancel.argtypes = [vp, c.c_uint64]
    L.dpd_queue_wait_all.argtypes = [vp, c.c_double]
    L.dpd_queue_get_stats.argtypes = [vp, c.POINTER(QueueStats)]
    for name in ("dpd_queue_create", "dpd_queue_destroy", "dpd_queue_submit", "dpd_queue_poll",
                 "dpd_queue_result", "dpd_queue_cancel", "dpd_queue_wait_all",
                 "dpd_queue_get_stats", "dpd_queue_submit_state", "dpd_queue_final_state"):
        getattr(L, name).restype = c.c_int
    return L


_declared = False


def _lib():
    global _declared
    from . import dpd
    L = dpd.lib()
    if not _declared:
        _declare(L)
        _declared = True
    return L


def _check(rc):
    from . import dpd
    return dpd.check(rc)


def make_request(L, rho=0.0, n=0, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=0,
                 steps=1000, body_force=0.0, body_mode=0, flow_axis=2, grad_axis=0,
                 noise=0) -> Request:
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    return Request((ctypes.c_double * 3)(*L3), rho, int(n), a, gamma, kT, rc, dt, int(seed),
                   int(steps), body_force, body_mode, flow_axis, grad_axis, noise)


class Queue:
    """Continuous-batching queue of DPD runs on the current CUDA device."""

    def __init__(self, hbm_budget_bytes: int, max_boxes=0, chunk_steps=0, sample_every=0,
                 nbins=0, policy=POLICY_FIFO, stencil=0, chunk_timeout_s=0.0):
        opts = QueueOpts(max_boxes, chunk_steps, sample_every, nbins, policy, stencil, 0,
                         chunk_timeout_s)
        self._q = ctypes.c_void_p()
        _check(_lib().dpd_queue_create(ctypes.byref(self._q), int(hbm_budget_bytes),
                                       ctypes.byref(opts)))

    def close(self):
        if getattr(self, "_q", None) and self._q.value:
            _lib().dpd_queue_destroy(self._q)
            self._q = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, req: Request) -> int:
        t = ctypes.c_uint64()
        _check(_lib().dpd_queue_submit(self._q, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def submit_state(self, req: Request, pos, vel, keep_final: bool = False) -> int:
        """Submit with the caller's initial state (n x 3 float32 host arrays,
        req.n = n); keep_final keeps the final state for final_state()."""
        x = np.ascontiguousarray(pos, dtype=np.float32)
        v = np.ascontiguousarray(vel, dtype=np.float32)
        if x.shape != (req.n, 3) or v.shape != (req.n, 3):
            raise ValueError("pos and vel must be n x 3 with n = req.n")
        t = ctypes.c_uint64()
        _check(_lib().dpd_queue_submit_state(self._q, ctypes.byref(req),
                                             x.ctypes.data_as(ctypes.c_void_p),
                                             v.ctypes.data_as(ctypes.c_void_p),
                                             int(bool(keep_final)), ctypes.byref(t)))
        return t.value

    def final_state(self, ticket: int, n: int):
        """(positions, velocities) of a finished run kept with keep_final."""
        x = np.empty((n, 3), dtype=np.float32)
        v = np.empty((n, 3), dtype=np.float32)
        _check(_lib().dpd_queue_final_state(self._q, ticket, x.ctypes.data_as(ctypes.c_void_p),
                                            v.ctypes.data_as(ctypes.c_void_p)))
        return x, v

    def done(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(_lib().dpd_queue_poll(self._q, ticket, ctypes.byref(d)))
        return bool(d.value)

    def result(self, ticket: int) -> dict:
        r = Result()
        _check(_lib().dpd_queue_result(self._q, ticket, ctypes.byref(r)))
        return r.as_dict()

    def cancel(self, ticket: int):
        _check(_lib().dpd_queue_cancel(self._q, ticket))

    def wait_all(self, timeout_s: float = 600.0):
        _check(_lib().dpd_queue_wait_all(self._q, timeout_s))

    def stats(self) -> dict:
        s = QueueStats()
        _check(_lib().dpd_queue_get_stats(self._q, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in QueueStats._fields_}
