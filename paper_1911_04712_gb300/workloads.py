"""Seeded synthetic inputs for the DPD fluid step.

This module draws the initial particle states, the multi-box mixes and the
request streams that both the CUDA path and the FP64 oracle consume.  It holds
none of the method's arithmetic (no forces, no random pair noise, no
integration): only the sampling of starting conditions, so that both sides
read the very same FP32 arrays.

Recipes (the paper's periodic-Poiseuille benchmark, Sec. 5.1, is itself a
uniformly filled periodic cube, so nothing here stands in for a dataset):

* single box: positions i.i.d. uniform in [0, L)^3, velocities i.i.d.
  N(0, kT/m) per component with the mean momentum removed, rounded to FP32;
* box mix: per box an integer edge, a density and Groot-Warren parameters
  drawn from one master-seeded generator;
* request stream: Poisson arrivals with per-request box, density, parameters
  and step count.
"""

from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass, field

import numpy as np

__all__ = [
    "uniform_box_state",
    "BoxSpec",
    "box_mix",
    "RequestSpec",
    "request_stream",
    "particles_for",
]


def particles_for(L, rho: float) -> int:
    """Number of particles filling a box of edges ``L`` at number density ``rho``."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    return int(round(rho * float(L[0] * L[1] * L[2])))


def uniform_box_state(L, rho: float | None = None, n: int | None = None,
                      kT: float = 1.0, mass: float = 1.0, seed: int = 0):
    """Uniform positions and Maxwellian velocities, FP32, shape (n, 3).

    ``L`` is a scalar or three edges.  Exactly one of ``rho`` and ``n`` sets
    the particle count.  Positions that round up to the box edge in FP32 are
    folded to 0 so every coordinate lies in [0, L).
    """
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    if n is None:
        if rho is None:
            raise ValueError("give rho or n")
        n = particles_for(L, rho)
    rng = np.random.default_rng(np.random.SeedSequence([0xD9D, int(seed)]))
    pos = (rng.random((n, 3)) * L).astype(np.float32)
    L32 = L.astype(np.float32)
    pos = np.where(pos >= L32, np.float32(0.0), pos).astype(np.float32)
    vel = rng.normal(0.0, math.sqrt(kT / mass), (n, 3))
    if n > 0:
        vel -= vel.mean(axis=0)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel.astype(np.float32))


@dataclass
class BoxSpec:
    """One independent periodic box of a multi-box mix."""
    L: float
    rho: float
    a: float
    gamma: float
    kT: float
    dt: float
    seed: int
    steps: int
    n: int = 0
    rc: float = 1.0

    def __post_init__(self):
        if self.n == 0:
            self.n = particles_for(self.L, self.rho)


def box_mix(nbox: int = 512, master_seed: int = 0, L_range=(6, 24), rhos=(3, 4, 5),
            a_range=(10.0, 80.0), gamma_range=(2.0, 8.0), kT_range=(0.5, 2.0),
            dt: float = 0.005, steps: int = 500) -> list[BoxSpec]:
    """Mix of uneven boxes: integer edge U{L_range}, density from ``rhos``,
    a, gamma, kT uniform in their ranges, seeds 0..nbox-1."""
    rng = np.random.default_rng(np.random.SeedSequence([0xB0C5, int(master_seed)]))
    out = []
    for b in range(nbox):
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        rho = float(rng.choice(rhos))
        a = float(rng.uniform(*a_range))
        g = float(rng.uniform(*gamma_range))
        kT = float(rng.uniform(*kT_range))
        out.append(BoxSpec(L=float(L), rho=rho, a=a, gamma=g, kT=kT, dt=dt, seed=b, steps=steps))
    return out


def box_mix_manifest(specs: list[BoxSpec]) -> str:
    """JSON manifest of a box mix, so that a run can be replayed exactly."""
    return json.dumps([asdict(s) for s in specs])


@dataclass
class RequestSpec:
    """One served DPD run: a periodic box simulated for ``steps`` steps."""
    t_arrival: float
    L: float
    rho: float
    a: float
    gamma: float
    kT: float
    steps: int
    seed: int
    dt: float = 0.005
    pois_f: float = 0.0
    n: int = 0

    def __post_init__(self):
        if self.n == 0:
            self.n = particles_for(self.L, self.rho)


def request_stream(nreq: int = 10_000, rate: float = 200.0, master_seed: int = 0,
                   L_median: float = 16.0, L_sigma: float = 0.5, L_clip=(8.0, 48.0),
                   rhos=(3, 5), a_range=(10.0, 80.0), gamma_range=(2.0, 8.0),
                   kT_range=(0.5, 2.0), steps_range=(1000, 20000),
                   pois_f: float = 0.0) -> list[RequestSpec]:
    """Poisson arrivals at ``rate`` per second; log-normal box edge (non-integer
    edges allowed) clipped to ``L_clip``; step counts uniform in ``steps_range``."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5E4E, int(master_seed)]))
    t = 0.0
    out = []
    for k in range(nreq):
        t += float(rng.exponential(1.0 / rate))
        L = float(np.clip(rng.lognormal(math.log(L_median), L_sigma), *L_clip))
        out.append(RequestSpec(
            t_arrival=t, L=L, rho=float(rng.choice(rhos)),
            a=float(rng.uniform(*a_range)), gamma=float(rng.uniform(*gamma_range)),
            kT=float(rng.uniform(*kT_range)),
            steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
            seed=k, pois_f=pois_f))
    return out
