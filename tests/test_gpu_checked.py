"""The checked build (libdpd_checked.so, -DDPD_CHECKED=1): every kernel tests
the indices it derives from device data -- cell indices, cell starts and
segment ends, pair-list entries and fill, scatter targets -- and a failed
test is reported as DPD_ERR_INTERNAL instead of touching memory out of
bounds.  With no memory checker available for the GPU, this build run over
the small and degenerate cases of every form (one box with either stencil
and every force-kernel variant, Gaussian noise, several species, staged
tiles, a packed set with bands of different variants, the served queue, the
allocation-free call) shows that no index leaves its array, and that the
results still match the oracle.

The checked library is exercised in a child process (one library per
process in the binding)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch
import oracle as O
import paper_1911_04712_gb300.dpd as dpd
import paper_1911_04712_gb300.batch as B
import paper_1911_04712_gb300.serve as S
from paper_1911_04712_gb300.workloads import box_mix, uniform_box_state

worst = 0.0
cases = 0

def check_forces(fg, fr):
    global worst, cases
    rms = math.sqrt((fr ** 2).sum(1).mean()) if len(fr) > 1 else 1.0
    worst = max(worst, float(np.abs(fg.astype(np.float64) - fr).max() / max(rms, 1e-30)))
    cases += 1

boxes = [((5.0, 6.5, 7.25), 3, None), (3.0, 5, None), ((3.0, 11.0, 4.0), 4, None),
         (6.0, 3, 2), (4.0, 3, 4000), (8.0, 10, None)]
ref = {}
for stencil in (0, 1):
    for variant in range(-1, B.NUM_FORCE_VARIANTS):
        for k, (L, rho, n) in enumerate(boxes):
            x, v = uniform_box_state(L, rho=rho, n=n, seed=7)
            L3 = tuple(np.broadcast_to(np.asarray(L, float), (3,)))
            if k not in ref:
                p = O.Params(L=L3, a=25.0, gamma=4.5, kT=1.0, dt=0.005, seed=3)
                ref[k] = O.forces(p, x, v, 0)[0]
            box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=3, stencil=stencil)
            box.set_param(dpd.PARAM_FORCE_VARIANT, variant)
            box.set_state(x, v)
            check_forces(box.get_forces(), ref[k])
            box.step(6)
            box.get_state()
            box.stats()
            box.close()

# Gaussian noise, several species (general kernels), staged tiles
L = (5.0, 6.5, 7.25)
x, v = uniform_box_state(L, rho=5, seed=8)
sp = np.random.default_rng(8).integers(0, 3, len(x)).astype(np.int32)
A = np.array([[25, 40, 30], [40, 25, 35], [30, 35, 20]], float)
G = np.array([[4.5, 3.0, 5.0], [3.0, 4.5, 2.0], [5.0, 2.0, 6.0]])
R = np.array([[1.0, 0.8, 0.9], [0.8, 1.0, 0.7], [0.9, 0.7, 0.95]])
for stencil in (0, 1):
    p = O.Params(L=L, a=25.0, gamma=4.5, kT=1.0, dt=0.005, seed=5, noise=1)
    p.set_species(sp, A, G, R)
    box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=5, stencil=stencil)
    box.set_param(dpd.PARAM_NOISE, 1)
    box.set_species(A, G, R)
    box.set_state(x, v, species=sp)
    fr, _ = O.forces(p, x, v, 0)
    check_forces(box.get_forces(), fr)
    box.step(6)
    box.get_state()
    box.close()
for tiling in (dict(tiles=1), dict(tiles=1, tile_cells=1), dict(tiles=1, stage_cap=64)):
    for L, rho in (((5.0, 6.5, 7.25), 3), (3.0, 5), (4.0, 10)):
        x, v = uniform_box_state(L, rho=rho, seed=9)
        L3 = tuple(np.broadcast_to(np.asarray(L, float), (3,)))
        p = O.Params(L=L3, a=25.0, gamma=4.5, kT=1.0, dt=0.005, seed=4)
        box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=4, **tiling)
        box.set_state(x, v)
        fr, _ = O.forces(p, x, v, 0)
        check_forces(box.get_forces(), fr)
        box.step(6)
        box.get_state()
        box.close()

# a packed set: a mix of small boxes, bands of different variants, both stencils
specs = box_mix(24, master_seed=6, L_range=(3, 9))
states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=200 + k) for k, s in enumerate(specs)]
descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
         for s, st in zip(specs, states)]
for stencil in (0, 1):
    for variants in ((0, 4, 7, 10), (12, 2, 9, 5)):
        for t in (2 * stencil, 2 * stencil + 1):
            B.tuning_set(t, [3.5, 4.5, 5.5, 1e9], list(variants))
        bt = B.Batch(descs, stencil=stencil)
        for k, (x, v) in enumerate(states):
            bt.set_state(k, x, v)
        for k in (0, 7, 23):
            s, (x, v) = specs[k], states[k]
            p = O.Params(L=(s.L,) * 3, a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
            fr, _ = O.forces(p, x, v, 0)
            check_forces(bt.get_forces(k), fr)
        bt.step(6)
        bt.stats()
        bt.get_state(5)
        bt.close()

# the served queue, and the allocation-free call
q = S.Queue(int(2e9), max_boxes=3, chunk_steps=10, sample_every=5, nbins=4, stencil=1)
tickets = [q.submit(S.make_request(L=float(Lq), rho=3.0, seed=k, steps=30))
           for k, Lq in enumerate((3.0, 4.5, 6.0, 5.0, 3.5))]
q.wait_all(300.0)
status = [q.result(t)["status"] for t in tickets]
q.close()
x, v = uniform_box_state(6.0, rho=3, seed=2)
f = dpd.forces_noalloc(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), 6.0, seed=1)
torch.cuda.synchronize()
p = O.Params(L=(6.0,) * 3, a=25.0, gamma=4.5, kT=1.0, dt=0.005, seed=1)
fr, _ = O.forces(p, x, v, 0)
check_forces(f.cpu().numpy(), fr)
print(json.dumps({"version": dpd.version(), "cases": cases, "worst": worst, "queue": status}))
"""


def test_checked_build_keeps_every_index_in_bounds():
    from paper_1911_04712_gb300 import build
    build.build()
    path = build.build(checked=True)
    env = dict(os.environ, DPD_LIBRARY=path)
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert "checked" in res["version"]
    assert res["cases"] > 150
    assert res["worst"] <= 1e-5, res
    assert res["queue"] == [0] * 5, res
