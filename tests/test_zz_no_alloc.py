"""dpd_forces_noalloc against the allocating entry points.

The allocation-free call serves callers that cannot allocate device memory
where they need forces (inside a host callback or a custom allocator, under a
framework that owns all device memory, in a loop that must not meet
cudaMalloc's implicit synchronisation).  Its scratch is a static device
array shared by every call, so this test makes two calls in a row on
different states and checks each against dpd_set_state + dpd_get_forces.
The file is named to be collected last.
"""

import math

import numpy as np
import pytest

from paper_1911_04712_gb300.workloads import uniform_box_state

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


@pytest.fixture(scope="module")
def dpd():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.dpd as d
    return d


def _reference_forces(dpd, L, x, v, seed, a, gamma, kT):
    box = dpd.Box(L, a=a, gamma=gamma, kT=kT, rc=1.0, dt=0.005, seed=seed)
    box.set_state(x, v)
    f = box.get_forces()
    box.close()
    return f.astype(np.float64)


def test_noalloc_forces_match_allocating_path_two_calls(dpd):
    import torch
    cases = [((8.0, 8.0, 8.0), 3, 0, 25.0, 4.5, 1.0),
             ((5.0, 6.5, 7.25), 5, 7, 40.0, 2.0, 0.7)]
    states = []
    for L, rho, seed, a, gamma, kT in cases:
        x, v = uniform_box_state(L, rho=rho, seed=seed)
        states.append((L, x, v, seed, a, gamma, kT))
    outs = []
    for L, x, v, seed, a, gamma, kT in states:          # two calls in a row, one scratch
        f = dpd.forces_noalloc(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), L,
                               a=a, gamma=gamma, kT=kT, seed=seed, step=0)
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy().astype(np.float64))
    for (L, x, v, seed, a, gamma, kT), got in zip(states, outs):
        want = _reference_forces(dpd, L, x, v, seed, a, gamma, kT)
        rms = math.sqrt((want ** 2).sum(1).mean())
        assert np.abs(got - want).max() <= FORCE_TOL * rms


def test_noalloc_repeated_call_is_unchanged_and_rejects_large_inputs(dpd):
    import torch
    import oracle as O
    x, v = uniform_box_state(6.0, rho=3, seed=3)
    xd, vd = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
    f1 = dpd.forces_noalloc(xd, vd, 6.0, seed=3, step=5).cpu().numpy()
    f2 = dpd.forces_noalloc(xd, vd, 6.0, seed=3, step=5).cpu().numpy()
    assert np.array_equal(f1, f2)
    # the step reaches the pair noise: the FP64 oracle's forces at step 5
    p = O.Params(L=(6.0, 6.0, 6.0), a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=3)
    want, _ = O.forces(p, x, v, 5)
    rms = math.sqrt((want ** 2).sum(1).mean())
    assert np.abs(f1.astype(np.float64) - want).max() <= FORCE_TOL * rms
    with pytest.raises(ValueError):                 # an output of the wrong dtype
        dpd.forces_noalloc(xd, vd, 6.0, out=torch.empty_like(xd, dtype=torch.float16))
    big = torch.zeros((dpd.NOALLOC_MAX_PARTICLES + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(dpd.DPDError) as ei:
        dpd.forces_noalloc(big, big, 40.0)
    assert ei.value.code == dpd.ERR_ARG and "at most" in str(ei.value)
    with pytest.raises(dpd.DPDError):
        dpd.forces_noalloc(xd, vd, 40.0)          # 64000 cells > the cell limit
