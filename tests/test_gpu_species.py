"""Several species per box on the GPU against the FP64 oracle (the particle
vectors of Sec. 3.1 with per-pair interactions and cut-offs): forces from an
identical state, a 100-step trajectory, momentum, checkpoints and errors."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
A = np.array([[25.0, 40.0, 31.0], [40.0, 18.0, 55.0], [31.0, 55.0, 12.0]])
G = np.array([[4.5, 2.0, 6.0], [2.0, 3.5, 1.5], [6.0, 1.5, 8.0]])
RC = np.array([[1.0, 0.8, 0.9], [0.8, 0.7, 0.95], [0.9, 0.95, 0.85]])


@pytest.fixture(scope="module")
def dpd():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.dpd as d
    return d


def _setup(dpd, L, rho, seed, stencil, S=3):
    x, v = uniform_box_state(L, rho=rho, seed=seed)
    sp = np.random.default_rng(seed).integers(0, S, len(x)).astype(np.int32)
    L3 = tuple(np.broadcast_to(np.asarray(L, float), (3,)))
    p = O.Params(L=L3, kT=1.0, dt=0.005, seed=seed)
    p.set_species(sp, A[:S, :S], G[:S, :S], RC[:S, :S])
    box = dpd.Box(L3, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=seed, stencil=stencil)
    box.set_species(A[:S, :S], G[:S, :S], RC[:S, :S])
    return x, v, sp, p, box


def _min_image(d, L):
    L = np.asarray(L, float)
    return d - L * np.round(d / L)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("L,rho,S", [((5.0, 6.5, 7.25), 4, 3), (8.0, 3, 2), (4.0, 10, 3)])
def test_mixture_forces_match_oracle(dpd, stencil, L, rho, S):
    x, v, sp, p, box = _setup(dpd, L, rho, 31, stencil, S)
    box.set_state(x, v, species=sp)
    f_ref, vir = O.forces(p, x, v, 0, mode=O.MODE_CELLS)
    fg = box.get_forces().astype(np.float64)
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    assert np.abs(fg - f_ref).max() <= FORCE_TOL * rms
    assert box.stats()["virial"] == pytest.approx(vir, rel=1e-5)
    assert box.get_species()[0] == S


@pytest.mark.parametrize("stencil", [0, 1])
def test_mixture_trajectory_and_momentum(dpd, stencil):
    L = 8.0
    x, v, sp, p, box = _setup(dpd, L, 3, 12, stencil)
    box.set_state(x, v, species=sp)
    ref = O.State(p, x, v, mode=O.MODE_CELLS)
    box.step(100)
    ref.run(100)
    xg, vg = box.get_state()
    assert np.abs(_min_image(xg.astype(np.float64) - ref.x, L)).max() < 1e-3
    P = vg.astype(np.float64).sum(0)
    assert np.abs(P - v.astype(np.float64).sum(0)).max() <= 1e-6 * np.abs(vg).sum()


def test_equal_tables_match_one_species(dpd):
    L = 7.0
    x, v = uniform_box_state(L, rho=3, seed=5)
    one = dpd.Box(L, a=30.0, gamma=4.0, kT=1.0, rc=1.0, dt=0.005, seed=5)
    one.set_state(x, v)
    mix = dpd.Box(L, a=30.0, gamma=4.0, kT=1.0, rc=1.0, dt=0.005, seed=5)
    mix.set_species(np.full((3, 3), 30.0), np.full((3, 3), 4.0), np.ones((3, 3)))
    mix.set_state(x, v, species=np.arange(len(x)) % 3)
    f1, f3 = one.get_forces().astype(np.float64), mix.get_forces().astype(np.float64)
    rms = math.sqrt((f1 ** 2).sum(1).mean())
    assert np.abs(f1 - f3).max() <= 1e-6 * rms


def test_species_from_device_memory_and_checkpoint(dpd):
    import torch
    L = 6.0
    x, v, sp, p, box = _setup(dpd, L, 3, 8, 0)
    box.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(),
                  species=torch.from_numpy(sp).cuda())
    host = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=8)
    host.set_species(A, G, RC)
    host.set_state(x, v, species=sp)
    assert np.array_equal(box.get_forces(), host.get_forces())
    box.step(30)
    ck = box.checkpoint()
    box.step(20)
    again = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=8)
    again.set_species(A, G, RC)
    again.restore(ck)
    again.step(20)
    assert np.array_equal(box.get_state()[0], again.get_state()[0])
    plain = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=8)
    with pytest.raises(dpd.DPDError) as ei:           # one species: other parameters
        plain.restore(ck)
    assert ei.value.code == dpd.ERR_STATE
    bad = torch.full((len(x),), 3, dtype=torch.int32, device="cuda")
    with pytest.raises(dpd.DPDError) as ei:
        box.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), species=bad)
    assert ei.value.code == dpd.ERR_ARG


def test_species_argument_errors(dpd):
    """Species tables and labels are validated on the host."""
    box = dpd.Box(6.0, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=0)
    A = np.array([[25.0, 40.0], [40.0, 18.0]])
    G = np.array([[4.5, 2.0], [2.0, 3.5]])
    R = np.array([[1.0, 0.8], [0.8, 0.7]])
    box.set_species(A, G, R)
    S, a, g, r = box.get_species()
    assert S == 2 and np.array_equal(a, A) and np.array_equal(r, R)
    for bad in ((A + np.triu(np.ones((2, 2)), 1), G, R),     # not symmetric
                (A, G, np.array([[1.0, 1.2], [1.2, 0.7]])),  # cut-off above rc
                (A, -G, R),                                   # gamma < 0
                (np.ones((5, 5)), np.ones((5, 5)), np.ones((5, 5)))):   # too many species
        with pytest.raises(dpd.DPDError) as ei:
            box.set_species(*bad)
        assert ei.value.code == dpd.ERR_ARG
    with pytest.raises(dpd.DPDError) as ei:
        box.set_state(np.zeros((4, 3), np.float32), np.zeros((4, 3), np.float32),
                      species=np.array([0, 1, 2, 0]))
    assert ei.value.code == dpd.ERR_ARG
    with pytest.raises(dpd.DPDError) as ei:
        box.set_param(dpd.PARAM_FORCE_TILES, 1)
    assert ei.value.code == dpd.ERR_ARG
    box.set_species()
    assert box.get_species()[0] == 1
