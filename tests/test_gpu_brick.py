"""The brick force kernel (half stencil staged through shared memory) against
the FP64 oracle: box shapes whose staged regions wrap on every axis, boxes
wide enough for several chunks per block, the Poiseuille body force, a
dense region that makes the kernel narrow its chunks and split bricks into
single rows, and the capacity error when even one row's stencil does not
fit.  Tolerances are the contract's (forces within 1e-5 of the force RMS)."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
BRICK = 13


@pytest.fixture(scope="module")
def dpd():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.dpd as d
    return d


def _params(L, seed, **kw):
    L3 = tuple(np.broadcast_to(np.asarray(L, float), (3,)))
    base = dict(a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005)
    base.update(kw)
    return O.Params(L=L3, seed=seed, **base)


def _brick_box(dpd, p, variant=BRICK):
    box = dpd.Box(p.L, a=p.a, gamma=p.gamma, kT=p.kT, rc=p.rc, dt=p.dt, seed=p.seed, stencil=1)
    box.set_param(dpd.PARAM_FORCE_VARIANT, variant)
    if p.fb_mode:
        box.set_param(dpd.PARAM_FLOW_AXIS, p.fb_flow)
        box.set_param(dpd.PARAM_GRAD_AXIS, p.fb_grad)
        box.set_param(dpd.PARAM_POISEUILLE_F, p.fb)
    return box


def _check(f_gpu, f_ref):
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    err = np.abs(f_gpu.astype(np.float64) - f_ref).max()
    assert err <= FORCE_TOL * rms, f"max force error {err:.3e} > {FORCE_TOL} x rms {rms:.3f}"


@pytest.mark.parametrize("L,rho,kw", [
    ((3.0, 3.0, 3.0), 5, {}),                        # smallest grid: every staged row wraps
    ((6.0, 7.3, 3.2), 10, {}),                       # non-integer edges, dense
    ((24.0, 13.5, 10.0), 3, {}),                     # several chunks per block
    ((33.0, 9.0, 17.0), 4, dict(fb=0.2, fb_mode=O.FB_POISEUILLE, fb_flow=0, fb_grad=1)),
    ((16.0, 16.0, 16.0), 3, dict(rc=1.3)),           # cells wider than 1
])
def test_brick_forces_match_oracle(dpd, L, rho, kw):
    x, v = uniform_box_state(L, rho=rho, seed=21)
    p = _params(L, 21, **kw)
    mode = O.MODE_CELLS if len(x) > 6000 else O.MODE_BRUTE
    f_ref, vir = O.forces(p, x, v, 0, mode=mode)
    box = _brick_box(dpd, p)
    box.set_state(x, v)
    _check(box.get_forces(), f_ref)
    assert box.stats()["virial"] == pytest.approx(vir, rel=1e-5)
    # five steps: the same trajectory as the per-lane kernel
    box.step(5)
    xb, _ = box.get_state()
    ref = _brick_box(dpd, p, variant=0)
    ref.set_state(x, v)
    ref.step(5)
    xr, _ = ref.get_state()
    d = xb.astype(np.float64) - xr
    d -= np.asarray(p.L) * np.round(d / np.asarray(p.L))
    assert np.abs(d).max() < 1e-4
    box.close()
    ref.close()


def _clustered(L, rho, region, rho_region, seed):
    """A box of density rho with one cube of edge `region` at rho_region."""
    rng = np.random.default_rng(seed)
    n_out = int(rho * (L ** 3 - region ** 3))
    n_in = int(rho_region * region ** 3)
    xs = rng.uniform(0, L, size=(3 * n_out, 3))
    keep = ~np.all((xs >= 2.0) & (xs < 2.0 + region), axis=1)
    x = np.concatenate([xs[keep][:n_out], 2.0 + rng.uniform(0, region, size=(n_in, 3))])
    v = rng.normal(0, 1, size=x.shape)
    v -= v.mean(0)
    return x.astype(np.float32), v.astype(np.float32)


def test_dense_region_narrows_chunks_and_splits_rows(dpd):
    # density 24 in a 5^3 cube: a 4 x 4-row brick's single slice stages
    # about 30 rows x 5 slices x 12 = 1800 particles, more than the capacity,
    # so the kernel falls back to single rows there
    L = 16.0
    x, v = _clustered(L, 3.0, 5.0, 24.0, seed=2)
    p = _params(L, 4)
    f_ref, vir = O.forces(p, x, v, 0, mode=O.MODE_CELLS)
    box = _brick_box(dpd, p)
    box.set_state(x, v)
    _check(box.get_forces(), f_ref)
    assert box.stats()["virial"] == pytest.approx(vir, rel=1e-5)
    box.close()


def test_capacity_error_is_reported(dpd):
    # density 200 in a 3^3 cube: one row's stencil holds more than the
    # staging capacity; the call reports it instead of returning wrong forces
    L = 12.0
    x, v = _clustered(L, 3.0, 3.0, 200.0, seed=3)
    box = _brick_box(dpd, _params(L, 5))
    with pytest.raises(dpd.DPDError) as ei:
        box.set_state(x, v)
        box.get_forces()
    assert ei.value.code == dpd.ERR_NUMERIC and "capacity" in str(ei.value)
    box.close()
