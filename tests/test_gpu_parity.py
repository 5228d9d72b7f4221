"""GPU path against the FP64 oracle, through the C ABI.

Tolerances (fixed by the contract of the method's FP32 implementation):
* noise words bit-exact; FP32 xi within 1 ulp of the FP64 value;
* per-particle forces from an identical state within 1e-5 of the force RMS;
* 100-step trajectories within 1e-3 rc (minimum image, matched by id);
* total momentum within 1e-6 of the summed momentum magnitude sum_i m |v_i|.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
TRAJ_TOL = 1e-3


@pytest.fixture(scope="module")
def dpd():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.dpd as d
    return d


def _params(L, seed=0, **kw):
    L3 = tuple(np.broadcast_to(np.asarray(L, float), (3,)))
    base = dict(a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005)
    base.update(kw)
    return O.Params(L=L3, seed=seed, **base)


def _box(dpd, p: O.Params, stencil=0):
    box = dpd.Box(p.L, a=p.a, gamma=p.gamma, kT=p.kT, rc=p.rc, dt=p.dt, seed=p.seed,
                  stencil=stencil, kexp=p.kexp, mass=p.mass)
    if p.fb_mode:
        box.set_param(dpd.PARAM_FLOW_AXIS, p.fb_flow)
        box.set_param(dpd.PARAM_GRAD_AXIS, p.fb_grad)
        box.set_param(dpd.PARAM_BODYFORCE if p.fb_mode == O.FB_CONST else dpd.PARAM_POISEUILLE_F,
                      p.fb)
    return box


def _min_image(d, L):
    L = np.asarray(L, float)
    return d - L * np.round(d / L)


def _force_check(f_gpu, f_ref):
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    err = np.abs(f_gpu.astype(np.float64) - f_ref).max()
    assert err <= FORCE_TOL * rms, f"max force error {err:.3e} > {FORCE_TOL} x rms {rms:.3f}"
    return err / rms


# ---------------------------------------------------------------- noise
def test_rng_words_bit_exact(dpd):
    rng = np.random.default_rng(5)
    n = 1 << 16
    lo = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    lo[:4] = [0, 0xFFFFFFFF, 7, 7]
    hi[:4] = [0, 0xFFFFFFFF, 7, 3]
    for step, seed in ((0, 0), (123456789012, 0xDEADBEEFCAFEF00D), (1, 2)):
        words, xi = dpd.debug_rng(lo, hi, step, seed)
        ref_w, ref_xi = O.pair_rng(lo, hi, step, seed)
        assert np.array_equal(words, ref_w)
        ulp = np.spacing(np.abs(ref_xi).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(xi.astype(np.float64) - ref_xi) <= ulp)


# ---------------------------------------------------------------- forces
@pytest.mark.parametrize("stencil", [0, 1])
def test_forces_identical_state_L8(dpd, stencil):
    x, v = uniform_box_state(8, rho=3, seed=0)
    p = _params(8, seed=0)
    box = _box(dpd, p, stencil)
    box.set_state(x, v)
    f_ref, vir = O.forces(p, x, v, 0)
    _force_check(box.get_forces(), f_ref)
    st = box.stats()
    assert st["virial"] == pytest.approx(vir, rel=1e-5)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("L,rho,n", [
    ((5.0, 6.5, 7.25), 3, None),     # non-integer edges, ragged count
    (3.0, 5, None),                  # minimum box: 3 cells per axis
    ((3.0, 11.0, 4.0), 4, None),     # thin box
    (6.0, 3, 1),                     # one particle
    (6.0, 3, 2),                     # one pair
    (4.0, 3, 4000),                  # dense: ~62 per cell, lists drain often
])
def test_forces_ragged_and_edge_boxes(dpd, stencil, L, rho, n):
    x, v = uniform_box_state(L, rho=rho, n=n, seed=3)
    if n == 2:
        x[1] = x[0] + np.float32(0.5)
        x[1] = np.mod(x[1], np.float32(L))
    p = _params(L, seed=9)
    box = _box(dpd, p, stencil)
    box.set_state(x, v)
    f_ref, _ = O.forces(p, x, v, 0)
    if x.shape[0] >= 2:
        _force_check(box.get_forces(), f_ref)
    else:
        assert np.all(box.get_forces() == 0)


def test_particles_on_cell_and_box_faces(dpd):
    L = 6.0
    x, v = uniform_box_state(L, rho=3, seed=4)
    rng = np.random.default_rng(4)
    idx = rng.choice(len(x), 200, replace=False)
    faces = rng.integers(0, 6, (200, 3)).astype(np.float32)
    x[idx] = np.where(rng.random((200, 3)) < 0.5, faces, x[idx])
    x[idx[:20], 0] = np.float32(np.nextafter(np.float32(L), np.float32(0)))
    p = _params(L, seed=4)
    box = _box(dpd, p)
    box.set_state(x, v)
    f_ref, _ = O.forces(p, x, v, 0)
    _force_check(box.get_forces(), f_ref)


def test_positions_outside_box_are_wrapped(dpd):
    L = 5.0
    x, v = uniform_box_state(L, rho=3, seed=6)
    shifted = x + np.float32(L) * np.random.default_rng(6).integers(-2, 3, x.shape).astype(np.float32)
    p = _params(L, seed=6)
    box = _box(dpd, p)
    box.set_state(shifted, v)
    xg, _ = box.get_state()
    d = _min_image(xg.astype(np.float64) - x, L)
    assert np.abs(d).max() < 1e-5
    assert np.all(xg >= 0) and np.all(xg < L)


def test_body_forces_match_oracle(dpd):
    x, v = uniform_box_state(6, rho=3, seed=7)
    for mode, flow, grad in ((O.FB_CONST, 0, 1), (O.FB_POISEUILLE, 2, 0), (O.FB_POISEUILLE, 0, 1)):
        p = _params(6, seed=7, fb=0.5, fb_mode=mode, fb_flow=flow, fb_grad=grad)
        box = _box(dpd, p)
        box.set_state(x, v)
        f_ref, _ = O.forces(p, x, v, 0)
        _force_check(box.get_forces(), f_ref)


def test_weight_exponent_and_mass(dpd):
    x, v = uniform_box_state(6, rho=4, seed=8)
    p = _params(6, seed=8, kexp=0.5, mass=2.0)
    box = _box(dpd, p)
    box.set_state(x, v)
    f_ref, _ = O.forces(p, x, v, 0)
    _force_check(box.get_forces(), f_ref)
    box.step(30)
    s = O.State(p, x, v)
    s.run(30)
    xg, vg = box.get_state()
    assert np.abs(_min_image(xg - s.x, 6.0)).max() < TRAJ_TOL


# ---------------------------------------------------------- trajectories
@pytest.mark.parametrize("stencil", [0, 1])
def test_trajectory_100_steps_L8(dpd, stencil):
    L = 8.0
    x, v = uniform_box_state(L, rho=3, seed=0)
    p = _params(L, seed=0)
    box = _box(dpd, p, stencil)
    box.set_state(x, v)
    box.step(100)
    xg, vg = box.get_state()
    s = O.State(p, x, v)
    s.run(100)
    dx = np.abs(_min_image(xg.astype(np.float64) - s.x, L)).max()
    dv = np.abs(vg.astype(np.float64) - s.v).max()
    assert dx < TRAJ_TOL, dx
    assert dv < 0.05, dv
    # momentum: |P(t) - P(0)| within 1e-6 of sum_i m |v_i|
    P0 = v.astype(np.float64).sum(0)
    st = box.stats()
    scale = np.linalg.norm(vg.astype(np.float64), axis=1).sum()
    assert np.abs(st["momentum"] - P0).max() <= 1e-6 * scale
    assert st["step"] == 100
    ref = s.stats()
    assert st["kT"] == pytest.approx(ref["kT"], rel=1e-3)
    assert st["pressure"] == pytest.approx(ref["pressure"], rel=1e-3)


def test_constant_body_force_momentum(dpd):
    L, f0, nst = 6.0, 0.05, 64
    x, v = uniform_box_state(L, rho=3, seed=2)
    p = _params(L, seed=2, fb=f0, fb_mode=O.FB_CONST, fb_flow=0)
    box = _box(dpd, p)
    box.set_state(x, v)
    P0 = box.stats()["momentum"]
    box.step(nst)
    _, vg = box.get_state()
    P = box.stats()["momentum"]
    scale = np.linalg.norm(vg.astype(np.float64), axis=1).sum()
    want = np.array([len(x) * f0 * nst * p.dt, 0.0, 0.0])
    assert np.abs(P - P0 - want).max() <= 1e-6 * scale


def test_free_streaming(dpd):
    L = (5.0, 6.0, 7.0)
    x, v = uniform_box_state(L, rho=3, seed=3)
    p = _params(L, a=0.0, gamma=0.0, kT=0.0)
    box = _box(dpd, p)
    box.set_state(x, v)
    box.step(100)
    xg, vg = box.get_state()
    want = np.mod(x.astype(np.float64) + 100 * 0.005 * v.astype(np.float64), np.asarray(L))
    assert np.abs(_min_image(xg - want, L)).max() < 1e-4
    assert np.array_equal(vg, v)


def test_empty_box(dpd):
    box = _box(dpd, _params(5.0))
    box.set_state(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    box.step(10)
    xg, vg = box.get_state()
    assert xg.shape == (0, 3)
    assert box.stats()["step"] == 10


# ------------------------------------------------------- reproducibility
def test_full_stencil_is_bitwise_reproducible_and_graph_equals_direct(dpd):
    L = 8.0
    x, v = uniform_box_state(L, rho=3, seed=1)
    p = _params(L, seed=1)
    outs = []
    for chunks in ((40,), (1,) * 40, (33, 7)):
        box = _box(dpd, p)
        box.set_state(x, v)
        for c in chunks:
            box.step(c)
        outs.append(box.get_state())
    for xg, vg in outs[1:]:
        assert np.array_equal(xg, outs[0][0]) and np.array_equal(vg, outs[0][1])


def test_reloading_a_state_equals_a_fresh_context(dpd):
    """A context that loads a new state of the same size keeps its packing,
    tables and captured graphs: its run from the new state is the run of a
    fresh context, bitwise (full stencil), also after a parameter change
    between the two runs; a state of another size takes a new layout."""
    L = 8.0
    x1, v1 = uniform_box_state(L, rho=3, seed=1)
    x2, v2 = uniform_box_state(L, rho=3, seed=2)
    x3, v3 = uniform_box_state(L, rho=4, seed=3)
    p = _params(L, seed=1)
    box = _box(dpd, p)
    box.set_state(x1, v1)
    box.step(40)                                 # graphs captured
    box.set_param(dpd.PARAM_BODYFORCE, 0.3)
    for x, v in ((x2, v2), (x3, v3), (x3, v3)):
        box.set_state(x, v)
        box.step(45)
        ref = _box(dpd, p)
        ref.set_param(dpd.PARAM_BODYFORCE, 0.3)
        ref.set_state(x, v)
        ref.step(45)
        (xa, va), (xb, vb) = box.get_state(), ref.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.array_equal(box.get_forces(), ref.get_forces())
        assert box.stats()["step"] == ref.stats()["step"] == 45
        ref.close()
    box.close()


@pytest.mark.parametrize("body", [False, True])
def test_fused_integrate_gives_the_same_bits(dpd, body):
    """Full stencil: the force kernel doing the next step's kick, drift and
    binning (default) against separate kernels: identical state, forces and
    statistics after graph chunks and direct steps."""
    L = (7.0, 8.5, 6.25)
    x, v = uniform_box_state(L, rho=4, seed=21)
    p = _params(L, seed=21, fb=0.3 if body else 0.0, fb_mode=O.FB_POISEUILLE if body else 0)
    outs = []
    for fuse in (1, 0):
        box = _box(dpd, p)
        box.set_param(dpd.PARAM_FUSE, fuse)
        assert box.get_param(dpd.PARAM_FUSE) == fuse
        box.set_state(x, v)
        for c in (70, 3, 1):            # two 32-step graphs + 6 direct, then short calls
            box.step(c)
        xs, vs = box.get_state()
        outs.append((xs, vs, box.get_forces(), box.stats()))
    (x1, v1, f1, s1), (x0, v0, f0, s0) = outs
    assert np.array_equal(x1, x0) and np.array_equal(v1, v0) and np.array_equal(f1, f0)
    assert s1["virial"] == s0["virial"] and s1["step"] == s0["step"] == 74


def test_box_sums_match_fp64_sums_of_the_state(dpd):
    """The statistics' box sums against FP64 sums of the same FP32 velocities
    read back: momentum to 1e-10 of sum |v| (the per-thread sums are
    error-free pairs of FP32 numbers, the rest FP64); the kinetic energy to
    1e-7 (|v|^2 is formed in FP32)."""
    L = 24.0
    x, v = uniform_box_state(L, rho=3, seed=3)
    p = _params(L, seed=3)
    box = _box(dpd, p)
    box.set_state(x, v)
    box.step(7)
    st = box.stats()
    _, vg = box.get_state()
    vd = vg.astype(np.float64)
    P = vd.sum(0)
    assert np.abs(np.asarray(st["momentum"]) - P).max() <= 1e-10 * np.abs(vd).sum()
    ke = 0.5 * (vd ** 2).sum()
    assert st["kinetic"] == pytest.approx(ke, rel=1e-7)


def test_device_pointer_io_matches_host(dpd):
    import torch
    L = 6.0
    x, v = uniform_box_state(L, rho=3, seed=5)
    p = _params(L, seed=5)
    b1 = _box(dpd, p)
    b1.set_state(x, v)
    b2 = _box(dpd, p)
    b2.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda())
    b1.step(10)
    b2.step(10)
    xh, vh = b1.get_state()
    xd, vd = b2.get_state(device=True)
    assert np.array_equal(xh, xd.cpu().numpy()) and np.array_equal(vh, vd.cpu().numpy())
    assert np.array_equal(b1.get_forces(), b2.get_forces(device=True).cpu().numpy())


def test_user_stream(dpd):
    import torch
    L = 6.0
    x, v = uniform_box_state(L, rho=3, seed=5)
    p = _params(L, seed=5)
    s = torch.cuda.Stream()
    b1 = _box(dpd, p)
    b1.set_stream(s)
    b1.set_state(x, v)
    b1.step(40)
    b2 = _box(dpd, p)
    b2.set_state(x, v)
    b2.step(40)
    assert np.array_equal(b1.get_state()[0], b2.get_state()[0])


def test_non_finite_input_is_reported(dpd):
    L = 5.0
    x, v = uniform_box_state(L, rho=3, seed=1)
    v[3, 1] = np.nan
    box = _box(dpd, _params(L))
    box.set_state(x, v)
    box.step(2)
    with pytest.raises(dpd.DPDError) as ei:
        box.get_state()
    assert ei.value.code == dpd.ERR_NUMERIC


# -------------------------------------------------- full-size sampled parity
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("L", [64.0, 128.0])
def test_full_size_forces_sampled(dpd, L, stencil):
    """Full-size boxes in the launch configuration the benchmark times (the
    half stencil with its tuned variant at L = 128) and with the full stencil:
    sampled forces against the oracle, and properties that hold at any size."""
    x, v = uniform_box_state(L, rho=3, seed=0)
    p = _params(L, seed=0)
    box = _box(dpd, p, stencil)
    box.set_state(x, v)
    box.step(3)                         # exercise binning at full size
    xg, vg = box.get_state()
    box2 = _box(dpd, p, stencil)
    box2.set_state(xg, vg)
    fg = box2.get_forces()
    which = np.random.default_rng(1).choice(len(x), 1500, replace=False)
    f_ref = O.forces_subset(p, xg, vg, which, 0)
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    err = np.abs(fg[which].astype(np.float64) - f_ref).max()
    assert err <= FORCE_TOL * rms, (err, rms)
    # properties at full size: zero net pair force, ids intact, positions in box
    ssum = np.abs(fg.astype(np.float64).sum(0)).max()
    assert ssum <= 1e-6 * np.abs(fg).sum()
    assert np.all(xg >= 0) and np.all(xg < L)
    # momentum balance over 20 more steps at full size
    box.step(20)
    _, v2 = box.get_state()
    dP = v2.astype(np.float64).sum(0) - vg.astype(np.float64).sum(0)
    assert np.abs(dP).max() <= 1e-6 * np.abs(v2).sum()
    box.close()
    box2.close()


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("L,rho,a,fb", [
    (48.0, 3.0, 25.0, 0.05),              # the density sweep, with its Poiseuille force
    (48.0, 5.0, 15.0, 0.05),
    (48.0, 10.0, 7.5, 0.05),
    ((47.3, 31.9, 20.6), 5.0, 40.0, 0.0),  # a served-stream-like box: non-integer edges
])
def test_workload_sizes_sampled_forces(dpd, L, rho, a, fb, stencil):
    """Boxes at the sizes of the density sweep and of the served stream:
    sampled forces after a few steps against the oracle, with the body
    force and both stencils."""
    x, v = uniform_box_state(L, rho=rho, seed=21)
    kw = dict(fb=fb, fb_mode=O.FB_POISEUILLE, fb_flow=0, fb_grad=1) if fb else {}
    p = _params(L, seed=21, a=a, **kw)
    box = _box(dpd, p, stencil)
    box.set_state(x, v)
    box.step(4)
    xg, vg = box.get_state()
    box2 = _box(dpd, p, stencil)
    box2.set_state(xg, vg)
    fg = box2.get_forces()
    which = np.random.default_rng(2).choice(len(x), 1000, replace=False)
    f_ref = O.forces_subset(p, xg, vg, which, 0)
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    assert np.abs(fg[which].astype(np.float64) - f_ref).max() <= FORCE_TOL * rms
    box.close()
    box2.close()


@pytest.mark.parametrize("tiling", [dict(tiles=0), dict(tiles=1), dict(tiles=1, tile_cells=1),
                                    dict(tiles=1, tile_cells=3), dict(tiles=1, tile_cells=5),
                                    dict(tiles=1, tile_cells=64),
                                    dict(tiles=1, stage_cap=64)])  # 64: blocks overflow -> global path
def test_force_tiling_variants(dpd, tiling):
    for L, rho in (((5.0, 6.5, 7.25), 3), (3.0, 5), (8.0, 3), (4.0, 10)):
        x, v = uniform_box_state(L, rho=rho, seed=11)
        p = _params(L, seed=11)
        box = dpd.Box(p.L, a=p.a, gamma=p.gamma, kT=p.kT, rc=p.rc, dt=p.dt, seed=p.seed, **tiling)
        box.set_state(x, v)
        f_ref, vir = O.forces(p, x, v, 0)
        _force_check(box.get_forces(), f_ref)
        assert box.stats()["virial"] == pytest.approx(vir, rel=1e-5)
        box.step(5)
        xg, vg = box.get_state()
        b2 = dpd.Box(p.L, a=p.a, gamma=p.gamma, kT=p.kT, rc=p.rc, dt=p.dt, seed=p.seed, tiles=0)
        b2.set_state(x, v)
        b2.step(5)
        x2, _ = b2.get_state()
        assert np.abs(_min_image(xg.astype(np.float64) - x2, L)).max() < 1e-4


def test_half_stencil_every_variant_matches_oracle(dpd):
    """Each force-kernel variant with the half stencil (per-lane, balanced and
    spread drains) against the oracle; rho = 10 overflows the pair lists, so
    every variant drains several times per row."""
    from paper_1911_04712_gb300 import batch as B
    for L, rho in (((5.0, 6.5, 7.25), 3), (4.0, 10), (9.0, 5)):
        x, v = uniform_box_state(L, rho=rho, seed=13)
        p = _params(L, seed=13)
        f_ref, vir = O.forces(p, x, v, 0)
        ref_traj = None
        for variant in range(B.NUM_FORCE_VARIANTS):
            box = _box(dpd, p, stencil=1)
            box.set_param(dpd.PARAM_FORCE_VARIANT, variant)
            box.set_state(x, v)
            _force_check(box.get_forces(), f_ref)
            assert box.stats()["virial"] == pytest.approx(vir, rel=1e-5)
            box.step(5)
            xg, _ = box.get_state()
            if ref_traj is None:
                ref_traj = xg.astype(np.float64)
            assert np.abs(_min_image(xg.astype(np.float64) - ref_traj, L)).max() < 1e-4, variant


def test_tiling_knobs_reported(dpd):
    box = dpd.Box(8.0, tiles=1, tile_cells=5, stage_cap=512)
    x, v = uniform_box_state(8.0, rho=3, seed=0)
    box.set_state(x, v)
    assert box.tiling() == {"tiles": 1, "tile_cells": 5, "stage_cap": 512}
    with pytest.raises(dpd.DPDError):
        box.set_param(dpd.PARAM_STAGE_CAP, 10)


# ------------------------------------------------------------ checkpoints
@pytest.mark.parametrize("stencil", [0, 1])
def test_checkpoint_resume(dpd, stencil):
    L = 7.0
    x, v = uniform_box_state(L, rho=3, seed=12)
    p = _params(L, seed=12)
    a = _box(dpd, p, stencil)
    a.set_state(x, v)
    a.step(50)
    ck = a.checkpoint()
    a.step(50)
    xa, va = a.get_state()
    b = _box(dpd, p, stencil)
    b.restore(ck)
    assert b.stats()["step"] == 50
    b.step(50)
    xb, vb = b.get_state()
    if stencil == 0:
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    else:
        assert np.abs(_min_image(xa.astype(np.float64) - xb, L)).max() < 1e-4
    other = _box(dpd, _params(L, seed=13), stencil)
    with pytest.raises(dpd.DPDError) as ei:
        other.restore(ck)
    assert ei.value.code == dpd.ERR_STATE


# ------------------------------------------------ Gaussian noise (Sec. 2.1)
def test_gaussian_noise_words_and_values(dpd):
    rng = np.random.default_rng(8)
    n = 1 << 14
    lo = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    w0, w1, xi = dpd.debug_rng(lo, hi, 123, 456, noise=dpd.NOISE_GAUSSIAN, word1=True)
    r0, r1, rxi = O.pair_rng_gauss(lo, hi, 123, 456)
    assert np.array_equal(w0, r0) and np.array_equal(w1, r1)
    assert np.abs(xi.astype(np.float64) - rxi).max() < 2e-6 * max(1.0, np.abs(rxi).max())


@pytest.mark.parametrize("stencil", [0, 1])
def test_gaussian_noise_forces_and_trajectory(dpd, stencil):
    L = 8.0
    x, v = uniform_box_state(L, rho=3, seed=2)
    p = _params(L, seed=2, noise=1)
    box = _box(dpd, p, stencil)
    box.set_param(dpd.PARAM_NOISE, dpd.NOISE_GAUSSIAN)
    box.set_state(x, v)
    f_ref, _ = O.forces(p, x, v, 0)
    _force_check(box.get_forces(), f_ref)
    box.step(100)
    xg, _ = box.get_state()
    s = O.State(p, x, v)
    s.run(100)
    assert np.abs(_min_image(xg.astype(np.float64) - s.x, L)).max() < TRAJ_TOL
