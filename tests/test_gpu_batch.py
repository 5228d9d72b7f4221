"""Batched form: many uneven boxes in one packed set, against each box alone
and against the oracle."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import box_mix, uniform_box_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.batch as B
    import paper_1911_04712_gb300.dpd as D
    return D, B


def _mix(nbox=10, seed=3):
    specs = box_mix(nbox, master_seed=seed, L_range=(3, 9))
    states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=100 + k) for k, s in enumerate(specs)]
    return specs, states


def _alone(D, s, x, v, nsteps, stencil=0):
    box = D.Box(s.L, a=s.a, gamma=s.gamma, kT=s.kT, rc=1.0, dt=s.dt, seed=s.seed,
                stencil=stencil)
    box.set_state(x, v)
    box.step(nsteps)
    out = box.get_state()
    f = box.get_forces()
    box.close()
    return out, f


@pytest.mark.parametrize("stencil", [0, 1])
def test_batch_equals_each_box_alone(mods, stencil):
    D, B = mods
    specs, states = _mix()
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    bt = B.Batch(descs, stencil=stencil)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    nst = 45                                    # one 32-step graph + 13 direct steps
    bt.step(nst)
    stats = bt.stats()
    for k, (s, (x, v)) in enumerate(zip(specs, states)):
        (xa, va), fa = _alone(D, s, x, v, nst, stencil)
        xb, vb = bt.get_state(k)
        fb = bt.get_forces(k)
        if stencil == 0:
            assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb), k
        else:   # atomics: same up to summation order (measured: ~2e-6 after 45 steps)
            d = xb.astype(np.float64) - xa
            d -= s.L * np.round(d / s.L)
            assert np.abs(d).max() < 1e-4, k
            rms = np.sqrt((fa.astype(np.float64) ** 2).sum(1).mean())
            assert np.abs(fb.astype(np.float64) - fa).max() < 1e-3 * rms, k
        assert stats[k]["step"] == nst and stats[k]["n"] == len(x)


@pytest.mark.parametrize("stencil", [0, 1])
def test_batch_every_variant_matches_each_box_alone(mods, stencil):
    """Every force-kernel variant on a packed mix, where warps straddle box
    boundaries: the same trajectory and forces as each box alone (bitwise
    for the full stencil, up to summation order for the half stencil)."""
    D, B = mods
    specs, states = _mix(8, seed=6)
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    alone = [_alone(D, s, x, v, 3, stencil) for s, (x, v) in zip(specs, states)]
    table = stencil + B.TUNING_PACKED
    up0, var0 = B.tuning_get(table)
    try:
        for variant in range(B.NUM_FORCE_VARIANTS):
            B.tuning_set(table, [1e9], [variant])
            bt = B.Batch(descs, stencil=stencil)
            for k, (x, v) in enumerate(states):
                bt.set_state(k, x, v)
            bt.step(3)
            for k, (s, ((xa, va), fa)) in enumerate(zip(specs, alone)):
                xb, _ = bt.get_state(k)
                fb = bt.get_forces(k)
                if stencil == 0:
                    assert np.array_equal(xa, xb) and np.array_equal(fa, fb), (variant, k)
                else:
                    d = xb.astype(np.float64) - xa
                    d -= s.L * np.round(d / s.L)
                    rms = np.sqrt((fa.astype(np.float64) ** 2).sum(1).mean())
                    assert np.abs(d).max() < 1e-5, (variant, k)
                    assert np.abs(fb.astype(np.float64) - fa).max() < 1e-4 * rms, (variant, k)
            bt.close()
    finally:
        B.tuning_set(table, up0, var0)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("variants", [(11, 10, 12), (7, 12, 8), (0, 9, 10), (12, 2, 11)])
def test_batch_bands_with_different_variants(mods, stencil, variants):
    """Several force bands, each its own launch with its own variant: the lanes
    past a band's end belong to the next band's box and must not take part in
    another box's drain."""
    D, B = mods
    specs, states = _mix()
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    alone = [_alone(D, s, x, v, 2, stencil) for s, (x, v) in zip(specs, states)]
    table = stencil + B.TUNING_PACKED
    up0, var0 = B.tuning_get(table)
    try:
        B.tuning_set(table, [3.5, 4.5, 1e9], list(variants))   # rho 3 / 4 / 5: three bands
        bt = B.Batch(descs, stencil=stencil)
        for k, (x, v) in enumerate(states):
            bt.set_state(k, x, v)
        bt.step(2)
        for k, (s, ((xa, va), fa)) in enumerate(zip(specs, alone)):
            fb = bt.get_forces(k).astype(np.float64)
            rms = np.sqrt((fa.astype(np.float64) ** 2).sum(1).mean())
            if stencil == 0:
                assert np.array_equal(fb, fa), (variants, k)
            else:
                assert np.abs(fb - fa).max() < 1e-4 * rms, (variants, k)
        bt.close()
    finally:
        B.tuning_set(table, up0, var0)


def test_batch_fused_integrate_with_step_limits(mods):
    """Full stencil, packed boxes of which some stop mid-chunk (their step
    limits): fused and unfused steps give the same bits."""
    D, B = mods
    specs, states = _mix(7, seed=8)
    limits = [0, 5, 33, 0, 64, 1, 40]
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed,
                         steps=lim) for s, st, lim in zip(specs, states, limits)]
    outs = []
    for fuse in (1, 0):
        bt = B.Batch(descs, stencil=0)
        bt.set_option(D.PARAM_FUSE, fuse)
        for k, (x, v) in enumerate(states):
            bt.set_state(k, x, v)
        bt.step(50)
        bt.step(20)
        outs.append([(bt.get_state(k), bt.get_forces(k)) for k in range(len(specs))])
        st = bt.stats()
        for k, lim in enumerate(limits):
            assert st[k]["step"] == (70 if lim == 0 else min(lim, 70))
        bt.close()
    for ((xa, va), fa), ((xb, vb), fb) in zip(*outs):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb)


@pytest.mark.parametrize("stencil", [0, 1])
def test_batch_with_species_equals_each_box_alone(mods, stencil):
    """Boxes of several species packed with one-species boxes (the general
    force kernel's bands beside the tuned ones): each box as alone in a
    context with the same tables (bitwise for the full stencil)."""
    D, B = mods
    specs, states = _mix(6, seed=9)
    A = np.array([[25.0, 40.0, 31.0], [40.0, 18.0, 55.0], [31.0, 55.0, 12.0]])
    G = np.array([[4.5, 2.0, 6.0], [2.0, 3.5, 1.5], [6.0, 1.5, 8.0]])
    R = np.array([[1.0, 0.8, 0.9], [0.8, 0.7, 0.95], [0.9, 0.95, 0.85]])
    tables = [None, (A, G, R), None, (A[:2, :2], G[:2, :2], R[:2, :2]), (A, G, R), None]
    labels = [None if t is None else
              np.random.default_rng(k).integers(0, t[0].shape[0], len(st[0])).astype(np.int32)
              for k, (t, st) in enumerate(zip(tables, states))]
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed,
                         species=t) for s, st, t in zip(specs, states, tables)]
    bt = B.Batch(descs, stencil=stencil)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v, species=labels[k])
    bt.step(40)
    for k, (s, (x, v)) in enumerate(zip(specs, states)):
        box = D.Box(s.L, a=s.a, gamma=s.gamma, kT=s.kT, rc=1.0, dt=s.dt, seed=s.seed,
                    stencil=stencil)
        if tables[k] is not None:
            box.set_species(*tables[k])
        box.set_state(x, v, species=labels[k])
        box.step(40)
        xa, fa = box.get_state()[0], box.get_forces()
        xb, fb = bt.get_state(k)[0], bt.get_forces(k)
        if stencil == 0:
            assert np.array_equal(xa, xb) and np.array_equal(fa, fb), k
        else:
            d = xb.astype(np.float64) - xa
            d -= s.L * np.round(d / s.L)
            assert np.abs(d).max() < 1e-4, k
        box.close()
    bt.close()


def test_batch_boxes_match_oracle(mods):
    D, B = mods
    specs, states = _mix(6, seed=4)
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    bt = B.Batch(descs)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    f0 = [bt.get_forces(k) for k in range(len(specs))]
    bt.step(40)
    for k, (s, (x, v)) in enumerate(zip(specs, states)):
        p = O.Params(L=(s.L,) * 3, a=s.a, gamma=s.gamma, kT=s.kT, rc=1.0, dt=s.dt, seed=s.seed)
        fr, _ = O.forces(p, x, v, 0)
        rms = math.sqrt((fr ** 2).sum(1).mean())
        assert np.abs(f0[k] - fr).max() <= 1e-5 * rms
        st = O.State(p, x, v)
        st.run(40)
        xb, _ = bt.get_state(k)
        d = xb.astype(np.float64) - st.x
        d -= s.L * np.round(d / s.L)
        assert np.abs(d).max() < 1e-3


@pytest.mark.parametrize("stencil", [0, 1])
def test_batch_step_limits_freeze_boxes(mods, stencil):
    """A box that reached its step limit stays as it stopped while the others
    go on: its positions, full-step velocities (which take the half kick of
    its last force) and forces as alone after the same steps (bitwise for
    the full stencil, up to summation order for the half stencil, whose
    reorder keeps a stopped box's slots and forces)."""
    D, B = mods
    x1, v1 = uniform_box_state(4.0, rho=3, seed=1)
    x2, v2 = uniform_box_state(5.0, rho=4, seed=2)
    descs = [B.make_desc(4.0, len(x1), seed=1, steps=10), B.make_desc(5.0, len(x2), seed=2)]
    bt = B.Batch(descs, stencil=stencil)
    bt.set_state(0, x1, v1)
    bt.set_state(1, x2, v2)
    bt.step(25)
    st = bt.stats()
    assert st[0]["step"] == 10 and st[1]["step"] == 25
    (xa, va), fa = _alone(D, type("S", (), dict(L=4.0, a=25.0, gamma=4.5, kT=1.0, dt=0.005,
                                                seed=1))(), x1, v1, 10, stencil)
    xb, vb = bt.get_state(0)
    fb = bt.get_forces(0)
    if stencil == 0:
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    else:
        rms = np.sqrt((fa.astype(np.float64) ** 2).sum(1).mean())
        assert np.abs(xb.astype(np.float64) - xa).max() < 1e-5
        assert np.abs(vb.astype(np.float64) - va).max() < 1e-4
        assert np.abs(fb.astype(np.float64) - fa).max() < 1e-4 * rms


def test_batch_rejects_bad_descs_and_unloaded_boxes(mods):
    D, B = mods
    with pytest.raises(D.DPDError) as ei:
        B.Batch([B.make_desc(4.0, 10), B.make_desc(2.0, 10)])
    assert "box 1" in str(ei.value)
    bt = B.Batch([B.make_desc(4.0, 10), B.make_desc(4.0, 10)])
    x, v = uniform_box_state(4.0, n=10, seed=0)
    bt.set_state(0, x, v)
    with pytest.raises(D.DPDError) as ei:
        bt.step(1)
    assert ei.value.code == D.ERR_STATE


def test_tuning_table_roundtrip_and_variants_agree(mods):
    D, B = mods
    up0, var0 = B.tuning_get(0)
    try:
        B.tuning_set(0, [3.5, 4.5, 1e9], [1, 3, 5])
        assert B.tuning_get(0) == ([3.5, 4.5, 1e9], [1, 3, 5])
        x, v = uniform_box_state(6.0, rho=3, seed=5)
        outs = []
        for variant in range(B.NUM_FORCE_VARIANTS):
            box = D.Box(6.0, seed=5)
            box.set_param(D.PARAM_FORCE_VARIANT, variant)
            box.set_state(x, v)
            box.step(20)
            outs.append(box.get_state()[0])
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
    finally:
        B.tuning_set(0, up0, var0)


def test_full_mix_in_the_benchmark_configuration(mods):
    """The 512-box mix at full size, packed and launched as the benchmark runs
    it (half stencil, tuned packed tables): every box's momentum balance after
    20 steps, and a sample of boxes against the oracle (forces at load within
    1e-5 of the RMS, 20-step trajectories within 1e-3 rc)."""
    D, B = mods
    specs = box_mix(512, master_seed=0)
    states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=s.seed) for s in specs]
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    bt = B.Batch(descs, stencil=1)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    sample = np.random.default_rng(5).choice(len(specs), 6, replace=False)
    f0 = {int(k): bt.get_forces(int(k)) for k in sample}
    bt.step(20)
    for k, (x, v) in enumerate(states):
        _, vb = bt.get_state(k)
        dP = vb.astype(np.float64).sum(0) - v.astype(np.float64).sum(0)
        assert np.abs(dP).max() <= 1e-6 * np.abs(vb).sum() + 1e-6, k
    for k in sample:
        k = int(k)
        s, (x, v) = specs[k], states[k]
        p = O.Params(L=(s.L,) * 3, a=s.a, gamma=s.gamma, kT=s.kT, rc=1.0, dt=s.dt, seed=s.seed)
        fr, _ = O.forces(p, x, v, 0, mode=O.MODE_CELLS)
        rms = math.sqrt((fr ** 2).sum(1).mean())
        assert np.abs(f0[k] - fr).max() <= 1e-5 * rms, k
        st = O.State(p, x, v, mode=O.MODE_CELLS)
        st.run(20)
        xb, _ = bt.get_state(k)
        d = xb.astype(np.float64) - st.x
        d -= s.L * np.round(d / s.L)
        assert np.abs(d).max() < 1e-3, k
    bt.close()


@pytest.mark.parametrize("variant", [10, 11, 12])
def test_grouped_launches_over_many_boxes(mods, variant):
    """Half stencil, the packed spread-drain variants: the force stage runs as
    box-grouped launches (no block spans two boxes; at most 240 boxes per
    launch, their constants in the launch parameters).  250 small boxes,
    most with fewer particles than one block, some with the periodic
    Poiseuille force, some stopped after one step and three empty (one of
    them beside the launch boundary), all in one density band so that they
    are packed in the caller's order: the first and last boxes, those on
    both sides of the launch boundary and the stopped ones as each box
    alone."""
    D, B = mods
    rng = np.random.default_rng(11)
    n = 250
    empty = {5, 240, 249}
    Ls = rng.choice([3.0, 3.5, 4.0, 4.5], n)
    rhos = rng.choice([2.5, 3.0], n)
    fb = [0.05 if k % 5 == 2 else 0.0 for k in range(n)]
    limits = [1 if k % 7 == 3 else 0 for k in range(n)]
    states = [(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32)) if k in empty
              else uniform_box_state(L, rho=r, seed=300 + k)
              for k, (L, r) in enumerate(zip(Ls, rhos))]
    descs = [B.make_desc(L, len(st[0]), seed=300 + k, steps=lim, body_force=f, body_mode=2,
                         flow_axis=0, grad_axis=1)
             for k, (L, st, lim, f) in enumerate(zip(Ls, states, limits, fb))]
    table = 1 + B.TUNING_PACKED
    up0, var0 = B.tuning_get(table)
    nst = 3
    try:
        B.tuning_set(table, [1e9], [variant])
        bt = B.Batch(descs, stencil=1)
        for k, (x, v) in enumerate(states):
            bt.set_state(k, x, v)
        bt.step(nst)
        st = bt.stats()
        for k in empty:
            assert st[k]["n"] == 0, k
        check = sorted(({0, 1, 238, 239, 241, 242, n - 2} | {k for k in range(n) if limits[k]})
                       - empty)
        for k in check:
            x, v = states[k]
            box = D.Box(Ls[k], seed=300 + k, stencil=1, poiseuille_f=fb[k] if fb[k] else None,
                        flow_axis=0, grad_axis=1)
            box.set_state(x, v)
            steps = limits[k] if limits[k] else nst
            box.step(steps)
            (xa, va), fa = box.get_state(), box.get_forces().astype(np.float64)
            box.close()
            assert st[k]["step"] == steps, k
            (xb, vb), fb_ = bt.get_state(k), bt.get_forces(k).astype(np.float64)
            d = xb.astype(np.float64) - xa
            d -= Ls[k] * np.round(d / Ls[k])
            rms = np.sqrt((fa ** 2).sum(1).mean())
            assert np.abs(d).max() < 1e-5, k
            assert np.abs(vb.astype(np.float64) - va).max() < 1e-4, k
            assert np.abs(fb_ - fa).max() < 1e-4 * rms, k
        bt.close()
    finally:
        B.tuning_set(table, up0, var0)
