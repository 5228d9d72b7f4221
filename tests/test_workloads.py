"""Seeded input generators: shapes, ranges, determinism, zero mean momentum."""

import numpy as np

from paper_1911_04712_gb300.workloads import box_mix, particles_for, request_stream, uniform_box_state


def test_uniform_box_state_ranges_and_determinism():
    L = (5.0, 6.5, 7.25)
    x, v = uniform_box_state(L, rho=3, kT=1.5, seed=3)
    assert x.dtype == np.float32 and v.dtype == np.float32
    assert x.shape == (particles_for(L, 3), 3)
    assert np.all(x >= 0) and np.all(x < np.asarray(L, dtype=np.float32))
    assert np.abs(v.astype(np.float64).mean(0)).max() < 1e-6
    assert abs(v.astype(np.float64).var() - 1.5) < 0.1
    x2, v2 = uniform_box_state(L, rho=3, kT=1.5, seed=3)
    assert np.array_equal(x, x2) and np.array_equal(v, v2)
    x3, _ = uniform_box_state(L, rho=3, kT=1.5, seed=4)
    assert not np.array_equal(x, x3)


def test_empty_box():
    x, v = uniform_box_state(4, n=0)
    assert x.shape == (0, 3) and v.shape == (0, 3)


def test_box_mix_and_request_stream_recipes():
    mix = box_mix(64, master_seed=0)
    assert len(mix) == 64
    assert all(6 <= b.L <= 24 and b.rho in (3, 4, 5) for b in mix)
    assert all(10 <= b.a <= 80 and 2 <= b.gamma <= 8 and 0.5 <= b.kT <= 2 for b in mix)
    assert [b.seed for b in mix] == list(range(64))
    reqs = request_stream(500, rate=200.0)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() - 1 / 200) < 0.2 / 200
    assert all(8 <= r.L <= 48 and r.rho in (3, 5) and 1000 <= r.steps <= 20000 for r in reqs)
