"""Pins for the oracle's pair forces, cell list and integrator.

Each test checks the oracle against something the paper or the mathematics
fixes, not against a retyping of the oracle's own formula:

* closed forms of Eqs. 3-5 on hand-built two-particle states (each term
  isolated by zeroing the others), the cut-off of Eq. 4, periodic images;
* exact antisymmetry F_ij = -F_ji (Newton's third law, Sec. 2.1), hence zero
  total force and conserved momentum;
* the Sec. 3.2 cell list against the plain O(N^2) sum on tiny boxes;
* free streaming when every force vanishes (Eq. 1 alone);
* time reversibility and bounded energy error of velocity-Verlet with only
  the conservative force, whose potential (a rc / 2)(1 - r/rc)^2 is the
  closed-form integral of Eq. 3;
* momentum gained from a body force (Sec. 4.2): exactly dt times its sum.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _two(rng, r, L=10.0):
    e = _unit(rng)
    xj = rng.uniform(3.0, L - 3.0, 3)
    xi = xj + r * e
    return xi, xj, e


@pytest.mark.parametrize("rc", [1.0, 1.3])
def test_conservative_term_closed_form(rc):
    rng = np.random.default_rng(0)
    p = O.Params(L=(10, 10, 10), a=25.0, gamma=0.0, kT=0.0, rc=rc)
    for r in np.linspace(0.05, rc * 0.999, 25):
        xi, xj, e = _two(rng, r)
        f, rfc = O.pair_force(p, xi, xj, np.zeros(3), np.zeros(3), 3, 8, 0)
        want = 25.0 * (1.0 - r / rc) * e          # repulsive: along r_i - r_j
        np.testing.assert_allclose(f, want, rtol=1e-12, atol=1e-12)
        assert rfc == pytest.approx(25.0 * (1.0 - r / rc) * r, rel=1e-12)


def test_dissipative_term_closed_form_and_sign():
    rng = np.random.default_rng(1)
    p = O.Params(L=(10, 10, 10), a=0.0, gamma=4.5, kT=0.0)
    for _ in range(50):
        r = rng.uniform(0.05, 0.99)
        xi, xj, e = _two(rng, r)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        f, _ = O.pair_force(p, xi, xj, vi, vj, 1, 2, 0)
        w = 1.0 - r
        want = -4.5 * w * w * np.dot(e, vi - vj) * e
        np.testing.assert_allclose(f, want, rtol=1e-11, atol=1e-13)
        # friction never adds relative kinetic energy
        assert np.dot(f, vi - vj) <= 1e-14


def test_random_term_amplitude_follows_fluctuation_dissipation():
    rng = np.random.default_rng(2)
    gamma, kT, dt = 4.5, 1.7, 0.005
    p = O.Params(L=(10, 10, 10), a=0.0, gamma=gamma, kT=kT, dt=dt, seed=99)
    sigma = math.sqrt(2.0 * gamma * kT)
    for k in range(50):
        r = rng.uniform(0.05, 0.99)
        xi, xj, e = _two(rng, r)
        f, _ = O.pair_force(p, xi, xj, np.zeros(3), np.zeros(3), 10 + k, 500 + k, 7)
        _, xis = O.pair_rng([10 + k], [500 + k], 7, 99)
        want = sigma * (1.0 - r) * xis[0] / math.sqrt(dt) * e
        np.testing.assert_allclose(f, want, rtol=1e-12, atol=1e-13)


def test_weight_exponent_k():
    rng = np.random.default_rng(3)
    k = 0.5
    gamma, kT, dt = 2.0, 1.0, 0.01
    r = 0.4
    xi, xj, e = _two(rng, r)
    w = 1.0 - r
    pr = O.Params(L=(10, 10, 10), a=0.0, gamma=gamma, kT=kT, dt=dt, kexp=k)
    f, _ = O.pair_force(pr, xi, xj, np.zeros(3), np.zeros(3), 4, 5, 1)
    _, xis = O.pair_rng([4], [5], 1, 0)
    np.testing.assert_allclose(f, math.sqrt(2 * gamma * kT) * w ** k * xis[0] / math.sqrt(dt) * e,
                               rtol=1e-12)
    pd = O.Params(L=(10, 10, 10), a=0.0, gamma=gamma, kT=0.0, dt=dt, kexp=k)
    vi = np.array([0.3, -1.0, 0.2])
    f, _ = O.pair_force(pd, xi, xj, vi, np.zeros(3), 4, 5, 1)
    np.testing.assert_allclose(f, -gamma * w ** (2 * k) * np.dot(e, vi) * e, rtol=1e-12)


def test_cutoff_and_periodic_image():
    p = O.Params(L=(5.0, 6.0, 7.0), a=25.0, gamma=4.5, kT=1.0)
    z = np.zeros(3)
    f, _ = O.pair_force(p, [1, 1, 1], [2.0, 1, 1], z, z, 0, 1, 0)        # r == rc
    assert np.all(f == 0)
    f, _ = O.pair_force(p, [1, 1, 1], [1, 1, 1], z, z, 0, 1, 0)          # r == 0
    assert np.all(f == 0)
    # a pair across the x faces: images 0.3 apart
    f_wrap, _ = O.pair_force(p, [0.1, 3, 3], [4.8, 3, 3], z, z, 0, 1, 0)
    f_near, _ = O.pair_force(p, [5.1, 3, 3], [4.8, 3, 3], z, z, 0, 1, 0)
    np.testing.assert_allclose(f_wrap, f_near, rtol=1e-12)
    assert f_wrap[0] > 0                                               # pushed away from j


def test_pair_forces_are_exactly_antisymmetric():
    rng = np.random.default_rng(4)
    p = O.Params(L=(6, 6, 6), a=25.0, gamma=4.5, kT=1.0, seed=3)
    for _ in range(200):
        xi, xj = rng.uniform(0, 6, 3), rng.uniform(0, 6, 3)
        xj = xi + rng.uniform(-0.6, 0.6, 3)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        a, b = rng.integers(0, 1000, 2)
        fij, _ = O.pair_force(p, xi, xj, vi, vj, a, b, 11)
        fji, _ = O.pair_force(p, xj, xi, vj, vi, b, a, 11)
        assert np.array_equal(fij, -fji)


def _state_with_boundary_particles(L, rho, seed):
    x, v = uniform_box_state(L, rho=rho, seed=seed)
    rng = np.random.default_rng(seed)
    L3 = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    n = x.shape[0]
    k = max(4, n // 8)
    idx = rng.choice(n, k, replace=False)
    # put some coordinates on or next to cell faces and box faces
    for j, i in enumerate(idx):
        ax = j % 3
        nd = math.floor(L3[ax])
        h = L3[ax] / nd
        face = rng.integers(0, nd) * h
        x[i, ax] = np.float32(min(max(face + rng.choice([-1e-6, 0.0, 1e-6]), 0.0), L3[ax] - 1e-5))
    return x, v


@pytest.mark.parametrize("L,rho", [(3, 3), (4, 5), (5, 3), (6, 4), ((3.0, 4.5, 5.25), 4),
                                   ((7.3, 3.1, 4.0), 3)])
def test_cell_list_equals_brute_force(L, rho):
    x, v = _state_with_boundary_particles(L, rho, seed=hash(str(L)) % 1000)
    p = O.Params(L=np.broadcast_to(np.asarray(L, float), (3,)), a=25.0, gamma=4.5, kT=1.0, seed=1)
    fb, vb = O.forces(p, x, v, 5, mode=O.MODE_BRUTE)
    fc, vc = O.forces(p, x, v, 5, mode=O.MODE_CELLS)
    rms = math.sqrt((fb ** 2).sum(1).mean())
    np.testing.assert_allclose(fc, fb, rtol=0, atol=1e-11 * rms)
    assert vc == pytest.approx(vb, rel=1e-12)
    which = np.arange(0, x.shape[0], 3)
    fs = O.forces_subset(p, x, v, which, 5)
    np.testing.assert_allclose(fs, fb[which], rtol=0, atol=1e-11 * rms)


def test_total_force_zero_and_momentum_conserved():
    x, v = uniform_box_state(8, rho=3, seed=0)
    p = O.Params(L=(8, 8, 8), seed=0)
    f, _ = O.forces(p, x, v, 0)
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).sum()
    s = O.State(p, x, v)
    P0 = s.stats()["P"]
    s.run(50)
    scale = np.abs(s.v).sum()
    assert np.abs(s.stats()["P"] - P0).max() <= 1e-12 * scale


def test_constant_body_force_adds_exact_momentum():
    x, v = uniform_box_state(6, rho=3, seed=1)
    f0 = 0.05
    p = O.Params(L=(6, 6, 6), fb=f0, fb_mode=O.FB_CONST, fb_flow=0, seed=2)
    s = O.State(p, x, v, mode=O.MODE_CELLS)
    P0 = s.stats()["P"].copy()
    nst = 40
    s.run(nst)
    dP = s.stats()["P"] - P0
    n = x.shape[0]
    assert dP[0] == pytest.approx(n * f0 * nst * p.dt, rel=1e-10)
    assert abs(dP[1]) < 1e-10 and abs(dP[2]) < 1e-10


def test_poiseuille_body_force_momentum_step_by_step():
    x, v = uniform_box_state(6, rho=3, seed=2)
    f0 = 0.5
    p = O.Params(L=(6, 6, 6), fb=f0, fb_mode=O.FB_POISEUILLE, fb_flow=2, fb_grad=0, seed=2)
    s = O.State(p, x, v, mode=O.MODE_CELLS)

    def fb_sum(xx):
        # Sec. 4.2: (0, 0, -f) for r_x <= L/2, (0, 0, +f) above
        return np.where(xx[:, 0] <= 3.0, -f0, f0).sum()

    for _ in range(20):
        P0 = s.stats()["P"][2]
        b0 = fb_sum(s.x)
        s.run(1)
        b1 = fb_sum(s.x)
        # velocity-Verlet: half a kick with the old body force, half with the new
        assert s.stats()["P"][2] - P0 == pytest.approx(0.5 * p.dt * (b0 + b1), abs=1e-10)


def test_free_streaming_without_forces():
    x, v = uniform_box_state((5, 6, 7), rho=3, seed=3)
    p = O.Params(L=(5, 6, 7), a=0.0, gamma=0.0, kT=0.0)
    s = O.State(p, x, v)
    nst = 60
    s.run(nst)
    L = np.array([5.0, 6.0, 7.0])
    want = np.mod(x.astype(np.float64) + nst * p.dt * v.astype(np.float64), L)
    d = s.x - want
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-12
    np.testing.assert_array_equal(s.v, v.astype(np.float64))


def _potential(x, L, a, rc):
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    iu = np.triu_indices(x.shape[0], 1)
    r = r[iu]
    r = r[r < rc]
    return (0.5 * a * rc * (1.0 - r / rc) ** 2).sum()


def test_conservative_dynamics_reversible_and_energy_bounded():
    L = 5.0
    x, v = uniform_box_state(L, rho=3, seed=4)
    p = O.Params(L=(L, L, L), a=25.0, gamma=0.0, kT=0.0, dt=0.005)
    s = O.State(p, x, v)
    e0 = 0.5 * (s.v ** 2).sum() + _potential(s.x, L, 25.0, 1.0)
    drift = []
    for _ in range(10):
        s.run(20)
        e = 0.5 * (s.v ** 2).sum() + _potential(s.x, L, 25.0, 1.0)
        drift.append(abs(e - e0) / e0)
    # velocity-Verlet is second order: the energy error stays O(dt^2), no drift
    assert max(drift) < 2e-3
    # reverse the velocities and integrate back to the start
    s.v *= -1.0
    s.f, s.virial = O.forces(p, s.x, s.v, s.step)
    s.run(200)
    d = s.x - x.astype(np.float64)
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-8
