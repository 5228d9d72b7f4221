"""Pins of the oracle's several-species interactions (the particle vectors of
Sec. 3.1, each pair of species with its own parameters and cut-off).

* Two particles, one pair of species at a time: the conservative force is
  a_st (1 - r / rc_st) along e_ij inside rc_st and zero between rc_st and the
  cell cut-off rc (Eqs. 3-4); the dissipative force is -gamma_st w^2 (e.v) e
  (Eq. 5).  The tables have distinct entries, so a transposed or misplaced
  index fails.
* The random force scales with sigma_st = sqrt(2 gamma_st kT) (the
  fluctuation-dissipation relation of Sec. 2.1) and uses the same pair noise
  as one species.
* Equal tables give the one-species forces exactly.
* Mean field (a / kT -> 0, g(r) -> 1): the excess pressure of a mixture with
  number fractions x_s is (2 pi / 3) rho^2 sum_st x_s x_t
  int_0^rc_st r^3 a_st (1 - r / rc_st) dr = (pi / 30) rho^2 sum_st x_s x_t
  a_st rc_st^4.
* The thermostat holds kT in a mixture.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state

A = np.array([[25.0, 40.0, 31.0], [40.0, 18.0, 55.0], [31.0, 55.0, 12.0]])
G = np.array([[4.5, 2.0, 6.0], [2.0, 3.5, 1.5], [6.0, 1.5, 8.0]])
RC = np.array([[1.0, 0.8, 0.9], [0.8, 0.7, 0.95], [0.9, 0.95, 0.85]])


def _pair(p, s, t, r, vrel=(0.0, 0.0, 0.0)):
    p.set_species([s, t], A, G, RC)
    xi = np.array([3.0, 3.0, 3.0])
    xj = xi - np.array([r, 0.0, 0.0])          # e_ij = +x
    return O.pair_force(p, xi, xj, np.array(vrel, float), np.zeros(3), 0, 1, 0)


@pytest.mark.parametrize("s,t", [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 1), (2, 2)])
def test_conservative_and_dissipative_per_species_pair(s, t):
    p = O.Params(L=(8.0, 8.0, 8.0), kT=0.0, rc=1.0)
    for r in (0.1, 0.5 * RC[s, t], 0.999 * RC[s, t]):
        f, rfc = _pair(p, s, t, r)
        w = 1.0 - r / RC[s, t]
        assert f[0] == pytest.approx(A[s, t] * w, rel=1e-12)
        assert f[1] == 0.0 and f[2] == 0.0
        assert rfc == pytest.approx(A[s, t] * w * r, rel=1e-12)
        # approaching along e: dissipative force opposes it with gamma_st w^2
        fd, _ = _pair(p, s, t, r, vrel=(-0.7, 0.0, 0.0))
        assert fd[0] - f[0] == pytest.approx(G[s, t] * w * w * 0.7, rel=1e-12)
    for r in (RC[s, t] * 1.0001, 0.5 * (RC[s, t] + 1.0) if RC[s, t] < 1.0 else 1.5):
        f, _ = _pair(p, s, t, r)
        assert np.all(f == 0.0)


def test_random_force_scales_with_sigma_of_the_pair():
    p = O.Params(L=(8.0, 8.0, 8.0), a=0.0, kT=1.3, dt=0.004, rc=1.0, seed=77)
    words, xi = O.pair_rng(np.array([0], np.uint32), np.array([1], np.uint32), 0, 77)
    for s, t in ((0, 1), (2, 2), (1, 2)):
        A0 = np.zeros_like(A)
        p.set_species([s, t], A0, G, RC)
        r = 0.4 * RC[s, t]
        f, _ = O.pair_force(p, np.array([3.0, 3.0, 3.0]), np.array([3.0 - r, 3.0, 3.0]),
                            np.zeros(3), np.zeros(3), 0, 1, 0)
        sigma = math.sqrt(2.0 * G[s, t] * p.kT)
        expect = sigma * xi[0] * (1.0 - r / RC[s, t]) / math.sqrt(p.dt)
        assert f[0] == pytest.approx(expect, rel=1e-12)


def test_equal_tables_give_one_species_forces():
    L = 6.0
    x, v = uniform_box_state(L, rho=3, seed=4)
    p1 = O.Params(L=(L, L, L), a=31.0, gamma=3.0, kT=1.0, seed=5)
    f1, vir1 = O.forces(p1, x, v, 3, mode=O.MODE_CELLS)
    rng = np.random.default_rng(0)
    p3 = O.Params(L=(L, L, L), a=31.0, gamma=3.0, kT=1.0, seed=5)
    p3.set_species(rng.integers(0, 3, len(x)), np.full((3, 3), 31.0), np.full((3, 3), 3.0),
                   np.ones((3, 3)))
    f3, vir3 = O.forces(p3, x, v, 3, mode=O.MODE_CELLS)
    assert np.array_equal(f1, f3) and vir1 == vir3


def test_cells_equal_brute_force_with_short_cut_offs():
    L = (5.0, 6.5, 7.25)
    x, v = uniform_box_state(L, rho=4, seed=6)
    p = O.Params(L=L, kT=1.0, seed=3)
    p.set_species(np.random.default_rng(1).integers(0, 3, len(x)), A, G, RC)
    fb, vb = O.forces(p, x, v, 2, mode=O.MODE_BRUTE)
    fc, vc = O.forces(p, x, v, 2, mode=O.MODE_CELLS)
    assert np.allclose(fb, fc, rtol=0, atol=1e-9) and vb == pytest.approx(vc, rel=1e-12)
    assert np.abs(fb.sum(0)).max() < 1e-9          # Newton's third law per pair


def test_pressure_mean_field_closed_form_for_a_mixture():
    L, rho, kT = 8, 3, 1000.0
    x, v = uniform_box_state(L, rho=rho, kT=kT, seed=2)
    n = len(x)
    sp = np.random.default_rng(3).integers(0, 3, n)
    frac = np.bincount(sp, minlength=3) / n
    p = O.Params(L=(L, L, L), kT=kT, dt=0.0003, seed=3)
    p.set_species(sp, A, G, RC)
    closed = (math.pi / 30.0) * rho ** 2 * sum(frac[s] * frac[t] * A[s, t] * RC[s, t] ** 4
                                                for s in range(3) for t in range(3))
    st = O.State(p, x, v, mode=O.MODE_CELLS)
    st.run(300)
    pex = []
    for _ in range(250):
        st.run(5)
        pex.append(st.virial / (3.0 * L ** 3))
    s = np.asarray(pex).reshape(10, -1).mean(1)
    m, err = s.mean(), s.std(ddof=1) / math.sqrt(10)
    print(f"mixture excess pressure {m:.4f} +- {err:.4f}, mean field {closed:.4f}")
    assert abs(m - closed) <= 0.005 * closed + 3.0 * err


def test_thermostat_in_a_mixture():
    L, kT = 6, 1.0
    x, v = uniform_box_state(L, rho=3, kT=kT, seed=9)
    p = O.Params(L=(L, L, L), kT=kT, dt=0.005, seed=11)
    p.set_species(np.random.default_rng(2).integers(0, 3, len(x)), A, G, RC)
    st = O.State(p, x, v, mode=O.MODE_CELLS)
    st.run(600)
    ks = []
    for _ in range(1000):
        st.run(5)
        ks.append(st.stats()["kT"])
    s = np.asarray(ks).reshape(20, -1).mean(1)
    m, err = s.mean(), s.std(ddof=1) / math.sqrt(20)
    print(f"mixture kT {m:.5f} +- {err:.5f}")
    assert abs(m - kT) <= 0.01 * kT + 3.0 * err
