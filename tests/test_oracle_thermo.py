"""Statistical pins for the oracle: thermostat and equation of state.

* Fluctuation-dissipation (Sec. 2.1): with sigma^2 = 2 gamma kT and
  w_D = w_R^2 the fluid equilibrates at the target kT, for any gamma.
* Pressure: the virial route p = rho kT + sum_{i<j} r_ij . F^C_ij / (3V).  When
  a / kT -> 0 the pair correlation g(r) -> 1 and the excess pressure tends to
  the closed form (2 pi / 3) rho^2 int_0^1 r^3 a (1 - r) dr = (pi / 30) a rho^2.
* The Groot-Warren fit p = rho kT + 0.101 a rho^2 is the dense-fluid
  asymptote of the same quantity: the excess coefficient approaches it from
  below as rho grows (measured values are recorded in the test output).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04712_gb300.workloads import uniform_box_state


def _block_mean(samples, nblock=20):
    s = np.asarray(samples)
    s = s[: len(s) // nblock * nblock].reshape(nblock, -1).mean(1)
    return s.mean(), s.std(ddof=1) / math.sqrt(nblock)


@pytest.mark.parametrize("gamma,kT,a", [(4.5, 1.0, 25.0), (2.0, 0.5, 15.0)])
def test_thermostat_reaches_target_temperature(gamma, kT, a):
    L, dt = 6, 0.005
    x, v = uniform_box_state(L, rho=3, kT=kT, seed=21)
    p = O.Params(L=(L, L, L), a=a, gamma=gamma, kT=kT, dt=dt, seed=17)
    s = O.State(p, x, v, mode=O.MODE_CELLS)
    s.run(600)
    samples = []
    for _ in range(1200):
        s.run(5)
        samples.append(s.stats()["kT"])
    m, err = _block_mean(samples)
    print(f"kT target {kT}: measured {m:.5f} +- {err:.5f}")
    assert abs(m - kT) <= 0.01 * kT + 3.0 * err


def test_pressure_mean_field_closed_form():
    L, rho, a, kT = 8, 3, 25.0, 1000.0
    x, v = uniform_box_state(L, rho=rho, kT=kT, seed=2)
    p = O.Params(L=(L, L, L), a=a, gamma=4.5, kT=kT, dt=0.0003, seed=3)
    s = O.State(p, x, v, mode=O.MODE_CELLS)
    s.run(300)
    al = []
    for _ in range(250):
        s.run(5)
        al.append(s.virial / (3.0 * L ** 3) / (a * rho ** 2))
    m, err = _block_mean(al, 10)
    print(f"excess coefficient at a/kT = {a / kT}: {m:.6f} +- {err:.6f} (pi/30 = {math.pi / 30:.6f})")
    assert abs(m - math.pi / 30.0) <= 0.005 * math.pi / 30.0 + 3.0 * err


@pytest.mark.slow
def test_pressure_approaches_groot_warren_fit():
    a, kT, L = 25.0, 1.0, 8
    coeffs, devs = [], []
    for rho in (3, 4, 5):
        x, v = uniform_box_state(L, rho=rho, seed=1)
        p = O.Params(L=(L, L, L), a=a, gamma=4.5, kT=kT, dt=0.005, seed=7)
        s = O.State(p, x, v, mode=O.MODE_CELLS)
        s.run(400)
        ps = []
        for _ in range(300):
            s.run(5)
            ps.append(s.stats()["pressure"])
        m, err = _block_mean(ps, 10)
        fit = rho * kT + 0.101 * a * rho ** 2
        coeffs.append((m - rho * kT) / (a * rho ** 2))
        devs.append(m / fit - 1.0)
        print(f"rho {rho}: p = {m:.3f} +- {err:.3f}, Groot-Warren fit {fit:.3f}, "
              f"deviation {100 * devs[-1]:+.2f}%")
    # excess coefficient grows with density, toward (and below) the mean-field pi/30
    assert coeffs[0] < coeffs[1] < coeffs[2] < math.pi / 30
    # ... and the distance to the 0.101 fit shrinks with density
    assert abs(devs[0]) > abs(devs[1]) > abs(devs[2])
    assert all(abs(d) < 0.10 for d in devs)


def test_thermostat_with_gaussian_noise():
    L, dt, kT = 6, 0.005, 1.0
    x, v = uniform_box_state(L, rho=3, kT=kT, seed=23)
    p = O.Params(L=(L, L, L), a=25.0, gamma=4.5, kT=kT, dt=dt, seed=19, noise=1)
    s = O.State(p, x, v, mode=O.MODE_CELLS)
    s.run(600)
    samples = []
    for _ in range(1200):
        s.run(5)
        samples.append(s.stats()["kT"])
    m, err = _block_mean(samples)
    print(f"Gaussian noise: kT {m:.5f} +- {err:.5f}")
    assert abs(m - kT) <= 0.01 * kT + 3.0 * err
