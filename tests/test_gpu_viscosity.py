"""Viscosity of the DPD fluid against Table 1 of the paper.

Table 1 lists, for several parameter sets, the viscosity the authors
measured (in a pipe).  Viscosity is a bulk property, so it is measured here
by periodic Poiseuille flow (Sec. 4.2): with a force -f along x where
y <= L/2 and +f above, the steady profile is v_x(y) = -rho f y (L/2 - y) /
(2 eta) on [0, L/2] (mirrored above).  The fitted eta must fall within 5 %
of the middle of the range the paper measured.
"""

import numpy as np
import pytest

from paper_1911_04712_gb300.workloads import uniform_box_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpd():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.dpd as d
    return d


def _shape(y, L):
    """Profile shape for unit rho f / (2 eta): -y(L/2 - y) below L/2, mirrored above."""
    h = L / 2
    return np.where(y <= h, -y * (h - y), (y - h) * (L - y))


# (a, gamma, rho, k, kT, dt) and the range of eta the paper measured
TABLE1 = [
    ((25.0, 6.75, 3, 1.0, 1.0, 0.04), (0.89, 0.90)),
    ((18.75, 4.5, 4, 1.0, 1.0, 0.005), (1.07, 1.08)),
    ((18.75, 4.5, 4, 0.25, 1.0, 0.005), (2.44, 2.45)),
    ((0.0, 20.25, 6, 1.0, 0.5, 0.01), (2.08, 2.10)),
]


@pytest.mark.parametrize("params,eta_range", TABLE1)
def test_viscosity_matches_table1(dpd, params, eta_range):
    a, gamma, rho, k, kT, dt = params
    L, nb = 16.0, 16
    eta_guess = sum(eta_range) / 2
    f = 2 * eta_guess * 0.4 / (rho * (L / 4) ** 2)           # peak velocity ~0.4
    x, v = uniform_box_state(L, rho=rho, kT=kT, seed=17)
    box = dpd.Box(L, a=a, gamma=gamma, kT=kT, rc=1.0, dt=dt, seed=17, kexp=k)
    box.set_param(dpd.PARAM_FLOW_AXIS, 0)
    box.set_param(dpd.PARAM_GRAD_AXIS, 1)
    box.set_param(dpd.PARAM_POISEUILLE_F, f)
    box.set_state(x, v)
    nu = eta_guess / rho
    t_relax = (L / (2 * np.pi)) ** 2 / nu                     # slowest mode of the profile
    box.step(int(6 * t_relax / dt))
    every = max(1, int(0.5 / dt))
    prof = np.zeros(nb)
    cnt = np.zeros(nb)
    nsamp = int(40 * t_relax / dt) // every
    for _ in range(nsamp):
        box.step(every)
        xg, vg = box.get_state()
        b = np.clip((xg[:, 1] / L * nb).astype(int), 0, nb - 1)
        prof += np.bincount(b, weights=vg[:, 0].astype(np.float64), minlength=nb)
        cnt += np.bincount(b, minlength=nb)
    prof /= cnt
    yc = (np.arange(nb) + 0.5) * L / nb
    g = _shape(yc, L)
    c = (g * prof).sum() / (g * g).sum()                      # v = c g, c = rho f / (2 eta)
    eta = rho * f / (2 * c)
    mid = sum(eta_range) / 2
    print(f"a={a} gamma={gamma} rho={rho} k={k} kT={kT} dt={dt}: eta = {eta:.4f} "
          f"(paper {eta_range[0]}-{eta_range[1]})")
    assert abs(eta / mid - 1) < 0.05, eta
