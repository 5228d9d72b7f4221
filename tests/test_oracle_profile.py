"""Pin of the oracle's velocity profile (Sec. 4.2: the flow velocity against
the coordinate across the flow): the mean flow-axis velocity in nbins equal
slabs along the gradient axis, on hand-built states whose expected bin means
are worked out by hand.  Slab k holds k Lg/nbins <= x_g < (k+1) Lg/nbins;
the faces used are dyadic, so the boundary cases are exact."""

import numpy as np

import oracle as O


def _profile(L, grad, flow, x, v, nbins):
    p = O.Params(L=L, fb_mode=O.FB_POISEUILLE, fb_flow=flow, fb_grad=grad)
    st = O.State.__new__(O.State)      # no forces needed: profile reads x and v only
    st.p, st.x, st.v, st.n = p, np.asarray(x, float), np.asarray(v, float), len(x)
    return st.profile(nbins)


def test_profile_slabs_along_y_of_a_non_integer_box():
    # gradient axis y (Ly = 7.5, 4 slabs, faces 1.875, 3.75, 5.625), flow axis x
    ys = [0.0, 1.875, 1.8749, 3.75, 7.4999, 5.625, 5.0]
    vx = [1.0, 2.0, 3.0, -1.0, 4.0, -2.0, 0.5]
    x = [[0.3 + 0.6 * k, y, 5.9 - 0.7 * k] for k, y in enumerate(ys)]
    v = [[u, 10.0 + k, -10.0 - k] for k, u in enumerate(vx)]
    prof, cnt = _profile((5.0, 7.5, 6.0), 1, 0, x, v, 4)
    assert cnt.tolist() == [2, 1, 2, 2]
    assert prof.tolist() == [2.0, 2.0, -0.25, 1.0]


def test_profile_axes_and_empty_slabs():
    # gradient axis z (Lz = 10, 5 slabs of 2), flow axis y; slab 1 stays empty
    zs = [0.5, 9.99, 4.0, 5.5, 8.0]
    vy = [-3.0, 6.0, 1.0, 2.0, 4.0]
    x = [[1.0, 9.0 - k, z] for k, z in enumerate(zs)]
    v = [[7.0 + k, u, -5.0] for k, u in enumerate(vy)]
    prof, cnt = _profile((3.0, 12.0, 10.0), 2, 1, x, v, 5)
    assert cnt.tolist() == [1, 0, 2, 0, 2]
    assert prof.tolist() == [-3.0, 0.0, 1.5, 0.0, 5.0]
