"""Served form: continuous batching of independent runs."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1911_04712_gb300 import build
    build.build()
    import paper_1911_04712_gb300.serve as S
    return S


def _reqs(S, k0, count):
    rng = np.random.default_rng(k0)
    out = []
    for k in range(count):
        out.append(S.make_request(float(rng.integers(4, 9)), rho=float(rng.choice([3, 5])),
                                  a=float(rng.uniform(10, 80)), gamma=float(rng.uniform(2, 8)),
                                  kT=float(rng.uniform(0.5, 2)), seed=k0 * 1000 + k,
                                  steps=int(rng.integers(60, 400))))
    return out


def test_results_identical_alone_and_in_the_mix(S):
    target = S.make_request(6.0, rho=4, a=30.0, gamma=5.0, kT=1.2, seed=4242, steps=340)
    q1 = S.Queue(1 << 30, chunk_steps=50, sample_every=10, nbins=8)
    t = q1.submit(target)
    q1.wait_all(300)
    alone = q1.result(t)
    q1.close()
    # in a mix: other runs before and after it, few resident slots, short chunks
    q2 = S.Queue(1 << 30, max_boxes=3, chunk_steps=37, sample_every=10, nbins=8)
    before = [q2.submit(r) for r in _reqs(S, 1, 5)]
    t2 = q2.submit(target)
    after = [q2.submit(r) for r in _reqs(S, 2, 4)]
    q2.wait_all(300)
    mixed = q2.result(t2)
    assert alone["status"] == 0 and mixed["status"] == 0
    assert alone["samples"] == mixed["samples"] == 340 // 2 // 10
    assert mixed["kT_mean"] == pytest.approx(alone["kT_mean"], rel=1e-12, abs=0)
    assert mixed["pressure_mean"] == pytest.approx(alone["pressure_mean"], rel=1e-12, abs=0)
    np.testing.assert_allclose(mixed["profile"], alone["profile"], rtol=1e-9, atol=1e-12)
    for tk in before + after:
        r = q2.result(tk)
        assert r["status"] == 0 and r["t_admit"] >= r["t_submit"] and r["t_done"] >= r["t_admit"]
    st = q2.stats()
    assert st["completed"] == 10 and st["pending"] == 0 and st["bytes_in_use"] == 0
    q2.close()


def test_thermostat_holds_target_temperature(S):
    q = S.Queue(1 << 30, chunk_steps=100, sample_every=5)
    ts = [q.submit(S.make_request(8.0, rho=3, kT=kT, seed=7 + i, steps=1200))
          for i, kT in enumerate((0.5, 1.0, 2.0))]
    q.wait_all(300)
    for t, kT in zip(ts, (0.5, 1.0, 2.0)):
        r = q.result(t)
        assert abs(r["kT_mean"] / kT - 1) < 0.05, r["kT_mean"]
        assert r["pressure_mean"] > 0
    q.close()


def test_poiseuille_profile_follows_the_force(S):
    q = S.Queue(1 << 30, chunk_steps=100, sample_every=10, nbins=8)
    t = q.submit(S.make_request(8.0, rho=3, seed=3, steps=1600, body_force=0.5, body_mode=2,
                                flow_axis=2, grad_axis=0))
    q.wait_all(300)
    prof = q.result(t)["profile"]
    assert prof[:4].mean() < -0.05 and prof[4:].mean() > 0.05   # -f below L/2, +f above
    q.close()


def test_budget_and_cancel(S):
    D = pytest.importorskip("paper_1911_04712_gb300.dpd")
    q = S.Queue(4 << 20, max_boxes=1, chunk_steps=50)
    with pytest.raises(D.DPDError) as ei:
        q.submit(S.make_request(40.0, rho=3, steps=10))      # ~17 MB > 4 MB budget
    assert ei.value.code == D.ERR_NOMEM
    a = q.submit(S.make_request(5.0, rho=3, seed=1, steps=3000))
    b = q.submit(S.make_request(5.0, rho=3, seed=2, steps=100))
    q.cancel(b)                                               # still waiting: ends at once
    assert q.done(b) and q.result(b)["status"] == D.ERR_STATE
    q.cancel(a)
    q.wait_all(120)
    assert q.result(a)["status"] == D.ERR_STATE
    with pytest.raises(D.DPDError):
        q.result(12345)
    q.close()


def test_bounded_wait_reports_timeout(S):
    """A chunk wait limit shorter than the chunk: the queue reports
    DPD_ERR_TIMEOUT for its runs (the GPU work itself completes normally)."""
    D = pytest.importorskip("paper_1911_04712_gb300.dpd")
    q = S.Queue(1 << 30, chunk_steps=100, chunk_timeout_s=1e-7)
    t = q.submit(S.make_request(32.0, rho=3, seed=1, steps=400))
    with pytest.raises(D.DPDError) as ei:
        q.wait_all(120)
    assert ei.value.code == D.ERR_TIMEOUT
    assert q.result(t)["status"] == D.ERR_TIMEOUT
    with pytest.raises(D.DPDError):
        q.submit(S.make_request(8.0, rho=3, steps=10))
    q.close()


def test_admission_respects_the_packed_set_capacity(S):
    """Two runs that each fit one packed set but not together (2 x 4.1e7
    particles against 2^26 particle slots) are admitted one after the other
    and both complete, under a budget that would hold both."""
    q = S.Queue(int(100e9), chunk_steps=2, stencil=1)
    t = [q.submit(S.make_request(240.0, rho=3.0, seed=70 + k, steps=2)) for k in range(2)]
    q.wait_all(600.0)
    r = [q.result(x) for x in t]
    q.close()
    assert all(x["status"] == 0 for x in r), r
    assert all(x["n"] == 41472000 for x in r)
    first, second = sorted(r, key=lambda x: x["t_admit"])
    assert second["t_admit"] >= first["t_done"] - 1e-6


def _oracle_params(L, seed, fb):
    import oracle as O
    return O.Params(L=(L, L, L), a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=seed,
                    fb=fb, fb_mode=O.FB_POISEUILLE, fb_flow=0, fb_grad=1)


def _near_face_counts(y, L, nbins, tol):
    """Per slab: particles within tol (in slab widths) of one of its faces."""
    u = np.asarray(y, np.float64) / L * nbins
    k = np.round(u).astype(int)
    hit = np.abs(u - k) < tol
    c = np.zeros(nbins)
    np.add.at(c, k[hit] % nbins, 1)          # the slab above the face
    np.add.at(c, (k[hit] - 1) % nbins, 1)    # the slab below
    return c


def test_served_run_matches_the_oracle(S):
    """A run given its initial state, stepped inside a mix with short chunks
    and repacks (three resident slots, other runs admitted and retired around
    it), against the FP64 oracle run from the same state: the sampled mean
    kT and pressure, the slab profile of the flow velocity (Sec. 4.2), and
    the final state (within 1e-3 rc)."""
    import oracle as O
    from paper_1911_04712_gb300.workloads import uniform_box_state
    L, seed, fb = 8.0, 11, 0.3
    steps, every, nbins = 60, 10, 8
    x0, v0 = uniform_box_state(L, rho=3, seed=seed)
    n = len(x0)
    req = S.make_request(L, n=n, a=25.0, gamma=4.5, kT=1.0, seed=seed, steps=steps,
                         body_force=fb, body_mode=2, flow_axis=0, grad_axis=1)
    q = S.Queue(1 << 30, max_boxes=3, chunk_steps=7, sample_every=every, nbins=nbins)
    others = [q.submit(r) for r in _reqs(S, 3, 3)]
    t = q.submit_state(req, x0, v0, keep_final=True)
    others += [q.submit(r) for r in _reqs(S, 4, 3)]
    q.wait_all(300)
    got = q.result(t)
    xg, vg = q.final_state(t, n)
    assert all(q.result(k)["status"] == 0 for k in others)
    q.close()
    assert got["status"] == 0 and got["samples"] == 3      # steps 40, 50, 60

    st = O.State(_oracle_params(L, seed, fb), x0, v0)
    kts, prs, sums, cnts = [], [], np.zeros(nbins), np.zeros(nbins)
    near = np.zeros(nbins)     # particles near a slab face at a sample, per adjacent slab
    for s in range(every, steps + 1, every):
        st.run(every)
        if s > steps // 2:
            d = st.stats()
            kts.append(d["kT"])
            prs.append(d["pressure"])
            prof, cnt = st.profile(nbins)
            sums += prof * cnt
            cnts += cnt
            near += _near_face_counts(st.x[:, 1], L, nbins, 1e-4)
    assert got["kT_mean"] == pytest.approx(np.mean(kts), rel=1e-4)
    assert got["pressure_mean"] == pytest.approx(np.mean(prs), rel=1e-4)
    # the FP32 and FP64 trajectories differ by ~1e-6 rc here: a particle within
    # 1e-4 of a face may sit in either slab, which moves a pooled slab mean by
    # at most 2 max|v| / count; every other difference must be round-off
    allow = 1e-3 + near * 2.0 * np.abs(st.v[:, 0]).max() * 1.5 / cnts
    assert np.all(np.abs(got["profile"] - sums / cnts) <= allow), (got["profile"], sums / cnts)
    assert (near == 0).sum() >= nbins // 2
    d = xg.astype(np.float64) - st.x
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-3
    assert np.abs(vg.astype(np.float64) - st.v).max() < 1e-2


def test_served_profile_bins_equal_the_oracle_on_the_sampled_state(S):
    """One sample taken at the last step, whose state is read back: the
    device's slab sums (k_sample) and kT against the oracle's profile and
    statistics on that same state, bin by bin."""
    import oracle as O
    from paper_1911_04712_gb300.workloads import uniform_box_state
    L, seed, fb, nbins = 7.5, 5, 0.2, 6
    x0, v0 = uniform_box_state(L, rho=3, seed=seed)
    n = len(x0)
    req = S.make_request(L, n=n, seed=seed, steps=2, body_force=fb, body_mode=2,
                         flow_axis=0, grad_axis=1)
    q = S.Queue(1 << 30, chunk_steps=100, sample_every=1, nbins=nbins)
    t = q.submit_state(req, x0, v0, keep_final=True)
    q.wait_all(120)
    got = q.result(t)
    xg, vg = q.final_state(t, n)
    q.close()
    assert got["samples"] == 1
    p = O.Params(L=(L, L, L), seed=seed, fb=fb, fb_mode=O.FB_POISEUILLE, fb_flow=0, fb_grad=1)
    st = O.State(p, xg, vg)
    prof, cnt = st.profile(nbins)
    # the device bins in FP32: only a particle within ~1e-6 of a face can differ
    near = _near_face_counts(xg[:, 1], L, nbins, 1e-5)
    allow = 1e-12 + near * 2.0 * np.abs(vg[:, 0]).max() * 1.5 / cnt
    assert np.all(np.abs(got["profile"] - prof) <= allow), (got["profile"], prof)
    assert got["kT_mean"] == pytest.approx(st.stats()["kT"], rel=1e-12)
