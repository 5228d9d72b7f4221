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
