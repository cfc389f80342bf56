"""The request loop (lfmm_server_*): results are the same alone and in the mix.

Requests of the serving stream (uniform and four-cluster point sets, N_tgt = N_src/4,
tolerance 1e-6 or 1e-10 each) are solved once through a one-slot server, one at a
time, and once all submitted together to a four-slot server, where they are admitted
as slots free up and overlap on the device.  Each result must agree between the two
runs within the request's own tolerance, and with the oracle on sampled targets.
"""
import numpy as np
import pytest

import oracle
from paper_1105_3505_gb300 import build, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lfmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1105_3505_gb300 import lfmm as m
    m.load()
    torch.cuda.init()
    return m


@pytest.fixture(scope="module")
def requests():
    return list(workloads.serve_stream(seed=4, n_requests=14, n_max=2e5))


def test_same_alone_and_in_the_mix(lfmm, requests):
    with lfmm.Server(n_slots=1) as sv:
        alone = []
        for r in requests:
            t = sv.submit(r.problem.src, r.problem.tgt, r.problem.f, r.tol)
            alone.append(sv.wait(t))
    with lfmm.Server(n_slots=4) as sv:
        tickets = [sv.submit(r.problem.src, r.problem.tgt, r.problem.f, r.tol) for r in requests]
        mixed = [sv.wait(t) for t in tickets]
    for r, (ua, sa), (um, sm) in zip(requests, alone, mixed):
        assert sa["status"] == 0 and sm["status"] == 0
        want = lfmm.LFMM_MIXED if r.tol >= 1e-6 else lfmm.LFMM_DF
        assert sa["precision"] == want and sm["precision"] == want
        assert 0.0 <= sm["queue_ms"] and 0.0 < sm["run_ms"] <= sm["total_ms"] + 1e-9
        scale = np.abs(ua).max()
        assert np.abs(ua - um).max() <= r.tol * scale, (r.index, r.tol, np.abs(ua - um).max() / scale)
        idx = np.random.default_rng(r.index).choice(r.problem.tgt.shape[0], min(64, r.problem.tgt.shape[0]),
                                                    replace=False)
        ref = oracle.lattice_sum(r.problem.src, r.problem.f, r.problem.tgt[idx])
        err = np.abs(um[idx] - ref).max() / np.abs(ref).max()
        assert err <= r.tol, (r.index, r.problem.src.shape[0], r.tol, err)


def test_budget_limits_concurrency(lfmm, requests):
    """A budget smaller than two requests admits one at a time (queueing shows up in the
    stats), yet every request completes correctly."""
    small = [r for r in requests if r.problem.src.shape[0] < 60000][:4]
    with lfmm.Server(n_slots=4, hbm_budget_bytes=1) as sv:
        tickets = [sv.submit(r.problem.src, r.problem.tgt, r.problem.f, r.tol) for r in small]
        out = [sv.wait(t) for t in tickets]
    assert all(s["status"] == 0 for _, s in out)
    # one at a time: every request after the first waited in the queue
    assert all(s["queue_ms"] > 0.0 for _, s in out[1:])
    for r, (u, _) in zip(small, out):
        idx = np.arange(min(32, r.problem.tgt.shape[0]))
        ref = oracle.lattice_sum(r.problem.src, r.problem.f, r.problem.tgt[idx])
        assert np.abs(u[idx] - ref).max() <= r.tol * np.abs(ref).max()
