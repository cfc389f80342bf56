"""Failure handling without a GPU fault.

Every failure here is made on the host or by a bounded wait that is told to give up:
  - allocation failures: lfmm_fault_inject_alloc makes the n-th device allocation fail
    as a full device would; the call reports LFMM_ENOMEM and the memory pool is back to
    where it was (nothing leaked), for every n up to the call's allocation count;
  - device waits: a barrier-stall hook sets a grid barrier's arrival count out of reach
    (as if blocks never arrived), and a one-poll budget makes the tensor-core pipeline's
    mbarrier waits give up; the plan reports LFMM_ETIMEOUT through lfmm_plan_status, which puts
    the barrier words back, and the next evaluation is bit-identical to one made before;
  - the server's overload policy: a bounded queue refuses with LFMM_EBUSY, a latency
    budget sheds waiting requests with LFMM_EBUSY, and a queued request can be cancelled
    (LFMM_ECANCELED) while the others complete correctly.
No kernel traps, faults or spins without a bound.
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


def _pool_settled(lfmm):
    torch.cuda.synchronize()
    return lfmm.lfmm_pool_used_bytes()


def _inject_until_success(lfmm, call, max_n=200):
    """Runs call() with the n-th allocation failing for n = 1, 2, ... until it succeeds;
    every failing run must report LFMM_ENOMEM and leave the pool as it found it."""
    base = _pool_settled(lfmm)
    for n in range(1, max_n):
        lfmm.lfmm_fault_inject_alloc(n)
        try:
            res = call()
        except lfmm.LfmmError as e:
            assert e.status == lfmm.LFMM_ENOMEM, (n, str(e))
            assert _pool_settled(lfmm) == base, n
            continue
        finally:
            lfmm.lfmm_fault_inject_alloc(0)
        return n, res
    raise AssertionError("call never succeeded")


def test_alloc_failure_plan_create_no_leak(lfmm):
    prob = workloads.uniform_box(20000, 15000, 700, seed=61)
    for prec, p in [(lfmm.LFMM_MIXED, 8), (lfmm.LFMM_DF, 16)]:
        opts = lfmm.make_opts(prec, p, tc_min_level=3)
        base = _pool_settled(lfmm)
        n, h = _inject_until_success(lfmm, lambda: lfmm.lfmm_plan_create(prob.src, prob.src.shape[0], prob.tgt,
                                                                          prob.tgt.shape[0], opts, None))
        assert n > 3  # plan creation makes several allocations, each one failed once
        u = np.empty(prob.tgt.shape[0])
        lfmm.lfmm_eval(h, prob.f, u, None)
        lfmm.lfmm_plan_destroy(h)
        assert _pool_settled(lfmm) == base
        idx = np.arange(0, prob.tgt.shape[0], 97)
        ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
        assert np.abs(u[idx] - ref).max() <= (1e-6 if prec == lfmm.LFMM_MIXED else 1e-10) * np.abs(ref).max()


def test_alloc_failure_eval_solve_forest_no_leak(lfmm):
    prob = workloads.uniform_box(8000, 6000, 500, seed=62)
    base = _pool_settled(lfmm)
    # host f and u are staged through buffers the plan allocates at its first evaluation;
    # those belong to the plan, so the pool is checked after the plan is destroyed
    u = np.empty(prob.tgt.shape[0])
    for n in range(1, 50):
        h = lfmm.lfmm_plan_create(prob.src, prob.src.shape[0], prob.tgt, prob.tgt.shape[0], lfmm.make_opts(), None)
        lfmm.lfmm_fault_inject_alloc(n)
        try:
            lfmm.lfmm_eval(h, prob.f, u, None)
            ok = True
        except lfmm.LfmmError as e:
            assert e.status == lfmm.LFMM_ENOMEM
            ok = False
        finally:
            lfmm.lfmm_fault_inject_alloc(0)
            lfmm.lfmm_plan_destroy(h)
        assert _pool_settled(lfmm) == base, n
        if ok:
            assert n > 1
            break
    # one-shot solve
    u2 = np.empty(prob.tgt.shape[0])
    _inject_until_success(lfmm, lambda: lfmm.lfmm_solve(prob.src, prob.tgt, prob.f, u2, lfmm.make_opts(), None))
    assert np.abs(u2 - u).max() <= 1e-6 * np.abs(u).max()
    # forest of three problems
    src = np.ascontiguousarray(np.concatenate([prob.src[:3000], prob.src[3000:5000] + 10 ** 6, prob.src[5000:]]))
    off = np.array([0, 3000, 5000, 8000], dtype=np.int64)
    n, hf = _inject_until_success(lfmm, lambda: lfmm.lfmm_forest_create(src, off, src, off, lfmm.make_opts(), None))
    assert n > 3
    lfmm.lfmm_plan_destroy(hf)
    assert _pool_settled(lfmm) == base


def _eval_dev(lfmm, h, f, nt):
    u = torch.empty(nt, dtype=torch.float64, device="cuda")
    lfmm.lfmm_eval(h, f, u, None)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("precision", ["mixed", "df"])
def test_grid_barrier_stall_times_out_and_recovers(lfmm, precision):
    """A grid barrier whose count is out of reach is never released: with a budget of
    2,000 polls every block gives up, the evaluation reports LFMM_ETIMEOUT, and after
    lfmm_plan_status the plan's next evaluation equals one made before the stall."""
    prob = workloads.uniform_box(60000, 60000, 1200, seed=63)
    prec, p = (lfmm.LFMM_MIXED, 8) if precision == "mixed" else (lfmm.LFMM_DF, 16)
    dev = torch.device("cuda:0")
    s, t, f = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    # uniform storage: its coarse levels run in the cooperative kernels with grid barriers
    h = lfmm.lfmm_plan_create(s, s.shape[0], t, t.shape[0], lfmm.make_opts(prec, p, tree=lfmm.LFMM_TREE_UNIFORM),
                              None)
    try:
        assert lfmm.lfmm_plan_get_info(h)["L"] >= 4
        u0 = _eval_dev(lfmm, h, f, t.shape[0])
        lfmm.lfmm_plan_status(h)  # clean
        lfmm.lfmm_plan_set_wait_budget(h, 2000)
        lfmm.lfmm_plan_inject_barrier_stall(h)
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            _eval_dev(lfmm, h, f, t.shape[0])
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        assert prof["m2m"][1] == 1  # the cooperative M2M kernel (all levels, grid barriers between)
        with pytest.raises(lfmm.LfmmError) as ei:
            lfmm.lfmm_plan_status(h)
        assert ei.value.status == lfmm.LFMM_ETIMEOUT
        lfmm.lfmm_plan_set_wait_budget(h, 0)
        u1 = _eval_dev(lfmm, h, f, t.shape[0])
        lfmm.lfmm_plan_status(h)  # the barrier words were put back
        assert np.array_equal(u0, u1)
    finally:
        lfmm.lfmm_plan_destroy(h)


def test_tensor_core_wait_budget_times_out_and_recovers(lfmm):
    """One poll per mbarrier wait: the tensor-core M2L pipeline gives up at its first
    wait for a TMA load, stops every role, waits (with the default bound) for the copies
    and products it issued, frees its tensor memory and exits; the plan reports
    LFMM_ETIMEOUT and evaluates normally afterwards.  Two tree levels with the tensor
    cores from level 2: no cooperative kernel (hence no grid barrier) runs, so the
    timeout can only come from the tensor-core pipeline."""
    prob = workloads.uniform_box(400, 400, 128, seed=64)
    dev = torch.device("cuda:0")
    s, t, f = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    h = lfmm.lfmm_plan_create(s, s.shape[0], t, t.shape[0], lfmm.make_opts(lfmm.LFMM_MIXED, 8, tc_min_level=2), None)
    try:
        assert lfmm.lfmm_plan_get_info(h)["L"] == 2
        u0 = _eval_dev(lfmm, h, f, t.shape[0])
        ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
        assert np.abs(u0 - ref).max() <= 1e-6 * np.abs(ref).max()
        lfmm.lfmm_plan_status(h)
        lfmm.lfmm_plan_set_wait_budget(h, 1)
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            _eval_dev(lfmm, h, f, t.shape[0])
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        assert prof["m2l_tc"][1] > 0  # the tensor-core levels ran
        with pytest.raises(lfmm.LfmmError) as ei:
            lfmm.lfmm_plan_status(h)
        assert ei.value.status == lfmm.LFMM_ETIMEOUT
        lfmm.lfmm_plan_set_wait_budget(h, 0)
        for _ in range(2):
            u1 = _eval_dev(lfmm, h, f, t.shape[0])
            lfmm.lfmm_plan_status(h)
            assert np.array_equal(u0, u1)
    finally:
        lfmm.lfmm_plan_destroy(h)


def test_tensor_core_list_wait_budget_times_out_and_recovers(lfmm):
    """The same for the tensor-core list M2L of a forest (four gathering producer warps):
    with one poll per wait it gives up, the producers announce what they issued, the
    teardown completes the stages some producers skipped and waits for every copy and
    product in flight before freeing tensor memory; the plan reports LFMM_ETIMEOUT and
    evaluates as before.  Forest evaluation runs one launch per level, so no grid
    barrier can time out."""
    rng = np.random.default_rng(65)
    srcs, fs = [], []
    for i in range(48):
        n = int(rng.integers(300, 3000))
        r = np.random.default_rng([65, i])
        srcs.append(workloads.distinct_in_box(r, n, int(np.ceil(4 * np.sqrt(n))), int(r.integers(-9000, 9000)), 0))
        fs.append(workloads.zero_sum(r.standard_normal(n)))
    src = np.ascontiguousarray(np.concatenate(srcs).astype(np.int32))
    off = np.concatenate([[0], np.cumsum([a.shape[0] for a in srcs])]).astype(np.int64)
    f = np.concatenate(fs)
    with lfmm.Forest(src, off, src, off, precision=lfmm.LFMM_MIXED, p=8) as fo:
        u0 = fo.eval(f)
        fo.status()
        lfmm.lfmm_plan_set_wait_budget(fo.handle, 1)
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            fo.eval(f)
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        assert prof["m2l_tc"][1] > 0  # the tensor-core list levels ran
        with pytest.raises(lfmm.LfmmError) as ei:
            fo.status()
        assert ei.value.status == lfmm.LFMM_ETIMEOUT
        lfmm.lfmm_plan_set_wait_budget(fo.handle, 0)
        for _ in range(2):
            u1 = fo.eval(f)
            fo.status()
            assert np.array_equal(u0, u1)
    ref = oracle.lattice_sum(srcs[5], fs[5], srcs[5])
    u5 = u0[off[5]:off[6]]
    assert np.abs(u5 - ref).max() <= 1e-6 * np.abs(ref).max()


def test_server_overload_policy_and_cancel(lfmm):
    """One slot, so requests queue behind the one running: a bounded queue refuses the
    excess at submit, a latency budget of 0.01 ms sheds whatever waits, cancel removes a
    waiting request; every request that runs matches the oracle."""
    reqs = [workloads.uniform_box(40000, 10000, 900, seed=70 + i) for i in range(6)]
    with lfmm.Server(n_slots=1) as sv:
        sv.set_limits(max_pending=2)
        tickets, refused = [], 0
        for r in reqs:
            try:
                tickets.append((r, sv.submit(r.src, r.tgt, r.f, 1e-6)))
            except lfmm.LfmmError as e:
                assert e.status == lfmm.LFMM_EBUSY
                refused += 1
        assert refused >= 1 and len(tickets) >= 2
        # cancel the last queued request (the first may already run)
        r_c, t_c = tickets[-1]
        try:
            sv.cancel(t_c)
            cancelled = True
        except lfmm.LfmmError as e:
            assert e.status == lfmm.LFMM_EINVAL  # it was admitted in the meantime
            cancelled = False
        for r, t in tickets:
            u, st = sv.wait_stats(t)
            if t == t_c and cancelled:
                assert st["status"] == lfmm.LFMM_ECANCELED and u is None
                continue
            assert st["status"] == lfmm.LFMM_OK
            idx = np.arange(0, r.tgt.shape[0], 211)
            ref = oracle.lattice_sum(r.src, r.f, r.tgt[idx])
            assert np.abs(u[idx] - ref).max() <= 1e-6 * np.abs(ref).max()
        # latency budget of 0.01 ms: a request is refused at submit once the run times
        # measured so far predict a longer wait, and whatever waits longer is shed
        sv.set_limits(max_pending=0, max_queue_ms=0.01)
        tickets, refused = [], 0
        for r in reqs:
            try:
                tickets.append(sv.submit(r.src, r.tgt, r.f, 1e-6))
            except lfmm.LfmmError as e:
                assert e.status == lfmm.LFMM_EBUSY and "predicted wait" in str(e)
                refused += 1
        stats = [sv.wait_stats(t)[1] for t in tickets]
        codes = [s["status"] for s in stats]
        assert refused + codes.count(lfmm.LFMM_EBUSY) >= 1 and refused < len(reqs)
        assert set(codes) <= {lfmm.LFMM_OK, lfmm.LFMM_EBUSY}
        for s in stats:
            if s["status"] == lfmm.LFMM_EBUSY:
                assert s["run_ms"] == 0.0 and s["queue_ms"] > 0.01
        # limits off: every request is served again
        sv.set_limits(0, 0.0)
        u, st = sv.wait(sv.submit(reqs[0].src, reqs[0].tgt, reqs[0].f, 1e-6))
        assert st["status"] == lfmm.LFMM_OK
