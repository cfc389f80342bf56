"""Evaluation through a recorded CUDA graph (LFMM_FLAG_GRAPH).

The graph replays exactly the launches of the eager evaluation of the same plan, and
no kernel of the evaluation uses atomics, so its results must be bit-identical to the
eager ones (lfmm_plan_set_flags switches one plan between the two): on the first call (record + launch), on replays with
the same pointers, after new pointers force a re-record, for host-staged arrays, and
for forests.  Two plans built from the same points may order the points of a leaf
differently (the bucket ranks come from atomics), so across plans the results agree
to rounding only.  One sampled check ties the graph path to the oracle directly.
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


def prec(lfmm, name):
    return {"fp64": (lfmm.LFMM_FP64, 16), "mixed": (lfmm.LFMM_MIXED, 8), "mixed16": (lfmm.LFMM_MIXED, 16),
            "df": (lfmm.LFMM_DF, 16)}[name]


def eager(lfmm, plan, f, parts=False):
    """The eager evaluation of a graph plan (graph flag cleared, then set again)."""
    plan.set_flags(graph=False)
    try:
        return plan.eval_parts(f) if parts else plan.eval(f)
    finally:
        plan.set_flags(graph=True)


@pytest.mark.parametrize("precision", ["mixed", "mixed16", "fp64", "df"])
def test_graph_equals_eager(lfmm, precision):
    prob = workloads.uniform_box(60000, 50000, 1024, seed=12)
    pr, p = prec(lfmm, precision)
    dev = torch.device("cuda:0")
    s_d, t_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt))
    f1 = torch.from_numpy(prob.f).to(dev)
    f2 = torch.from_numpy(workloads.zero_sum(np.random.default_rng(3).standard_normal(prob.f.shape[0]))).to(dev)
    with lfmm.Plan(s_d, t_d, precision=pr, p=p, graph=True) as g, lfmm.Plan(s_d, t_d, precision=pr, p=p) as other:
        assert g.info()["L"] >= 3  # deep enough for the fused and per-level far-field launches
        ue1, ue2 = eager(lfmm, g, f1), eager(lfmm, g, f2)
        out = torch.empty_like(ue1)
        for _ in range(3):  # record, then replays with the same pointers
            g.eval(f1, out)
            assert torch.equal(out, ue1)
        f1.copy_(f2)  # same pointer, new values: the replay reads them
        g.eval(f1, out)
        assert torch.equal(out, ue2)
        ug = g.eval(f2)  # new output pointer: re-recorded
        assert torch.equal(ug, ue2)
        uh = g.eval(prob.f)  # host arrays through the plan's staging buffers
        assert np.array_equal(uh, ue1.cpu().numpy())
        un, uf = g.eval_parts(f2)
        une, ufe = eager(lfmm, g, f2, parts=True)
        assert torch.equal(un, une) and torch.equal(uf, ufe)
        # another plan of the same points: equal to rounding
        uo = other.eval(f2)
        scale = float(ue2.abs().max())
        assert float((uo - ue2).abs().max()) <= (1e-6 if precision.startswith("mixed") else 1e-12) * scale
    idx = np.random.default_rng(1).choice(prob.tgt.shape[0], 48, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    err = np.abs(uh[idx] - ref).max() / np.abs(ref).max()
    assert err <= (1e-6 if precision.startswith("mixed") else 1e-10), err


def test_graph_forest_equals_eager(lfmm):
    rng = np.random.default_rng(8)
    srcs, fs = [], []
    for i in range(64):
        n = int(rng.integers(200, 3000))
        side = int(np.ceil(4 * np.sqrt(n)))
        r = np.random.default_rng([8, i])
        srcs.append(workloads.distinct_in_box(r, n, side, int(r.integers(-5000, 5000)), 0))
        fs.append(workloads.zero_sum(r.standard_normal(n)))
    src = np.ascontiguousarray(np.concatenate(srcs).astype(np.int32))
    off = np.concatenate([[0], np.cumsum([a.shape[0] for a in srcs])]).astype(np.int64)
    f = np.concatenate(fs)
    with lfmm.Forest(src, off, src, off, graph=True) as b:
        ua = eager(lfmm, b, f)
        for _ in range(2):
            assert np.array_equal(b.eval(f), ua)


def test_graph_with_profiling_runs_eager(lfmm):
    """While phase profiling is on, a graph plan evaluates eagerly (phases are timed)."""
    prob = workloads.uniform_box(8000, 8000, 400, seed=2)
    with lfmm.Plan(prob.src, prob.tgt, graph=True) as g:
        u0 = g.eval(prob.f)
        lfmm.lfmm_profile_enable(True)
        try:
            lfmm.lfmm_profile_read(reset=True)
            u1 = g.eval(prob.f)
            ph = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
    assert np.array_equal(u0, u1)
    assert ph["p2p"][1] >= 1 and ph["p2m"][1] >= 1


@pytest.mark.parametrize("precision", ["mixed", "df"])
def test_serial_equals_overlapped(lfmm, precision):
    """LFMM_FLAG_SERIAL runs the same kernels on one stream: bit-identical results."""
    prob = workloads.uniform_box(40000, 30000, 800, seed=13)
    pr, p = prec(lfmm, precision)
    with lfmm.Plan(prob.src, prob.tgt, precision=pr, p=p) as pl:
        u0 = pl.eval(prob.f)
        pl.set_flags(serial=True)
        u1 = pl.eval(prob.f)
        pl.set_flags(serial=True, graph=True)
        u2 = pl.eval(prob.f)
        pl.status()
    assert np.array_equal(u0, u1) and np.array_equal(u0, u2)


def test_solve_equals_plan_eval(lfmm):
    """lfmm_solve (one-shot, host inputs uploaded beside the tree build) gives the plan +
    eval result to rounding (its own plan may order a leaf's points differently), for
    host and device arrays, and meets the oracle."""
    prob = workloads.uniform_box(30000, 20000, 700, seed=14)
    with lfmm.Plan(prob.src, prob.tgt) as pl:
        u_ref = pl.eval(prob.f)
    u_h = np.empty(prob.tgt.shape[0])
    lfmm.lfmm_solve(prob.src, prob.tgt, prob.f, u_h, lfmm.make_opts())
    dev = torch.device("cuda:0")
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    u_d = torch.empty(prob.tgt.shape[0], dtype=torch.float64, device=dev)
    lfmm.lfmm_solve(s_d, t_d, f_d, u_d, lfmm.make_opts())
    torch.cuda.synchronize()
    scale = np.abs(u_ref).max()
    assert np.abs(u_h - u_ref).max() <= 1e-6 * scale
    assert np.abs(u_d.cpu().numpy() - u_ref).max() <= 1e-6 * scale
    idx = np.random.default_rng(5).choice(prob.tgt.shape[0], 48, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    assert np.abs(u_h[idx] - ref).max() <= 1e-6 * np.abs(ref).max()
