"""The autotuner (lfmm_autotune): the options it picks meet the requested accuracy
against the oracle, its own error estimate is honest, and the cache returns the same
choice without measuring."""
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
    m.tune_cache_clear()
    return m


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_autotune_meets_tolerance(lfmm, tol):
    prob = workloads.uniform_box(50000, 40000, 900, seed=21)
    opts, r = lfmm.autotune(prob.src, prob.tgt, tol)
    assert not r["from_cache"] and r["candidates"] >= 3
    assert r["precision"] == (lfmm.LFMM_MIXED if tol >= 1e-6 else lfmm.LFMM_DF)
    assert r["rel_err"] <= tol / 2 and r["ms"] > 0
    with lfmm.Plan(prob.src, prob.tgt, opts=opts) as pl:
        u = pl.eval(prob.f)
        pl.status()
    idx = np.random.default_rng(2).choice(prob.tgt.shape[0], 64, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    assert np.abs(u[idx] - ref).max() <= tol * np.abs(ref).max()
    # same size class and tolerance decade: cached
    prob2 = workloads.uniform_box(50000, 40000, 900, seed=22)
    opts2, r2 = lfmm.autotune(prob2.src, prob2.tgt, tol)
    assert r2["from_cache"] and r2["candidates"] == 0
    assert (opts2.p, opts2.leaf_size, opts2.tc_min_level, opts2.precision) == \
        (opts.p, opts.leaf_size, opts.tc_min_level, opts.precision)


def test_autotune_forest(lfmm):
    rng = np.random.default_rng(9)
    srcs, fs = [], []
    for i in range(48):
        n = int(rng.integers(300, 4000))
        r = np.random.default_rng([9, i])
        srcs.append(workloads.distinct_in_box(r, n, int(np.ceil(4 * np.sqrt(n))), int(r.integers(-9000, 9000)), 0))
        fs.append(workloads.zero_sum(r.standard_normal(n)))
    src = np.ascontiguousarray(np.concatenate(srcs).astype(np.int32))
    off = np.concatenate([[0], np.cumsum([a.shape[0] for a in srcs])]).astype(np.int64)
    opts, r = lfmm.autotune(src, src, 1e-6, off, off)
    assert r["precision"] == lfmm.LFMM_MIXED and r["rel_err"] <= 5e-7
    f = np.concatenate(fs)
    with lfmm.Forest(src, off, src, off, opts=opts) as fo:
        u = fo.eval(f)
    for i in (0, 17, 47):
        ref = oracle.lattice_sum(srcs[i], fs[i], srcs[i])
        ui = u[off[i]:off[i + 1]]
        assert np.abs(ui - ref).max() <= 1e-6 * np.abs(ref).max()
