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
    assert (opts2.p, opts2.leaf_size, opts2.tc_min_level, opts2.precision, opts2.m2l_tile, opts2.m2l_stages,
            opts2.m2l_split) == (opts.p, opts.leaf_size, opts.tc_min_level, opts.precision, opts.m2l_tile,
                                 opts.m2l_stages, opts.m2l_split)
    assert opts.m2l_tile in (0, 16, 32, 64, 128) and opts.m2l_stages in (0, 2, 3, 4) and 0 <= opts.m2l_split <= 9


@pytest.mark.parametrize("tile,stages,split", [(16, 2, 0), (32, 4, 0), (64, 3, 0), (128, 0, 0), (0, 0, 1), (0, 0, 3),
                                               (0, 0, 9)])
def test_m2l_tilings_agree(lfmm, tile, stages, split):
    """Every M2L tiling the autotuner can pick computes the same sums (to rounding) and
    meets the tolerance against the oracle: tensor-core tiles of each width and ring
    depth from level 3 on, and the coarse-level M2L split into 1 .. 9 chunks."""
    prob = workloads.uniform_box(60000, 60000, 1000, seed=23)
    dev = torch.device("cuda:0")
    s, t, f = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    tc = 3 if split == 0 else 0  # tensor cores on every level >= 3, else the default
    res = {}
    for name, kw in (("default", {}), ("tiled", dict(m2l_tile=tile, m2l_stages=stages, m2l_split=split))):
        o = lfmm.make_opts(lfmm.LFMM_MIXED, 8, tc_min_level=tc, tree=lfmm.LFMM_TREE_UNIFORM, **kw)
        with lfmm.Plan(s, t, opts=o) as pl:
            res[name] = pl.eval(f).cpu().numpy()
            pl.status()
    # two plans of the same points may rank a leaf's points differently (plan creation
    # uses atomics), so they agree to the mixed path's rounding, not bit for bit
    scale = np.abs(res["default"]).max()
    assert np.abs(res["tiled"] - res["default"]).max() <= 5e-7 * scale
    idx = np.random.default_rng(3).choice(prob.tgt.shape[0], 128, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    assert np.abs(res["tiled"][idx] - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("split", [1, 2, 5, 7])
def test_list_m2l_split_agrees(lfmm, split):
    """Pruned storage: the list M2L split into a fixed number of chunks gives the same
    result as the library's rule, for the float-float and mixed paths."""
    prob = workloads.clustered_4m(seed=7, n_total=24000, n_clusters=4, sigma=40.0, n_segments=2, seg_len=600.0,
                                  frac_lines=0.02, domain=4096)
    for prec, p, tol in ((lfmm.LFMM_DF, 16, 1e-12), (lfmm.LFMM_MIXED, 8, 2e-7)):
        out = []
        for sp in (0, split):
            with lfmm.Plan(prob.src, prob.tgt, precision=prec, p=p, opts=lfmm.make_opts(prec, p, m2l_split=sp)) as pl:
                assert pl.info()["tree"] == lfmm.LFMM_TREE_PRUNED
                out.append(pl.eval(prob.f))
        assert np.abs(out[1] - out[0]).max() <= tol * np.abs(out[0]).max()


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
