"""Pruned trees and forests through the C ABI, against the CPU oracle.

Pruned storage keeps only boxes with points below them (clustered inputs); a forest
evaluates many independent problems in one plan.  Both must reach the same bars as
the uniform tree: rel_err <= 1e-10 for binary64 at p = 16, <= 1e-6 mixed at p = 8.
"""
import zlib

import numpy as np
import pytest

import oracle
from paper_1105_3505_gb300 import build, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def lfmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1105_3505_gb300 import lfmm as m
    m.load()
    torch.cuda.init()
    return m


def rel_err(u, ref):
    return float(np.abs(np.asarray(u) - ref).max() / max(np.abs(ref).max(), 1e-300))


def prec_of(lfmm, name):
    return {"fp64": (lfmm.LFMM_FP64, 16, FP64_TOL), "df": (lfmm.LFMM_DF, 16, FP64_TOL),
            "mixed": (lfmm.LFMM_MIXED, 8, MIXED_TOL), "mixed16": (lfmm.LFMM_MIXED, 16, MIXED_TOL)}[name]


def small_clustered(seed=7):
    """Four Gaussian clusters and a line in a 4096^2 box: most leaves of the uniform
    tree are empty."""
    return workloads.clustered_4m(seed=seed, n_total=24000, n_clusters=4, sigma=40.0, n_segments=2,
                                  seg_len=600.0, frac_lines=0.02, domain=4096)


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_automatic_pruned_tree_equals_forced(lfmm, seed):
    """Automatic storage turns to the pruned builder as soon as a count shows a mostly
    empty level; the tree it gets (root, leaf level and side, boxes, fullest leaves) is the
    one the full leaf-level search and forced pruned storage give."""
    prob = small_clustered(seed=seed)
    infos = []
    for tree in (lfmm.LFMM_TREE_AUTO, lfmm.LFMM_TREE_PRUNED):
        with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=8, tree=tree) as pl:
            infos.append(pl.info())
    keys = ("tree", "x0", "y0", "K", "L", "leaf_side", "n_boxes", "max_leaf_src", "max_leaf_tgt")
    assert [infos[0][k] for k in keys] == [infos[1][k] for k in keys]
    assert infos[0]["tree"] == lfmm.LFMM_TREE_PRUNED


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed16", "df"])
def test_pruned_clustered_full_oracle(lfmm, precision):
    prob = small_clustered()
    prec, p, tol = prec_of(lfmm, precision)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
    with lfmm.Plan(prob.src, prob.tgt, precision=prec, p=p) as pl:
        u = pl.eval(prob.f)
        info = pl.info()
    assert info["tree"] == lfmm.LFMM_TREE_PRUNED  # chosen automatically
    tree = oracle.uniform_tree(prob.src, prob.tgt, 64, 32)
    assert (info["x0"], info["y0"], info["K"], info["L"], info["leaf_side"]) == \
        (tree["x0"], tree["y0"], tree["K"], tree["L"], tree["side"])
    assert rel_err(u, ref) <= tol, rel_err(u, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pruned_equals_uniform(lfmm, precision):
    """Same boxes, operators and summation structure: the two storages agree to rounding."""
    prob = workloads.uniform_box(6000, 4000, 700, seed=31)
    prec, p, _ = prec_of(lfmm, precision)
    with lfmm.Plan(prob.src, prob.tgt, precision=prec, p=p, tree=lfmm.LFMM_TREE_UNIFORM) as a:
        ua = a.eval(prob.f)
        ia = a.info()
    with lfmm.Plan(prob.src, prob.tgt, precision=prec, p=p, tree=lfmm.LFMM_TREE_PRUNED) as b:
        ub = b.eval(prob.f)
        ib = b.info()
        un, uf = b.eval_parts(prob.f)
    assert ia["tree"] == lfmm.LFMM_TREE_UNIFORM and ib["tree"] == lfmm.LFMM_TREE_PRUNED
    assert (ia["K"], ia["L"], ia["leaf_side"]) == (ib["K"], ib["L"], ib["leaf_side"])
    scale = np.abs(ua).max()
    assert np.abs(ua - ub).max() <= (1e-12 if precision == "fp64" else 1e-6) * scale
    assert np.abs(ub - (un + uf)).max() <= 1e-12 * scale


def forest_case(seed, n_problems, n_min=64, n_max=3000, targets_equal=True):
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_problems))).astype(int)
    probs = []
    for i, n in enumerate(sizes):
        r = np.random.default_rng([seed, i])
        side = int(np.ceil(4 * np.sqrt(n)))
        x0, y0 = r.integers(-100000, 100000, size=2)
        src = workloads.distinct_in_box(r, int(n), side, int(x0), int(y0))
        if targets_equal:
            tgt = src.copy()
        else:
            nt = max(1, int(n) // 3)
            tgt = workloads.distinct_in_box(r, nt, side, int(x0), int(y0))
        f = workloads.zero_sum(r.standard_normal(int(n)))
        probs.append((src, tgt, f))
    return probs


def concat(probs):
    src = np.ascontiguousarray(np.concatenate([p[0] for p in probs]).astype(np.int32))
    tgt = np.ascontiguousarray(np.concatenate([p[1] for p in probs]).astype(np.int32))
    f = np.concatenate([p[2] for p in probs])
    so = np.concatenate([[0], np.cumsum([p[0].shape[0] for p in probs])]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum([p[1].shape[0] for p in probs])]).astype(np.int64)
    return src, so, tgt, to, f


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed16", "df"])
@pytest.mark.parametrize("targets_equal", [True, False])
def test_forest_full_oracle(lfmm, precision, targets_equal):
    probs = forest_case(zlib.crc32(f"forest{targets_equal}".encode()), 40, targets_equal=targets_equal)
    src, so, tgt, to, f = concat(probs)
    prec, p, tol = prec_of(lfmm, precision)
    with lfmm.Forest(src, so, tgt, to, precision=prec, p=p) as fo:
        u = fo.eval(f)
        info = fo.info()
    assert info["n_problems"] == 40 and info["tree"] == lfmm.LFMM_TREE_PRUNED
    for i, (s, t, fi) in enumerate(probs):
        ref = oracle.lattice_sum(s, fi, t)
        ui = u[to[i]:to[i + 1]]
        assert rel_err(ui, ref) <= tol, (i, s.shape[0], rel_err(ui, ref))


def test_forest_edge_problems(lfmm):
    """One-point problems, a single leaf, coincident sources, a problem far from the
    others, and targets outside the sources' box - all in one forest."""
    rng = np.random.default_rng(5)
    probs = []
    probs.append((np.array([[3, 4]], np.int32), np.array([[3, 4]], np.int32), np.array([1.5])))
    probs.append((np.array([[0, 0]], np.int32), workloads.distinct_in_box(rng, 30, 20, -10, -10), np.array([2.0])))
    s = workloads.distinct_in_box(rng, 50, 10, 1000, 1000)
    probs.append((s, s.copy(), workloads.zero_sum(rng.standard_normal(50))))
    probs.append((np.full((40, 2), 7, np.int32), workloads.distinct_in_box(rng, 25, 64), rng.standard_normal(40)))
    off = (1 << 30) - 3000
    s = workloads.distinct_in_box(rng, 1500, 400, off, -off)
    probs.append((s, workloads.distinct_in_box(rng, 700, 400, off, -off), workloads.zero_sum(rng.standard_normal(1500))))
    s = workloads.distinct_in_box(rng, 800, 300)
    probs.append((s, workloads.distinct_in_box(rng, 200, 100, 2000, 2500), workloads.zero_sum(rng.standard_normal(800))))
    src, so, tgt, to, f = concat(probs)
    for precision in ("fp64", "mixed", "df"):
        prec, p, tol = prec_of(lfmm, precision)
        with lfmm.Forest(src, so, tgt, to, precision=prec, p=p) as fo:
            u = fo.eval(f)
            side = fo.info()["leaf_side"]
        for i, (s, t, fi) in enumerate(probs):
            ref = oracle.lattice_sum(s, fi, t)
            ui = u[to[i]:to[i + 1]]
            if np.abs(ref).max() == 0.0:
                # phi(0) = 0.  The mixed path deflates its binary32 near-field table by
                # phi0 = phi(s, 0) and adds phi0 * Q back in float pairs (Sec. 2 splits the
                # near sum; the constant is free), so a coincident pair leaves
                # (fl32(fl32(phi(0) - phi0) f32) + phi0 f): the rounding of phi0 and of one
                # binary32 product, at most 2^-23 |phi0| |f|.  The uniform tree of this
                # point alone has side 1, where phi0 = -1/4 and every step is exact; the
                # forest's shared leaf side is larger, and phi(s, 0) is not a binary32 number.
                bound = {"fp64": 0.0, "df": 1e-14 * np.abs(fi).sum(),
                         "mixed": 2.0 ** -23 * abs(float(oracle.phi(np.array([[side, 0]]))[0])) * np.abs(fi).sum()}
                assert np.abs(ui).max() <= bound[precision], (precision, side, np.abs(ui).max())
            elif i == 5 and precision == "mixed":
                # targets far from zero-sum sources (|u| is 4e-2 of the terms that cancel
                # in it): binary32 rounding of the cancelling terms, as for the uniform
                # tree's far-target case, 2e-7 (3.4 x 2^-24) of the natural scale
                d = (t[:, None, :].astype(np.int64) - s[None, :, :]).reshape(-1, 2)
                ph = oracle.phi(d).reshape(t.shape[0], s.shape[0])
                scale = (np.abs(fi)[None, :] * np.abs(ph - ph[:, :1])).sum(axis=1).max()
                assert np.abs(ui - ref).max() <= 2e-7 * scale
            else:
                assert rel_err(ui, ref) <= tol, (precision, i, rel_err(ui, ref))


@pytest.fixture(scope="module")
def forest_4096():
    probs = workloads.forest_4096()
    sel = np.random.default_rng(11).choice(4096, 24, replace=False)
    refs = {int(i): oracle.lattice_sum(probs[i].src, probs[i].f, probs[i].tgt) for i in sel}
    return probs, concat([(p.src, p.tgt, p.f) for p in probs]), refs


# p = 7 is the order the autotuner picks for this workload at 1e-6 (mixed)
@pytest.mark.parametrize("precision,p", [("mixed", 7), ("mixed", 8), ("mixed", 16), ("df", 16), ("fp64", 16)])
def test_forest_4096_sampled(lfmm, forest_4096, precision, p):
    """The full batched workload: 4,096 problems, N_src log-uniform in [512, 8192] in a
    box of side 4 sqrt(N), targets = sources; 24 problems checked in full."""
    probs, (src, so, tgt, to, f), refs = forest_4096
    prec, _, tol = prec_of(lfmm, precision)
    dev = torch.device("cuda:0")
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (src, tgt, f))
    with lfmm.Forest(s_d, so, t_d, to, precision=prec, p=p) as fo:
        u = fo.eval(f_d).cpu().numpy()
        info = fo.info()
    assert info["n_problems"] == 4096 and np.isfinite(u).all()
    for i, ref in refs.items():
        assert rel_err(u[to[i]:to[i + 1]], ref) <= tol, i


@pytest.fixture(scope="module")
def clustered_4m():
    prob = workloads.clustered_4m()
    idx = np.random.default_rng(321).choice(prob.tgt.shape[0], 256, replace=False)
    return prob, idx, oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])


@pytest.mark.parametrize("precision,p", [("mixed", 8), ("mixed", 16), ("df", 16), ("fp64", 16)])
def test_clustered_4m_sampled(lfmm, clustered_4m, precision, p):
    """The full clustered workload (4,194,304 points, 64 clusters + 16 segments) on the
    pruned tree; 256 seeded targets checked against the oracle."""
    prob, idx, ref = clustered_4m
    prec, _, tol = prec_of(lfmm, precision)
    dev = torch.device("cuda:0")
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    with lfmm.Plan(s_d, t_d, precision=prec, p=p) as pl:
        u = pl.eval(f_d).cpu().numpy()
        info = pl.info()
    assert info["tree"] == lfmm.LFMM_TREE_PRUNED and np.isfinite(u).all()
    assert rel_err(u[idx], ref) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed16", "df"])
def test_forest_persistent_sweeps_equal_per_level(lfmm, precision):
    """With LFMM_FLAG_PERSISTENT the upward and downward sweeps of a forest run as one
    persistent cooperative launch each (work queues per level, grid barriers between
    levels); by default the same plan runs one launch per level.  Same arithmetic per box
    (the list M2L on the CUDA cores in both forms: tc_min_level 99): the results are
    bit-identical, and the persistent form launches one kernel per sweep."""
    probs = forest_case(zlib.crc32(b"fused"), 60, n_min=200, n_max=9000)
    src, so, tgt, to, f = concat(probs)
    prec, p, tol = prec_of(lfmm, precision)
    with lfmm.Forest(src, so, tgt, to, precision=prec, p=p, tc_min_level=99) as fo:
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            u_level = fo.eval(f)
            prof_level = lfmm.lfmm_profile_read(reset=True)
            fo.set_flags(persistent=True)
            u_fused = fo.eval(f)
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        fo.status()
    assert np.array_equal(u_fused, u_level)
    assert prof["m2m"][1] == 1 and prof["m2l"][1] == 1 and prof["p2m"][1] == 0
    assert prof_level["m2l"][1] > 1
    for i in (0, 31, 59):
        ref = oracle.lattice_sum(probs[i][0], probs[i][2], probs[i][1])
        assert rel_err(u_fused[to[i]:to[i + 1]], ref) <= tol


@pytest.mark.parametrize("p", [8, 16])
def test_forest_persistent_sweeps_with_tensor_core_levels(lfmm, p):
    """Mixed path, default tensor-core levels: the persistent downward sweep takes the
    coarse levels and the levels of at least 1,024 boxes follow as tensor-core launches,
    the same kernels as in the per-level form, so the two forms stay bit-identical."""
    probs = forest_case(zlib.crc32(b"fused-tc"), 48, n_min=500, n_max=6000)
    src, so, tgt, to, f = concat(probs)
    with lfmm.Forest(src, so, tgt, to, precision=lfmm.LFMM_MIXED, p=p) as fo:
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            u_level = fo.eval(f)
            prof_level = lfmm.lfmm_profile_read(reset=True)
            fo.set_flags(persistent=True)
            u_fused = fo.eval(f)
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        fo.status()
    assert np.array_equal(u_fused, u_level)
    assert prof["m2l_tc"][1] > 0 and prof["m2l_tc"][1] == prof_level["m2l_tc"][1]
    assert prof["m2m"][1] == 1 and prof["m2l"][1] == 1 and prof_level["m2l"][1] > 1
    for i in (0, 47):
        ref = oracle.lattice_sum(probs[i][0], probs[i][2], probs[i][1])
        assert rel_err(u_fused[to[i]:to[i + 1]], ref) <= MIXED_TOL


def test_clustered_persistent_sweeps(lfmm):
    """A pruned tree of many levels (the persistent sweeps cross 9 grid barriers) against
    the per-level launches and the oracle."""
    prob = small_clustered()
    for prec, p, tol in ((lfmm.LFMM_MIXED, 8, MIXED_TOL), (lfmm.LFMM_DF, 16, FP64_TOL)):
        with lfmm.Plan(prob.src, prob.tgt, precision=prec, p=p, tc_min_level=99) as pl:
            u0 = pl.eval(prob.f)
            pl.set_flags(persistent=True)
            u1 = pl.eval(prob.f)
            pl.status()
        assert np.array_equal(u0, u1)
    idx = np.arange(0, prob.tgt.shape[0], 37)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    assert rel_err(u1[idx], ref) <= tol


@pytest.mark.parametrize("p", [8, 16])
@pytest.mark.parametrize("case", ["forest", "forest_separate_targets", "clustered"])
def test_tensor_core_list_m2l(lfmm, case, p):
    """Mixed path: the list M2L of every pruned / forest level with at least 1,024 boxes
    runs on the tensor cores (gathered A operand, 3xTF32 split, fresh accumulators per
    offset; p = 8: P_pad 32, one K-block per offset; p = 16: P_pad 64, two); against the
    CUDA-core list kernel (tc_min_level 99) to the mixed path's rounding, and against the
    oracle.  Class ranges are not multiples of the 128-box tile, so partial tiles are
    covered."""
    if case == "clustered":
        prob = small_clustered()
        make = lambda **kw: lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=p, **kw)
        f, tgt_ranges = prob.f, [(0, prob.tgt.shape[0], prob.src, prob.f, prob.tgt)]
    else:
        probs = forest_case(zlib.crc32(case.encode()), 48, targets_equal=(case == "forest"))
        src, so, tgt, to, f = concat(probs)
        make = lambda **kw: lfmm.Forest(src, so, tgt, to, precision=lfmm.LFMM_MIXED, p=p, **kw)
        tgt_ranges = [(to[i], to[i + 1], probs[i][0], probs[i][2], probs[i][1]) for i in (0, 23, 47)]
    out, prof = {}, {}
    for name, kw in (("tc", {}), ("simt", dict(tc_min_level=99))):
        with make(**kw) as pl:
            assert pl.info()["tree"] == lfmm.LFMM_TREE_PRUNED
            lfmm.lfmm_profile_enable(True)
            lfmm.lfmm_profile_read(reset=True)
            try:
                out[name] = pl.eval(f)
                prof[name] = lfmm.lfmm_profile_read(reset=True)
            finally:
                lfmm.lfmm_profile_enable(False)
            pl.status()
    assert prof["tc"]["m2l_tc"][1] > 0 and prof["simt"]["m2l_tc"][1] == 0
    scale = np.abs(out["simt"]).max()
    assert np.abs(out["tc"] - out["simt"]).max() <= MIXED_TOL * scale
    for a, b, s, fi, t in tgt_ranges:
        idx = np.arange(a, b, max(1, (b - a) // 200))
        ref = oracle.lattice_sum(s, fi, t[idx - a])
        assert rel_err(out["tc"][idx], ref) <= MIXED_TOL
