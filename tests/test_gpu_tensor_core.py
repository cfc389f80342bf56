"""The tensor-core M2L (tcgen05, 3xTF32 split, mixed path, P_pad 32 and 64) against the oracle.

tc_min_level = 2 puts every M2L level on the tensor-core kernel, so small problems
exercise it; the default (level >= 6) is exercised by the full-size test in
test_gpu_parity.py.  Levels whose parity class spans >= 128 boxes per row (level >= 8)
use row tiles (one class row per tile); a sparse point set in a 4096^2 box with leaves
capped at side 16 reaches level 8 with few points, so the oracle checks that shape in
full.  lfmm_plan_status must report no timed-out device wait."""
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
    return m


def rel_err(u, ref):
    return float(np.abs(u - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("p", [8, 12, 16])
@pytest.mark.parametrize("case", ["uniform_4k", "box_20k", "box_ragged"])
def test_tensor_core_m2l_parity(lfmm, case, p):
    """p = 8 (P_pad = 32: one 128-byte K-block per interaction offset) and p = 12, 16
    (P_pad = 64: two K-blocks accumulated per offset)."""
    if case == "uniform_4k":
        prob = workloads.uniform_4k()
    elif case == "box_20k":
        prob = workloads.uniform_box(20000, 15000, 1500, seed=44)
    else:
        prob = workloads.uniform_box(9000, 7000, 700, seed=45)  # partial CTA tiles
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
    with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=p, tc_min_level=2,
                   tree=lfmm.LFMM_TREE_UNIFORM) as pl:
        lfmm.lfmm_profile_enable(True)
        lfmm.lfmm_profile_read(reset=True)
        try:
            u_tc = pl.eval(prob.f)
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        pl.status()
        assert pl.info()["P_pad"] == (32 if p <= 9 else 64)
    assert prof["m2l_tc"][1] > 0 and prof["m2l"][1] == 0  # every M2L level on the tensor cores
    with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=p, tc_min_level=99,
                   tree=lfmm.LFMM_TREE_UNIFORM) as pl:
        u_simt = pl.eval(prob.f)
        pl.status()
    assert rel_err(u_tc, ref) <= 1e-6
    assert rel_err(u_simt, ref) <= 1e-6
    # the two M2L implementations differ only by rounding
    assert np.abs(u_tc - u_simt).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("p", [8, 16])
def test_tensor_core_row_windows_full_oracle(lfmm, p):
    prob = workloads.uniform_box(30000, 20000, 4096, seed=46)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
    with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=p, max_leaf_side=16,
                   tree=lfmm.LFMM_TREE_UNIFORM) as pl:
        info = pl.info()
        u = pl.eval(prob.f)
        pl.status()
    assert info["L"] == 8 and info["leaf_side"] == 16
    assert rel_err(u, ref) <= 1e-6, rel_err(u, ref)


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("tile", [16, 128])
def test_tensor_core_p16_tilings(lfmm, stages, tile):
    """P_pad = 64 with every ring depth and two tile widths (16 boxes: 8 rows per tile on
    the finer levels; 128: whole class rows), each within the mixed bar of the oracle."""
    prob = workloads.uniform_box(20000, 15000, 1500, seed=47)
    dev = torch.device("cuda:0")
    s, t, f = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    o = lfmm.make_opts(lfmm.LFMM_MIXED, 16, tc_min_level=2, tree=lfmm.LFMM_TREE_UNIFORM, m2l_tile=tile,
                       m2l_stages=stages)
    with lfmm.Plan(s, t, opts=o) as pl:
        u = pl.eval(f).cpu().numpy()
        pl.status()
    idx = np.random.default_rng(5).choice(prob.tgt.shape[0], 256, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    assert rel_err(u[idx], ref) <= 1e-6
