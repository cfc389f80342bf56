"""A plan's device footprint and the coarse-level M2L split along K.

Binary64-width (binary64, float-float) plans and mixed plans with few coarse-level tiles
split the fused coarse-level M2L along the 27 interaction offsets; its partial sums live
in a plan-owned buffer.  That buffer belongs to the plan from creation on, so
lfmm_plan_get_info reports the same device_bytes before and after the first evaluation,
and lfmm_plan_shape_noalloc (which a server uses to size a request before committing
memory) reports the same figure.  If the buffer were missing or too small the library
would fall back to one M2L launch per level; the phase counters show the single fused
launch instead, and the result matches the oracle.
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
    return m


@pytest.mark.parametrize("precision,p,tol", [("df", 16, 1e-10), ("fp64", 16, 1e-10), ("mixed", 8, 1e-6),
                                             ("mixed", 16, 1e-6)])
def test_split_m2l_footprint_and_launches(lfmm, precision, p, tol):
    prec = {"df": lfmm.LFMM_DF, "fp64": lfmm.LFMM_FP64, "mixed": lfmm.LFMM_MIXED}[precision]
    prob = workloads.uniform_box(10000, 10000, 400, seed=44)
    dev = torch.device("cuda:0")
    s, t, f = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    opts = lfmm.make_opts(prec, p)
    shape = lfmm.lfmm_plan_shape_noalloc(s, s.shape[0], t, t.shape[0], opts)
    with lfmm.Plan(s, t, precision=prec, p=p) as pl:
        before = pl.info()
        assert 2 <= before["L"] <= 6  # every M2L level in the fused coarse-level kernel
        lfmm.lfmm_profile_enable(True)
        try:
            lfmm.lfmm_profile_read(reset=True)
            u = pl.eval(f)
            torch.cuda.synchronize()
            prof = lfmm.lfmm_profile_read(reset=True)
        finally:
            lfmm.lfmm_profile_enable(False)
        after = pl.info()
    assert before["device_bytes"] == after["device_bytes"] == shape["device_bytes"]
    assert prof["m2l"][1] == 1 and prof["m2l_tc"][1] == 0, prof
    idx = np.random.default_rng(9).choice(prob.tgt.shape[0], 512, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    err = np.abs(u.cpu().numpy()[idx] - ref).max() / np.abs(ref).max()
    assert err <= tol, err
