"""The tensor-core M2L (tcgen05, 3xTF32 split, mixed path) against the oracle.

tc_min_level = 2 puts every M2L level on the tensor-core kernel, so small problems
exercise it; the default (level >= 8) is exercised by the full-size test in
test_gpu_parity.py.  lfmm_plan_status must report no timed-out device wait."""
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


@pytest.mark.parametrize("case", ["uniform_4k", "box_20k", "box_ragged"])
def test_tensor_core_m2l_parity(lfmm, case):
    if case == "uniform_4k":
        prob = workloads.uniform_4k()
    elif case == "box_20k":
        prob = workloads.uniform_box(20000, 15000, 1500, seed=44)
    else:
        prob = workloads.uniform_box(9000, 7000, 700, seed=45)  # partial CTA tiles
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
    with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=8, tc_min_level=2) as pl:
        u_tc = pl.eval(prob.f)
        pl.status()
    with lfmm.Plan(prob.src, prob.tgt, precision=lfmm.LFMM_MIXED, p=8, tc_min_level=99) as pl:
        u_simt = pl.eval(prob.f)
        pl.status()
    assert rel_err(u_tc, ref) <= 1e-6
    assert rel_err(u_simt, ref) <= 1e-6
    # the two M2L implementations differ only by rounding
    assert np.abs(u_tc - u_simt).max() <= 1e-6 * np.abs(ref).max()
