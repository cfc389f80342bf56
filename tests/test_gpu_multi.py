"""Several charge vectors per plan (lfmm_eval_multi): every vector's result is
bit-identical to lfmm_eval of that vector on the same plan (the batched near field does
each vector's operations in the same order), for every path, host and device arrays,
forests, and vector counts that are not a multiple of the four per near-field pass;
one vector is checked against the oracle."""
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


def charges(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(np.stack([workloads.zero_sum(rng.standard_normal(n)) for _ in range(k)]))


@pytest.mark.parametrize("precision,p", [("mixed", 8), ("mixed", 16), ("fp64", 16), ("df", 16)])
def test_multi_equals_single(lfmm, precision, p):
    pr = {"mixed": lfmm.LFMM_MIXED, "fp64": lfmm.LFMM_FP64, "df": lfmm.LFMM_DF}[precision]
    prob = workloads.uniform_box(40000, 30000, 900, seed=17)
    F = charges(prob.src.shape[0], 19, 3)  # more than one group of 16
    with lfmm.Plan(prob.src, prob.tgt, precision=pr, p=p) as pl:
        assert pl.info()["L"] >= 2
        U = pl.eval_multi(F)
        single = np.stack([pl.eval(F[r]) for r in range(F.shape[0])])
        U3 = pl.eval_multi(F[:3])  # a smaller k after a larger one
        pl.status()
    assert np.array_equal(U, single)
    assert np.array_equal(U3, single[:3])
    idx = np.random.default_rng(2).choice(prob.tgt.shape[0], 48, replace=False)
    ref = oracle.lattice_sum(prob.src, F[4], prob.tgt[idx])
    tol = 1e-6 if precision == "mixed" else 1e-10
    assert np.abs(U[4][idx] - ref).max() <= tol * np.abs(ref).max()


def test_multi_device_arrays_and_forest(lfmm):
    dev = torch.device("cuda:0")
    prob = workloads.uniform_box(20000, 20000, 700, seed=18)
    F = charges(prob.src.shape[0], 9, 4)
    with lfmm.Plan(prob.src, prob.tgt) as pl:
        Ud = pl.eval_multi(torch.from_numpy(F).to(dev)).cpu().numpy()
        Uh = pl.eval_multi(F)
        u0 = pl.eval(F[8])
    assert np.array_equal(Ud, Uh) and np.array_equal(Uh[8], u0)
    # a forest evaluates the vectors one after another
    src = np.ascontiguousarray(np.concatenate([prob.src[:5000], prob.src[5000:9000] + 100000]))
    off = np.array([0, 5000, 9000], dtype=np.int64)
    Ff = charges(9000, 2, 5)
    with lfmm.Forest(src, off, src, off) as fo:
        Uf = fo.eval_multi(Ff)
        assert np.array_equal(Uf[1], fo.eval(Ff[1]))
