"""lfmm_plan_shape_noalloc against lfmm_plan_create.

The entry point serves callers that cannot allocate device memory when they need to
size a problem (admission control before memory is committed, host code running under
CUDA stream capture, processes whose device memory belongs to another allocator).  It
must report exactly the tree and footprint a real plan gets: integers, compared
exactly.  Two calls in a row check that the shared static scratch carries nothing over
from one call to the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1105_3505_gb300 import build, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ["n_src", "n_tgt", "x0", "y0", "K", "L", "leaf_side", "P", "P_pad", "precision",
          "max_leaf_src", "max_leaf_tgt", "device_bytes", "tree", "n_problems", "n_boxes"]


@pytest.fixture(scope="module")
def lfmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1105_3505_gb300 import lfmm as m
    m.load()
    return m


def _dev(prob):
    d = torch.device("cuda:0")
    return torch.from_numpy(prob.src).to(d), torch.from_numpy(prob.tgt).to(d)


def test_shape_noalloc_matches_plan_twice(lfmm):
    cases = [(workloads.uniform_box(50_000, 30_000, 2000, seed=31), lfmm.make_opts(lfmm.LFMM_MIXED, 8)),
             (workloads.uniform_4k(), lfmm.make_opts(lfmm.LFMM_FP64, 16))]
    for prob, opts in cases:  # two calls in a row on different inputs share the scratch
        s, t = _dev(prob)
        shape = lfmm.lfmm_plan_shape_noalloc(s, s.shape[0], t, t.shape[0], opts)
        torch.cuda.synchronize()
        h = lfmm.lfmm_plan_create(s, s.shape[0], t, t.shape[0], opts, None)
        info = lfmm.lfmm_plan_get_info(h)
        lfmm.lfmm_plan_destroy(h)
        assert {k: shape[k] for k in FIELDS} == {k: info[k] for k in FIELDS}


def test_shape_noalloc_rejects_beyond_scratch(lfmm):
    # a sparse set spread over 2^26 cells per axis with leaf side <= 32 needs level >= 21
    rng = np.random.default_rng(3)
    src = rng.integers(0, 1 << 26, size=(1000, 2)).astype(np.int32)
    s = torch.from_numpy(src).cuda()
    with pytest.raises(lfmm.LfmmError) as ei:
        lfmm.lfmm_plan_shape_noalloc(s, 1000, s, 1000, lfmm.make_opts())
    assert ei.value.status == lfmm.LFMM_EINVAL and "supports levels up to" in str(ei.value)
    # host coordinates are refused (copying them would need a device buffer)
    with pytest.raises(lfmm.LfmmError):
        lfmm.lfmm_plan_shape_noalloc(src, 1000, src, 1000, lfmm.make_opts())
