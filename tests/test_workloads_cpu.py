"""The synthetic inputs have the shapes, sizes and properties of the configurations:
distinct lattice points, exact zero-sum charges (c11 reading), sizes and seeds as
stated, and request generation independent of order (serving)."""
import math

import numpy as np

from paper_1105_3505_gb300 import workloads


def _distinct(p):
    return np.unique(p, axis=0).shape[0] == p.shape[0]


def test_zero_sum_is_exact():
    rng = np.random.default_rng(0)
    for n in (1, 2, 17, 4096):
        f = workloads.zero_sum(rng.standard_normal(n) * 1e3)
        assert math.fsum(f.tolist()) == 0.0 or abs(math.fsum(f.tolist())) <= np.spacing(np.abs(f).max())


def test_uniform_4k():
    p = workloads.uniform_4k()
    assert p.src.shape == (4096, 2) and p.src.dtype == np.int32 and _distinct(p.src)
    assert p.src.min() >= 0 and p.src.max() < 256
    assert np.array_equal(p.src, p.tgt) and p.same_points
    assert abs(math.fsum(p.f.tolist())) <= 1e-12
    assert np.array_equal(workloads.uniform_4k().src, p.src)  # seeded


def test_uniform_box_and_distinct_in_box():
    rng = np.random.default_rng(3)
    pts = workloads.distinct_in_box(rng, 1000, 40, -7, 11)
    assert _distinct(pts) and pts[:, 0].min() >= -7 and pts[:, 0].max() < 33
    assert pts[:, 1].min() >= 11 and pts[:, 1].max() < 51
    b = workloads.uniform_box(500, 300, 64, seed=9)
    assert b.src.shape == (500, 2) and b.tgt.shape == (300, 2) and _distinct(b.src) and _distinct(b.tgt)


def test_clustered_small_instance():
    p = workloads.clustered_4m(seed=2, n_total=20000, n_clusters=4, sigma=30.0, n_segments=2, seg_len=500.0,
                               frac_lines=0.02, domain=4096)
    assert p.src.shape == (20000, 2) and _distinct(p.src) and np.array_equal(p.src, p.tgt)
    # U(-1, 1) shifted by its mean and with the last entry fixed: |f| just above 1 at most
    assert abs(math.fsum(p.f.tolist())) <= 1e-12 and np.abs(p.f).max() <= 1.1


def test_forest_sizes():
    s = workloads.forest_sizes()
    assert s.shape == (4096,) and s.min() >= 512 and s.max() <= 8192
    assert 2400 < s.mean() < 3200  # E[N] = (8192 - 512) / ln 16 = 2770


def test_serve_requests_independent_of_order():
    sch = workloads.serve_schedule(seed=4, n_requests=50)
    assert np.all(np.diff(sch["arrival_s"]) > 0)
    assert set(np.unique(sch["tol"]).tolist()) <= {1e-6, 1e-10}
    full = workloads.serve_schedule(seed=4, n_requests=20_000)
    for k in ("arrival_s", "n_src", "kind", "tol"):  # a short stream is a prefix of the full one
        assert np.array_equal(full[k][:50], sch[k])
    a = workloads.serve_request(sch, 7)
    b = [r for r in workloads.serve_stream(seed=4, n_requests=8)][7]
    assert np.array_equal(a.problem.src, b.problem.src) and np.array_equal(a.problem.f, b.problem.f)
    n = int(sch["n_src"][7])
    assert a.problem.src.shape == (n, 2) and a.problem.tgt.shape == (max(1, n // 4), 2) and _distinct(a.problem.src)
