"""Pins of the oracle's brute-force lattice sum.

The decisive pin is the identity A u = f (eq. 1.1 with eq. 1.7): applying the
5-point operator of eq. 1.2 to the computed potential must return the charges,
at every lattice site whose full stencil was evaluated, including sites far
enough away that the asymptotic branch of phi is used.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1105_3505_gb300 import workloads


def _stencil_targets(src, pad):
    xs = range(src[:, 0].min() - pad, src[:, 0].max() + pad + 1)
    ys = range(src[:, 1].min() - pad, src[:, 1].max() + pad + 1)
    return np.array([(x, y) for x in xs for y in ys], dtype=np.int32)


@pytest.mark.parametrize("offset", [0, 1000, -70000])
def test_A_u_equals_f_zero_sum(offset):
    rng = np.random.default_rng(11)
    src = workloads.distinct_in_box(rng, 24, 12) + offset
    f = workloads.zero_sum(rng.standard_normal(24))
    tgt = _stencil_targets(src, 2)
    u = oracle.lattice_sum(src, f, tgt)
    u_of = {(int(x), int(y)): v for (x, y), v in zip(tgt, u)}
    f_of = {(int(x), int(y)): v for (x, y), v in zip(src, f)}
    scale = np.abs(u).max()
    worst = 0.0
    for (x, y) in u_of:
        if all(k in u_of for k in [(x + 1, y), (x - 1, y), (x, y + 1), (x, y - 1)]):
            r = oracle.apply_A(u_of, (x, y)) - f_of.get((x, y), 0.0)
            worst = max(worst, abs(r))
    assert worst < 1e-12 * max(scale, 1.0)


def test_A_u_equals_f_far_from_sources():
    """Stencils around sites 300-400 lattice units away use eq. 3.1 for phi."""
    rng = np.random.default_rng(5)
    src = workloads.distinct_in_box(rng, 16, 8)
    f = workloads.zero_sum(rng.standard_normal(16))
    centres = [(350, 3), (-290, 280), (10, -400)]
    tgt = np.array([(cx + dx, cy + dy) for cx, cy in centres
                    for dx, dy in [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]], dtype=np.int32)
    u = oracle.lattice_sum(src, f, tgt)
    for k in range(len(centres)):
        c = u[5 * k: 5 * k + 5]
        assert abs(4 * c[0] - c[1:].sum()) < 2e-14  # a wrong eq. 3.1 term leaves ~1e-11


def test_single_charge_reproduces_phi_and_symmetry():
    src = np.array([[5, -3]], dtype=np.int32)
    tgt = np.array([[5, -3], [6, -3], [6, -2], [105, 40], [-400, 17]], dtype=np.int32)
    u = oracle.lattice_sum(src, np.array([1.0]), tgt)
    assert u[0] == 0.0                           # phi(0) = 0
    assert u[1] == -0.25                         # phi(e1) = -1/4
    assert abs(u[2] + 1 / math.pi) < 1e-16       # phi(1,1) = -1/pi
    # reciprocity phi(x - y) = phi(y - x)
    u2 = oracle.lattice_sum(tgt[3:4], np.array([1.0]), src)
    assert u2[0] == u[3]


def test_linearity_and_duplicates():
    rng = np.random.default_rng(3)
    src = workloads.distinct_in_box(rng, 50, 30)
    tgt = workloads.distinct_in_box(rng, 40, 30)
    f1, f2 = rng.standard_normal(50), rng.standard_normal(50)
    u = oracle.lattice_sum(src, 2 * f1 - f2, tgt)
    ref = 2 * oracle.lattice_sum(src, f1, tgt) - oracle.lattice_sum(src, f2, tgt)
    assert np.allclose(u, ref, rtol=0, atol=1e-13)
    # a duplicated source point adds its charges
    src_d = np.concatenate([src, src[:5]])
    f_d = np.concatenate([f1, f1[:5]])
    f_m = f1.copy()
    f_m[:5] *= 2
    assert np.allclose(oracle.lattice_sum(src_d, f_d, tgt), oracle.lattice_sum(src, f_m, tgt), atol=1e-13)


def test_near_sum_locality():
    rng = np.random.default_rng(9)
    src = workloads.distinct_in_box(rng, 200, 64)
    tgt = workloads.distinct_in_box(rng, 100, 64)
    f = rng.standard_normal(200)
    # one leaf holding everything: near field = whole sum
    assert np.allclose(oracle.near_sum(src, f, tgt, 0, 0, 64), oracle.lattice_sum(src, f, tgt), atol=1e-14)
    # leaves of side 8: the near sum only sees sources in the 3x3 leaf block
    s = 8
    un = oracle.near_sum(src, f, tgt, 0, 0, s)
    for i in range(0, 100, 7):
        bt = tgt[i] // s
        mask = np.all(np.abs(src // s - bt) <= 1, axis=1)
        ref = oracle.lattice_sum(src[mask], f[mask], tgt[i:i + 1])[0]
        assert abs(un[i] - ref) < 1e-14


def test_uniform_tree_rule():
    p = workloads.uniform_4k()
    t = oracle.uniform_tree(p.src, p.tgt, 64)
    assert (t["K"], t["L"], t["side"]) == (8, 4, 16)
    # definition check: level L-1 overflows, level L does not
    for level, ok in [(t["L"], True), (t["L"] - 1, False)]:
        sh = t["K"] - level
        keys = ((p.src[:, 0] - t["x0"]) >> sh) * (1 << level) + ((p.src[:, 1] - t["y0"]) >> sh)
        assert (np.bincount(keys).max() <= 64) == ok
    # leaf side cap
    t2 = oracle.uniform_tree(p.src, p.tgt, 10_000, max_leaf_side=32)
    assert t2["side"] == 32
    # coincident points cannot be separated: leaves of side 1
    pts = np.zeros((100, 2), dtype=np.int32)
    pts[99] = 7
    t3 = oracle.uniform_tree(pts, pts, 64)
    assert t3["side"] == 1 and t3["K"] == 3 and t3["L"] == 3
    pts[50:] = 7   # two stacks of 50 separate at level 1
    t4 = oracle.uniform_tree(pts, pts, 64)
    assert t4["side"] == 4 and t4["L"] == 1


def test_workload_generators():
    p = workloads.uniform_4k()
    assert p.src.shape == (4096, 2) and p.src.min() >= 0 and p.src.max() < 256
    assert len({(int(x), int(y)) for x, y in p.src}) == 4096
    assert abs(math.fsum(p.f)) < 1e-12
    q = workloads.uniform_4k()
    assert np.array_equal(p.src, q.src) and np.array_equal(p.f, q.f)
    sizes = workloads.forest_sizes()
    assert sizes.shape == (4096,) and sizes.min() >= 512 and sizes.max() <= 8192
