"""Lattices with local modifications (Sec. 10.1) through the GPU lattice FMM: the
GMRES solution mu on the modified nodes equals the dense oracle solve, the potential
u = v - S (B v + mu) equals the oracle's, and (A + B) u = 0 around the modifications."""
import numpy as np
import pytest

import oracle
from oracle import inclusions as inc
from paper_1105_3505_gb300 import build

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


def random_bars(seed, n, box):
    """n changed bars of the unit lattice in [0, box)^2: removed, strengthened or weakened
    lattice bars and a few new diagonal bars; distinct."""
    rng = np.random.default_rng(seed)
    seen, bars, delta = set(), [], []
    while len(bars) < n:
        x, y = (int(v) for v in rng.integers(0, box, size=2))
        kind = rng.integers(0, 4)
        if kind == 0:
            bx, by, d = x + 1, y, -1.0
        elif kind == 1:
            bx, by, d = x, y + 1, float(rng.uniform(-0.9, 3.0))
        elif kind == 2:
            bx, by, d = x + 1, y, float(rng.uniform(-0.9, 3.0))
        else:
            bx, by, d = x + 1, y + 1, float(rng.uniform(0.2, 2.0))
        key = (x, y, bx, by)
        if key in seen:
            continue
        seen.add(key)
        bars.append(key)
        delta.append(d)
    return np.array(bars, dtype=np.int64), np.array(delta)


@pytest.mark.parametrize("n_bars,box", [(6, 10), (300, 64)])
def test_inclusions_match_dense_oracle(lfmm, n_bars, box):
    from paper_1105_3505_gb300.inclusions import LatticeInclusions
    bars, delta = random_bars(n_bars, n_bars, box)
    c1, c2 = 0.4, 1.1
    nodes, mu_ref, Bv_ref = inc.solve_dense(bars, delta, c1, c2)
    li = LatticeInclusions(bars, delta)
    try:
        mu = li.solve(c1, c2, tol=1e-12)
        assert np.array_equal(li.nodes, nodes.astype(np.int32))
        assert li.residual <= 1e-11, (li.iterations, li.residual)
        assert np.abs(mu - mu_ref).max() <= 1e-9 * np.abs(mu_ref).max()
        # potential near and far from the modifications, and the lattice equation
        rng = np.random.default_rng(1)
        centres = [tuple(p) for p in rng.integers(-5, box + 5, size=(40, 2))] + [(box * 20, -box * 15)]
        pts = sorted({(x + dx, y + dy) for x, y in centres for dx, dy in [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]}
                     | {tuple(p) for p in nodes})
        u = li.potential(np.array(pts))
        u_ref = inc.potential(nodes, mu_ref, Bv_ref, c1, c2, np.array(pts))
        w_scale = np.abs(u_ref - (c1 * np.array(pts)[:, 0] + c2 * np.array(pts)[:, 1])).max()
        assert np.abs(u - u_ref).max() <= 1e-9 * w_scale
        u_of = {p: val for p, val in zip(pts, u)}
        for m in centres:
            r = oracle.apply_A(u_of, m)
            for (ax, ay, bx, by), d in zip(bars, delta):
                if (ax, ay) == m:
                    r += d * (u_of[(ax, ay)] - u_of[(bx, by)])
                if (bx, by) == m:
                    r += d * (u_of[(bx, by)] - u_of[(ax, ay)])
            assert abs(r) <= 1e-8 * max(1.0, w_scale), (m, r)
    finally:
        li.close()


def test_inclusions_mixed_path(lfmm):
    """The mixed path as the operator: mu to its ~1e-6 accuracy."""
    from paper_1105_3505_gb300.inclusions import LatticeInclusions
    bars, delta = random_bars(7, 300, 64)
    nodes, mu_ref, _ = inc.solve_dense(bars, delta, 1.0, 0.0)
    li = LatticeInclusions(bars, delta, precision=lfmm.LFMM_MIXED, p=8)
    try:
        mu = li.solve(1.0, 0.0, tol=1e-8)
        assert np.abs(mu - mu_ref).max() <= 1e-5 * np.abs(mu_ref).max()
    finally:
        li.close()
