"""Dirichlet problems on finite lattice domains (Sec. 10.2) through the GPU lattice FMM:
the GMRES density equals the dense oracle solve, the solution on the interior equals
the oracle's double layer, the unit density gives D 1 = -1, and on a digital disk with
about seven million interior nodes harmonic boundary data is reproduced and A u = 0."""
import numpy as np
import pytest

import oracle
from oracle import bvp as obvp
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


def rect(nx, ny, x0=0, y0=0):
    return np.array([(x0 + x, y0 + y) for x in range(nx) for y in range(ny)])


def disk(r, cx=0, cy=0):
    x, y = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    keep = x * x + y * y <= r * r
    return np.stack([x[keep] + cx, y[keep] + cy], axis=1)


def notched(n):
    """A square with a slot cut in from one side (a non-convex, simply connected domain)."""
    return np.array([(x, y) for x in range(n) for y in range(n) if not (n // 3 <= x < n // 3 + 3 and y >= n // 4)])


@pytest.mark.parametrize("name,nodes", [("rect", rect(41, 29, -7, 12)), ("disk", disk(23, 300, -40)),
                                        ("notched", notched(36))])
def test_bvp_matches_dense_oracle(lfmm, name, nodes):
    from paper_1105_3505_gb300.bvp import LatticeDirichlet
    gamma, omega, edges = obvp.boundary_of(nodes)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(gamma.shape[0])
    _, _, _, q_ref = obvp.solve_dense(nodes, g)
    bv = LatticeDirichlet(nodes)
    try:
        assert np.array_equal(bv.gamma, gamma) and np.array_equal(bv.omega, omega)
        # the unit density: D 1 = -1 on the boundary
        assert np.abs(bv.apply_D(np.ones(gamma.shape[0])) + 1.0).max() <= 1e-12
        # GMRES to 1e-12 (the float-float operator is accurate to ~1e-13, so tighter
        # tolerances stagnate); the boundary equation's condition number is below 100
        # (61 for the notched square), so q and u are good to ~1e-10
        q = bv.solve(g, tol=1e-12)
        assert bv.iterations < 80, bv.iterations
        assert np.abs(q - q_ref).max() <= 1e-9 * np.abs(q_ref).max()
        u = bv.potential()
        u_ref = obvp.apply_D(gamma, edges, q_ref, omega)
        assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(g).max()
    finally:
        bv.close()


def test_bvp_large_disk_harmonic_data(lfmm):
    """r = 1500: ~7.07e6 nodes, ~8.5e3 boundary nodes.  Data x^2 - y^2 + 3 x y + phi(m - m0)
    (m0 outside) is discrete harmonic, so u equals it on the whole interior."""
    from paper_1105_3505_gb300.bvp import LatticeDirichlet
    r = 1500
    nodes = disk(r, 250, -125)
    m0 = np.array([250 + r + 40, -125 + 17])

    def h(p):
        p = np.asarray(p, dtype=np.float64)
        x, y = p[:, 0] - 250.0, p[:, 1] + 125.0
        return (x * x - y * y + 3.0 * x * y) / r ** 2 + oracle.phi(np.asarray(p, dtype=np.int64) - m0)

    bv = LatticeDirichlet(nodes)
    try:
        q = bv.solve(h(bv.gamma), tol=1e-12)
        assert bv.iterations < 80, bv.iterations
        assert bv.residual <= 1e-12
        rng = np.random.default_rng(5)
        pick = bv.omega[rng.choice(bv.omega.shape[0], 300, replace=False)]
        # the interior sample, and the solution on the whole interior in one evaluation
        u_all = bv.potential()
        assert u_all.shape[0] == bv.omega.shape[0] > 7_000_000
        idx = np.searchsorted(bv.omega[:, 0] * (1 << 20) + bv.omega[:, 1], pick[:, 0] * (1 << 20) + pick[:, 1])
        scale = np.abs(h(bv.gamma)).max()
        assert np.abs(u_all[idx] - h(pick)).max() <= 1e-10 * scale
        # A u = 0 at the sample (the five-point stencil around each picked node)
        stencil = np.concatenate([pick] + [pick + np.array(s) for s in [(1, 0), (-1, 0), (0, 1), (0, -1)]])
        us = bv.potential(stencil).reshape(5, -1)
        assert np.abs(4.0 * us[0] - us[1:].sum(axis=0)).max() <= 1e-10 * scale
        # the oracle's dipole sum at a few nodes
        few = pick[:20]
        ref = obvp.apply_D(bv.gamma, [(int(i), tuple(o)) for i, o in zip(bv.edge_node, bv.edge_out)], q, few)
        assert np.abs(bv.potential(few) - ref).max() <= 1e-11 * scale
    finally:
        bv.close()


def test_bvp_mixed_precision(lfmm):
    from paper_1105_3505_gb300.bvp import LatticeDirichlet
    nodes = disk(60, 5, 5)
    gamma, omega, edges = obvp.boundary_of(nodes)
    g = np.cos(0.05 * gamma[:, 0]) + 0.3 * np.sin(0.11 * gamma[:, 1])
    _, _, _, q_ref = obvp.solve_dense(nodes, g)
    bv = LatticeDirichlet(nodes, precision=lfmm.LFMM_MIXED, p=8)
    try:
        q = bv.solve(g, tol=1e-7)
        assert np.abs(q - q_ref).max() <= 1e-5 * np.abs(q_ref).max()
    finally:
        bv.close()
