"""Plan-time precomputation of the library (host side, no GPU), checked against the oracle.

- phi near the origin by the 1-D integral of Remark 3.1 vs the oracle's exact table;
- eq. 3.1 far from the origin vs the oracle's independent transcription;
- skeletons and translation operators of the model boxes (Sec. 5, 7, 8.1, Remark 8.2):
  the outgoing expansion reproduces the far field of arbitrary charges in the box,
  the incoming expansion interpolates any field of well-separated sources, both to the
  accuracy Table 4.1 ties to the expansion length.
"""
import numpy as np
import pytest

import oracle
from oracle.phi_exact import phi_octant
from paper_1105_3505_gb300 import build, lfmm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lfmm.load()


def test_phi_table_matches_exact_oracle():
    lib_tab = lfmm.lfmm_phi_table(128)
    exact = phi_octant(128)
    assert np.abs(lib_tab - exact).max() <= 4.5e-16


def test_phi_far_field_matches_oracle_asymptotics():
    rng = np.random.default_rng(1)
    d = rng.integers(-10**6, 10**6, size=(500, 2))
    d = d[np.abs(d).max(axis=1) > 256]
    assert np.abs(lfmm.lfmm_phi(d) - oracle.phi(d)).max() < 2e-15
    # between the library's switch radius (128) and the oracle's (256): eq. 3.1 error bound
    d2 = np.array([[129, 0], [150, 150], [200, 17], [-256, 3]])
    r = np.hypot(d2[:, 0], d2[:, 1])
    assert np.all(np.abs(lfmm.lfmm_phi(d2) - oracle.phi(d2)) <= 0.2 / r ** 6 + 1e-15)


def _far_points(side, n, rng):
    """Lattice points outside the 3x3 block of boxes around [0, side)^2 (interaction region)."""
    pts = []
    while len(pts) < n:
        x, y = rng.integers(-3 * side, 4 * side, size=2)
        if -side <= x < 2 * side and -side <= y < 2 * side:
            continue
        pts.append((x, y))
    return np.array(pts)


@pytest.mark.parametrize("side,p,tol", [(8, 8, 1e-13), (16, 8, 2e-8), (16, 12, 1e-11), (16, 16, 1e-13),
                                        (32, 8, 2e-8), (32, 16, 1e-12)])
def test_leaf_outgoing_and_incoming(side, p, tol):
    rng = np.random.default_rng(side * 100 + p)
    sk = lfmm.lfmm_model_skeleton(side, p, 64, 0)
    T = lfmm.lfmm_model_tofs(side, p, 64)
    assert T.shape == (sk.shape[0], side * side)
    assert sk.shape[0] <= 4 * (p - 1)
    # skeleton points lie on the box boundary (Sec. 5)
    on_edge = (sk[:, 0] == 0) | (sk[:, 0] == side - 1) | (sk[:, 1] == 0) | (sk[:, 1] == side - 1)
    assert on_edge.all() or sk.shape[0] == side * side
    box = np.array([(j % side, j // side) for j in range(side * side)])
    # outgoing: charges anywhere in the box, field at well-separated points
    q = rng.standard_normal(side * side)
    X = _far_points(side, 150, rng)
    direct = np.array([(oracle.phi(x - box) * q).sum() for x in X])
    equiv = np.array([(oracle.phi(x - sk) * (T @ q)).sum() for x in X])
    assert np.abs(direct - equiv).max() <= tol * np.abs(direct).max()
    # incoming: well-separated sources, field inside the box interpolated from the skeleton
    Y = _far_points(side, 40, rng)
    fy = rng.standard_normal(40)
    u_box = np.array([(oracle.phi(x - Y) * fy).sum() for x in box])
    u_sk = np.array([(oracle.phi(x - Y) * fy).sum() for x in sk])
    assert np.abs(T.T @ u_sk - u_box).max() <= 4 * tol * np.abs(u_box).max()


@pytest.mark.parametrize("p,k,tol", [(8, 1, 5e-8), (8, 4, 5e-8), (16, 1, 1e-13), (16, 4, 1e-13)])
def test_parent_from_children(p, k, tol):
    """T_ofo = column blocks of S: the parent's expansion reproduces the children's far field."""
    side0 = 16
    rng = np.random.default_rng(7 * k + p)
    skp = lfmm.lfmm_model_skeleton(side0, p, 64, k)
    skc = lfmm.lfmm_model_skeleton(side0, p, 64, k - 1)
    S = lfmm.lfmm_model_s(side0, p, 64, k)
    side = side0 << k
    half = side // 2
    Y = np.concatenate([skc + [(c & 1) * half, (c >> 1) * half] for c in range(4)])
    assert S.shape == (skp.shape[0], Y.shape[0])
    # the parent skeleton is a subset of the children's (Sec. 7)
    assert {tuple(v) for v in skp} <= {tuple(v) for v in Y}
    qc = rng.standard_normal(Y.shape[0])
    X = _far_points(side, 120, rng)
    direct = np.array([(oracle.phi(x - Y) * qc).sum() for x in X])
    equiv = np.array([(oracle.phi(x - skp) * (S @ qc)).sum() for x in X])
    assert np.abs(direct - equiv).max() <= tol * np.abs(direct).max()


def test_expansion_length_against_table_4_1():
    """Table 4.1: ~27 skeleton points reach 1e-8 and ~49 reach 1e-13; our lengths 4(p-1) = 28
    and 60 (capped by numerical rank) do at least as well (the tests above), and the
    numerical rank at 1e-14 stays near Table 4.1's 1e-13 column."""
    for k in range(1, 5):
        n = lfmm.lfmm_model_skeleton(16, 16, 64, k).shape[0]
        assert 49 <= n <= 60
