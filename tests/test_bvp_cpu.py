"""The dense reference for Dirichlet problems on finite lattice domains (Sec. 10.2),
pinned by things other than itself:
  - the lattice Gauss lemma: the double layer of the unit density is -1 on the domain and
    0 outside it (this fixes which nodes form the boundary and how the normals are taken;
    a corner with one normal fails it);
  - a sparse direct solve (scipy.sparse.linalg.spsolve) of A u = 0 on Omega, u = g on
    Gamma, for random boundary data;
  - discrete harmonic functions (x^2 - y^2, x y, affine, phi(m - m0) with m0 outside the
    domain) reproduced exactly;
  - the boundary equation stays well conditioned as the domain grows, and is singular for
    a domain with a hole (which the library rejects)."""
import numpy as np
import pytest

import oracle
from oracle import bvp

sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")


def rect(nx, ny, x0=0, y0=0):
    return np.array([(x0 + x, y0 + y) for x in range(nx) for y in range(ny)])


def l_shape(n):
    return np.array([(x, y) for x in range(n) for y in range(n) if not (x >= n // 2 and y >= n // 2)])


def disk(r, cx=0, cy=0):
    return np.array([(cx + x, cy + y) for x in range(-r, r + 1) for y in range(-r, r + 1) if x * x + y * y <= r * r])


DOMAINS = {"rect": lambda: rect(23, 14, -5, 3), "L": lambda: l_shape(20), "disk": lambda: disk(11, 4, -2)}


def sparse_dirichlet(nodes, g_of):
    """u on Omega from the 5-point equations A u = 0 on Omega with u = g on Gamma."""
    gamma, omega, _ = bvp.boundary_of(nodes)
    idx = {tuple(p): i for i, p in enumerate(omega)}
    rows, cols, vals, rhs = [], [], [], np.zeros(len(omega))
    for i, p in enumerate(omega):
        rows.append(i)
        cols.append(i)
        vals.append(4.0)
        for a, b in bvp.STEPS:
            q = (int(p[0]) + a, int(p[1]) + b)
            if q in idx:
                rows.append(i)
                cols.append(idx[q])
                vals.append(-1.0)
            else:
                rhs[i] += g_of[q]
    M = sp.csr_matrix((vals, (rows, cols)), shape=(len(omega), len(omega)))
    return omega, spla.spsolve(M.tocsc(), rhs)


def ring_outside(nodes, width=3):
    D = {tuple(p) for p in nodes}
    lo, hi = nodes.min(0) - width, nodes.max(0) + width
    return np.array([(x, y) for x in range(lo[0], hi[0] + 1) for y in range(lo[1], hi[1] + 1) if (x, y) not in D])


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_gauss_lemma(name):
    nodes = DOMAINS[name]()
    gamma, omega, edges = bvp.boundary_of(nodes)
    q = np.ones(gamma.shape[0])
    inside = bvp.apply_D(gamma, edges, q, nodes)
    outside = bvp.apply_D(gamma, edges, q, np.concatenate([ring_outside(nodes), [[500, -300], [-2000, 40]]]))
    assert np.abs(inside + 1.0).max() <= 1e-12
    assert np.abs(outside).max() <= 1e-12
    # the dense matrix agrees with the dipole sum
    M = bvp.dlp_matrix(gamma, edges, nodes)
    assert np.abs(M.sum(axis=1) + 1.0).max() <= 1e-12


def test_gauss_lemma_needs_both_corner_normals():
    nodes = rect(9, 7)
    gamma, _, edges = bvp.boundary_of(nodes)
    corner = [k for k, (i, _) in enumerate(edges) if sum(1 for j, _ in edges if j == i) == 2]
    assert len(corner) == 8  # four corners, two outward bars each
    one_normal = [e for k, e in enumerate(edges) if k != corner[0]]
    inside = bvp.apply_D(gamma, one_normal, np.ones(gamma.shape[0]), nodes)
    assert np.abs(inside + 1.0).max() > 1e-3


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_dense_solve_matches_sparse_direct_dirichlet(name):
    nodes = DOMAINS[name]()
    gamma, omega, edges = bvp.boundary_of(nodes)
    rng = np.random.default_rng(7)
    g = rng.standard_normal(gamma.shape[0])
    _, _, _, q = bvp.solve_dense(nodes, g)
    u = bvp.apply_D(gamma, edges, q, omega)
    om2, u_ref = sparse_dirichlet(nodes, {tuple(p): v for p, v in zip(gamma, g)})
    assert np.array_equal(om2, omega)
    assert np.abs(u - u_ref).max() <= 1e-10 * np.abs(g).max()
    # and D q = g on the boundary
    assert np.abs(bvp.apply_D(gamma, edges, q, gamma) - g).max() <= 1e-11 * np.abs(g).max()


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_harmonic_data_reproduced(name):
    nodes = DOMAINS[name]()
    gamma, omega, edges = bvp.boundary_of(nodes)
    m0 = nodes.max(0) + np.array([3, 2])  # outside the domain
    fns = [lambda p: p[:, 0] ** 2 - p[:, 1] ** 2 + 3.0 * p[:, 0] * p[:, 1],
           lambda p: 2.0 * p[:, 0] - p[:, 1] + 5.0,
           lambda p: oracle.phi(p - m0)]
    for fn in fns:
        _, _, _, q = bvp.solve_dense(nodes, fn(gamma).astype(np.float64))
        u = bvp.apply_D(gamma, edges, q, omega)
        ex = fn(omega)
        assert np.abs(u - ex).max() <= 1e-11 * max(1.0, np.abs(ex).max())


def test_conditioning_and_holes():
    conds = []
    for n in (10, 20, 40):
        nodes = rect(n, (3 * n) // 4)
        gamma, _, edges = bvp.boundary_of(nodes)
        conds.append(np.linalg.cond(bvp.dlp_matrix(gamma, edges, gamma)))
    assert max(conds) < 10.0 and max(conds) - min(conds) < 0.5
    # a hole makes the unit density on the hole's boundary a null vector
    holed = np.array([(x, y) for x in range(16) for y in range(12) if not (5 <= x < 10 and 4 <= y < 8)])
    gamma, _, edges = bvp.boundary_of(holed)
    s = np.linalg.svd(bvp.dlp_matrix(gamma, edges, gamma), compute_uv=False)
    assert s[-1] < 1e-12 * s[0]


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_library_boundary_matches_oracle(name):
    """The library's host-side boundary detection (grid based) against the oracle's
    (set based): same boundary and interior nodes, same outward bars."""
    from paper_1105_3505_gb300 import bvp as lib_bvp
    nodes = DOMAINS[name]()
    gamma, omega, edges = bvp.boundary_of(nodes)
    g2, o2, en, eo = lib_bvp.boundary_of(nodes[::-1])
    assert np.array_equal(g2, gamma) and np.array_equal(o2, omega)
    assert sorted((int(i), tuple(int(v) for v in o)) for i, o in zip(en, eo)) == \
        sorted((i, tuple(o)) for i, o in edges)


def test_library_rejects_holes_and_bad_domains():
    from paper_1105_3505_gb300 import bvp as lib_bvp
    holed = np.array([(x, y) for x in range(16) for y in range(12) if not (5 <= x < 10 and 4 <= y < 8)])
    with pytest.raises(ValueError, match="holes"):
        lib_bvp.boundary_of(holed)
    with pytest.raises(ValueError, match="empty"):
        lib_bvp.boundary_of(np.zeros((0, 2), dtype=np.int64))
    with pytest.raises(ValueError, match="repeated"):
        lib_bvp.boundary_of(np.array([[0, 0], [0, 0], [1, 0]]))
    # a single node is its own boundary with four outward bars; two disjoint squares are fine
    g, o, en, _ = lib_bvp.boundary_of(np.array([[3, -4]]))
    assert g.tolist() == [[3, -4]] and o.shape[0] == 0 and en.tolist() == [0, 0, 0, 0]
    lib_bvp.boundary_of(np.concatenate([rect(4, 4), rect(4, 4, 10, 0)]))
