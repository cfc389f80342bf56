"""Dirichlet problems on finite lattice domains (Sec. 10.2), with the lattice FMM
applying the double-layer operator D.

The domain is a finite set D of nodes of Z^2 without holes (its complement is
4-connected).  Gamma = nodes of D with a neighbour outside D, Omega = the rest; the
problem is A u = 0 on Omega (A of eq. 1.2), u = g on Gamma.  The outward normals of a
boundary node n are the unit steps nu with n + nu outside D (two at a convex corner), and

    (D q)(m) = sum_{n in Gamma} sum_{nu} (phi(m - n - nu) - phi(m - n)) q(n),

so D q is one lattice sum with a charge -k(n) q(n) on each boundary node (k(n) its number
of outward bars) and the sum of q over the adjacent boundary nodes on each outside node.
A (D q) = 0 on Omega; the boundary equation D q = g on Gamma is of the second kind (the
unit density gives D 1 = -1 on D, 0 outside) and restarted GMRES converges in a number of
iterations that does not grow with the domain.  Each iteration is one evaluation of an
lfmm plan (dipole nodes as sources, Gamma as targets) replayed as a recorded CUDA graph;
the solution on Omega, or anywhere, is one more evaluation.

A domain with a hole makes the unit density on the hole's boundary a null vector of the
boundary equation; such domains are rejected.  The O(N_Gamma) direct inversion of the
boundary equation that Sec. 10.2 refers to is not part of this module: GMRES takes its
place.
"""
from __future__ import annotations

import numpy as np

from . import lfmm
from .inclusions import gmres

_STEPS = ((1, 0), (-1, 0), (0, 1), (0, -1))


def _grid(nodes: np.ndarray):
    """Occupancy grid of the bounding box padded by one node: (grid[y, x], x0, y0)."""
    xs, ys = nodes[:, 0], nodes[:, 1]
    lo = np.array([xs.min(), ys.min()]) - 1
    hi = np.array([xs.max(), ys.max()]) + 1
    grid = np.zeros((int(hi[1] - lo[1] + 1), int(hi[0] - lo[0] + 1)), dtype=bool)
    grid[ys - lo[1], xs - lo[0]] = True
    return grid, int(lo[0]), int(lo[1])


def boundary_of(nodes):
    """(gamma, omega, edge_node, edge_out) for the domain given as (n, 2) integer nodes.
    gamma and omega are sorted by (x, y); edge_node[k] indexes gamma and edge_out[k] is
    the outside node of outward bar k.  Raises ValueError for an empty domain, repeated
    nodes, or a domain with holes."""
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1, 2)
    if nodes.shape[0] == 0:
        raise ValueError("empty domain")
    grid, x0, y0 = _grid(nodes)
    if int(grid.sum()) != nodes.shape[0]:
        raise ValueError("repeated nodes in the domain")
    outside = ~grid
    try:
        from scipy import ndimage
        _, n_comp = ndimage.label(outside)  # 4-connectivity by default
    except ImportError:  # pragma: no cover - scipy is present where this runs
        n_comp = _count_components(outside)
    if n_comp != 1:
        raise ValueError("the domain has holes: its boundary equation is singular")
    interior = grid.copy()
    interior[1:-1, 1:-1] &= grid[1:-1, 2:] & grid[1:-1, :-2] & grid[2:, 1:-1] & grid[:-2, 1:-1]
    is_gamma = grid & ~interior

    def sorted_xy(mask):
        xs, ys = np.nonzero(mask.T)  # row-major over (x, y): sorted by x, then y
        out = np.empty((xs.shape[0], 2), dtype=np.int64)
        out[:, 0] = xs + x0
        out[:, 1] = ys + y0
        return out

    gamma, omega = sorted_xy(is_gamma), sorted_xy(grid & interior)
    gy, gx = gamma[:, 1] - y0, gamma[:, 0] - x0
    edge_node, edge_out = [], []
    for a, b in _STEPS:
        out = ~grid[gy + b, gx + a]
        k = np.nonzero(out)[0]
        edge_node.append(k)
        edge_out.append(gamma[k] + np.array([a, b]))
    edge_node = np.concatenate(edge_node)
    edge_out = np.concatenate(edge_out)
    order = np.lexsort((edge_out[:, 1], edge_out[:, 0], edge_node))
    return gamma, omega, edge_node[order], edge_out[order]


def _count_components(mask: np.ndarray) -> int:
    seen = np.zeros_like(mask)
    n = 0
    H, W = mask.shape
    for y0, x0 in zip(*np.nonzero(mask)):
        if seen[y0, x0]:
            continue
        n += 1
        stack = [(y0, x0)]
        seen[y0, x0] = True
        while stack:
            y, x = stack.pop()
            for dx, dy in _STEPS:
                yy, xx = y + dy, x + dx
                if 0 <= yy < H and 0 <= xx < W and mask[yy, xx] and not seen[yy, xx]:
                    seen[yy, xx] = True
                    stack.append((yy, xx))
    return n


class LatticeDirichlet:
    """A u = 0 on the interior of the domain `nodes` ((n, 2) int), u = g on its boundary.
    solve(g) finds the double-layer density q on the boundary; potential(targets) gives
    u = D q (by default on the interior nodes)."""

    def __init__(self, nodes, precision: int = lfmm.LFMM_DF, p: int = 16):
        self.gamma, self.omega, self.edge_node, self.edge_out = boundary_of(nodes)
        ng = self.gamma.shape[0]
        # dipole nodes: the boundary nodes, then the distinct outside nodes
        outs, self._out_of_edge = np.unique(self.edge_out, axis=0, return_inverse=True)
        self._out_of_edge = self._out_of_edge.reshape(-1)
        self.sources = np.ascontiguousarray(np.concatenate([self.gamma, outs]).astype(np.int32))
        self._k = np.bincount(self.edge_node, minlength=ng).astype(np.float64)
        self._n_out = outs.shape[0]
        self.precision, self.p = precision, p
        self.plan = lfmm.Plan(self.sources, np.ascontiguousarray(self.gamma.astype(np.int32)),
                              precision=precision, p=p, graph=True)
        self.q = None
        self.iterations = 0
        self.residual = None

    def charges(self, q: np.ndarray) -> np.ndarray:
        """The lattice-sum charges of the double layer with density q."""
        q = np.asarray(q, dtype=np.float64)
        c_out = np.bincount(self._out_of_edge, weights=q[self.edge_node], minlength=self._n_out)
        return np.concatenate([-self._k * q, c_out])

    def apply_D(self, q: np.ndarray) -> np.ndarray:
        """(D q) on the boundary nodes."""
        return self.plan.eval(self.charges(q))

    def solve(self, g, tol: float = 1e-12, restart: int = 60, maxiter: int = 600) -> np.ndarray:
        """The density q with D q = g on the boundary (g in the order of self.gamma)."""
        g = np.asarray(g, dtype=np.float64).reshape(-1)
        if g.shape[0] != self.gamma.shape[0]:
            raise ValueError("one boundary value per boundary node")
        self.q, self.iterations, self.residual = gmres(self.apply_D, g, tol, restart, maxiter)
        return self.q

    def potential(self, targets=None) -> np.ndarray:
        """u = D q at the targets ((n, 2) int; default: the interior nodes)."""
        if self.q is None:
            raise RuntimeError("solve() first")
        t = self.omega if targets is None else np.asarray(targets).reshape(-1, 2)
        if t.shape[0] == 0:
            return np.zeros(0)
        t = np.ascontiguousarray(t.astype(np.int32))
        with lfmm.Plan(self.sources, t, precision=self.precision, p=self.p) as pl:
            return pl.eval(self.charges(self.q))

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None
