"""Dirichlet problems on finite lattice domains by the lattice double layer (Sec. 10.2),
solved densely - test infrastructure.

A domain is a finite set D of nodes of Z^2.  Its boundary Gamma is the set of nodes of D
with at least one of their four neighbours outside D, and Omega = D minus Gamma; every
neighbour of a node of Omega lies in D.  The Dirichlet problem is A u = 0 on Omega
(A of eq. 1.2) and u = g on Gamma.

The solution operator D of Sec. 10.2 applies the difference along the outward normal to
the source variable of phi.  On the lattice the outward normals of a boundary node n are
the unit steps nu with n + nu outside D (a corner node has two), so

    (D q)(m) = sum_{n in Gamma} sum_{nu: n + nu not in D} (phi(m - n - nu) - phi(m - n)) q(n),

a sum of dipoles, each harmonic away from its two nodes n (in Gamma) and n + nu
(outside D).  A (D q) therefore vanishes on Omega, and restricting D q = g to Gamma
gives the boundary equation of Sec. 10.2 for q.  The paper states neither which nodes
form Gamma nor how the normal is taken; the reading above is the one under which the
lattice form of Gauss's lemma holds: summing A phi(m - .) = delta_m over D and cancelling
the interior bars leaves the outward boundary bars, so D 1 = -1 on D and 0 outside it.
The boundary equation is then of the second kind (its condition number stays near 7 on
rectangles, L-shapes and digital disks of every size tried).

This module forms that dense matrix with the oracle's phi, solves it with
numpy.linalg.solve, and evaluates D q by brute force: the reference the GPU solver is
compared against.  The tests pin it to a sparse direct solve of the Dirichlet problem
itself and to discrete harmonic functions.
"""
from __future__ import annotations

import numpy as np

from . import lattice_sum, phi

STEPS = ((1, 0), (-1, 0), (0, 1), (0, -1))


def boundary_of(nodes):
    """(gamma, omega, edges) for the domain D given as an (n, 2) integer array:
    gamma and omega sorted lexicographically, edges a list of (index into gamma, the
    outside neighbour) with one entry per outward bar."""
    D = {(int(x), int(y)) for x, y in np.asarray(nodes).reshape(-1, 2)}
    gamma, omega = [], []
    for p in sorted(D):
        (gamma if any((p[0] + a, p[1] + b) not in D for a, b in STEPS) else omega).append(p)
    edges = [(i, (p[0] + a, p[1] + b)) for i, p in enumerate(gamma) for a, b in STEPS
             if (p[0] + a, p[1] + b) not in D]
    return np.array(gamma, dtype=np.int64).reshape(-1, 2), np.array(omega, dtype=np.int64).reshape(-1, 2), edges


def dlp_matrix(gamma, edges, targets) -> np.ndarray:
    """d(m, n) = sum over the outward bars of n of phi(m - n - nu) - phi(m - n), for m in
    targets (rows) and n in gamma (columns)."""
    t = np.asarray(targets, dtype=np.int64).reshape(-1, 2)
    M = np.zeros((t.shape[0], gamma.shape[0]))
    for i, q in edges:
        M[:, i] += phi(t - np.asarray(q)) - phi(t - gamma[i])
    return M


def apply_D(gamma, edges, q, targets) -> np.ndarray:
    """(D q)(m) at the targets by brute force: each outward bar of n contributes
    +q(n) at its outside node and -q(n) at n."""
    src = [gamma[i] for i, _ in edges] + [np.asarray(o) for _, o in edges]
    w = [-q[i] for i, _ in edges] + [q[i] for i, _ in edges]
    return lattice_sum(np.array(src, dtype=np.int64), np.array(w, dtype=np.float64), targets)


def solve_dense(nodes, g):
    """(gamma, omega, edges, q): g given on gamma (in boundary_of's order); q solves the
    boundary equation sum_n d(m, n) q(n) = g(m), m in gamma."""
    gamma, omega, edges = boundary_of(nodes)
    q = np.linalg.solve(dlp_matrix(gamma, edges, gamma), np.asarray(g, dtype=np.float64))
    return gamma, omega, edges, q
