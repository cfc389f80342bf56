"""Lattices with local modifications, solved densely (Sec. 10.1) - test infrastructure.

The lattice operator becomes A + B, where B collects the changed bars: a bar between
nodes a and b whose conductivity changes by delta adds delta (u(a) - u(b)) to node a
and delta (u(b) - u(a)) to node b (a removed bar: delta = -1; a new bar of
conductivity c: delta = c).  With u -> v = c1 m1 + c2 m2 at infinity and u = v + w,
(A + B) w = -B v; since S A w = w for a decaying w (S = convolution with phi),
    w + S B w = -S B v,
and with mu = B w (supported on the nodes Omega of the changed bars)
    mu + B S mu = -B S B v      on Omega,
    u = v - S (B v + mu).
(The recovery formula as printed in Sec. 10.1 carries the opposite sign in front of
mu; with mu = B w the derivation above gives the sign used here, and
tests/test_inclusions_cpu.py checks (A + B) u = 0 with it and not with the other.)

This module solves the dense system with the oracle's phi (numpy.linalg.solve) and
evaluates u by brute force: the reference the GPU solver is compared against.
"""
from __future__ import annotations

import numpy as np

from . import lattice_sum, phi


def nodes_of(bars: np.ndarray):
    """Omega (unique end nodes, sorted) and each bar's end indices into it."""
    bars = np.asarray(bars, dtype=np.int64).reshape(-1, 4)
    ends = np.concatenate([bars[:, 0:2], bars[:, 2:4]])
    nodes, inv = np.unique(ends, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    n = bars.shape[0]
    return nodes, inv[:n], inv[n:]


def apply_B(x: np.ndarray, a: np.ndarray, b: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """(B x) on Omega for x on Omega."""
    d = delta * (x[a] - x[b])
    y = np.zeros_like(x, dtype=np.float64)
    np.add.at(y, a, d)
    np.add.at(y, b, -d)
    return y


def solve_dense(bars, delta, c1: float, c2: float):
    """(nodes, mu, Bv): the dense solve of mu + B S mu = -B S B v on Omega."""
    nodes, a, b = nodes_of(bars)
    delta = np.asarray(delta, dtype=np.float64)
    n = nodes.shape[0]
    d = (nodes[:, None, :] - nodes[None, :, :]).reshape(-1, 2)
    Phi = phi(d).reshape(n, n)  # S restricted to Omega
    v = c1 * nodes[:, 0] + c2 * nodes[:, 1]
    Bv = apply_B(v, a, b, delta)
    BPhi = np.stack([apply_B(Phi[:, j], a, b, delta) for j in range(n)], axis=1)  # B S
    mu = np.linalg.solve(np.eye(n) + BPhi, -(BPhi @ Bv))
    return nodes, mu, Bv


def potential(nodes, mu, Bv, c1: float, c2: float, targets) -> np.ndarray:
    """u = v - S (B v + mu) at the targets, by brute force."""
    t = np.asarray(targets, dtype=np.int64).reshape(-1, 2)
    return c1 * t[:, 0] + c2 * t[:, 1] - lattice_sum(nodes, Bv + mu, t)
