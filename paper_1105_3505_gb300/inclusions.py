"""Lattices with local modifications (Sec. 10.1), with the lattice FMM as the solution
operator S.

A changed bar between nodes a and b (conductivity change delta: -1 removes a lattice
bar, c adds a new bar of conductivity c) adds delta (u(a) - u(b)) at a and
delta (u(b) - u(a)) at b: the operator B.  With u -> v = c1 m1 + c2 m2 at infinity,
mu = B (u - v) solves the dense equation on the nodes Omega of the changed bars

    mu + B S mu = -B S B v,

and u = v - S (B v + mu) everywhere (the derivation, and the sign in front of mu, are
in oracle/inclusions.py).  Every application of S is one evaluation of an lfmm plan
with Omega as sources and targets, replayed as a recorded CUDA graph; the Krylov
iteration (restarted GMRES with modified Gram-Schmidt and Givens rotations) works on
the |Omega| host values between those evaluations.
"""
from __future__ import annotations

import numpy as np

from . import lfmm


class LatticeInclusions:
    """Changed bars `bars` (n, 4) int (ax, ay, bx, by) with conductivity changes
    `delta` (n,).  solve(c1, c2) finds mu; potential(targets) evaluates u."""

    def __init__(self, bars, delta, precision: int = lfmm.LFMM_DF, p: int = 16):
        bars = np.asarray(bars, dtype=np.int64).reshape(-1, 4)
        self.delta = np.asarray(delta, dtype=np.float64).reshape(-1)
        if self.delta.shape[0] != bars.shape[0]:
            raise ValueError("one conductivity change per bar")
        ends = np.concatenate([bars[:, 0:2], bars[:, 2:4]])
        nodes, inv = np.unique(ends, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        self.nodes = np.ascontiguousarray(nodes.astype(np.int32))
        self.a, self.b = inv[:bars.shape[0]], inv[bars.shape[0]:]
        self.precision, self.p = precision, p
        self.plan = lfmm.Plan(self.nodes, self.nodes, precision=precision, p=p, graph=True)
        self.mu = None
        self.Bv = None
        self.iterations = 0
        self.residual = None

    def apply_B(self, x: np.ndarray) -> np.ndarray:
        d = self.delta * (x[self.a] - x[self.b])
        y = np.zeros(self.nodes.shape[0])
        np.add.at(y, self.a, d)
        np.add.at(y, self.b, -d)
        return y

    def apply_S(self, x: np.ndarray) -> np.ndarray:
        return self.plan.eval(np.ascontiguousarray(x, dtype=np.float64))

    def solve(self, c1: float, c2: float, tol: float = 1e-12, restart: int = 60, maxiter: int = 600):
        v = c1 * self.nodes[:, 0] + c2 * self.nodes[:, 1]
        self.c = (c1, c2)
        self.Bv = self.apply_B(v.astype(np.float64))
        rhs = -self.apply_B(self.apply_S(self.Bv))
        self.mu, self.iterations, self.residual = gmres(lambda m: m + self.apply_B(self.apply_S(m)), rhs, tol,
                                                        restart, maxiter)
        return self.mu

    def potential(self, targets) -> np.ndarray:
        """u = v - S (B v + mu) at the targets (n, 2) int."""
        if self.mu is None:
            raise RuntimeError("solve() first")
        t = np.ascontiguousarray(np.asarray(targets).reshape(-1, 2).astype(np.int32))
        with lfmm.Plan(self.nodes, t, precision=self.precision, p=self.p) as pl:
            s = pl.eval(self.Bv + self.mu)
        c1, c2 = self.c
        return c1 * t[:, 0] + c2 * t[:, 1] - s

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None


def gmres(matvec, b: np.ndarray, tol: float, restart: int, maxiter: int):
    """Restarted GMRES for matvec(x) = b from x = 0: (x, iterations, relative residual)."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    rel = 1.0
    while it < maxiter:
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= tol:
            break
        m = min(restart, maxiter - it)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for k in range(m):
            w = matvec(V[k])
            it += 1
            for i in range(k + 1):  # modified Gram-Schmidt
                H[i, k] = V[i] @ w
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):  # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = (1.0, 0.0) if den == 0.0 else (H[k, k] / den, H[k + 1, k] / den)
            H[k, k] = cs[k] * H[k, k] + sn[k] * H[k + 1, k]
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            rel = abs(g[k + 1]) / bnorm
            if rel <= tol:
                break
        kk = k + 1
        y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
        x = x + V[:kk].T @ y
        r = b - matvec(x)
        it += 1
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            break
    return x, it, rel
