"""The dense reference for lattices with local modifications (Sec. 10.1), pinned by the
equation itself: with mu from the dense solve, u = v - S (B v + mu) satisfies
(A + B) u = 0 at every node around the modified bars and far from them, and u - v
decays.  The other sign in front of mu violates the equation (the reading of the
recovery formula)."""
import numpy as np

import oracle
from oracle import inclusions as inc


def example():
    # three removed bars, two strengthened ones and one new diagonal bar
    bars = np.array([[0, 0, 1, 0], [1, 0, 1, 1], [5, 5, 5, 6],
                     [3, -2, 4, -2], [-4, 1, -4, 2],
                     [2, 3, 3, 4]], dtype=np.int64)
    delta = np.array([-1.0, -1.0, -1.0, 2.5, 0.75, 1.3])
    return bars, delta


def residual(u_of, bars, delta, m):
    """((A + B) u)(m) for the values in u_of (A of eq. 1.2 plus the changed bars)."""
    r = oracle.apply_A(u_of, m)
    for (ax, ay, bx, by), d in zip(bars, delta):
        if (ax, ay) == tuple(m):
            r += d * (u_of[(ax, ay)] - u_of[(bx, by)])
        if (bx, by) == tuple(m):
            r += d * (u_of[(bx, by)] - u_of[(ax, ay)])
    return r


def test_dense_solution_satisfies_the_lattice_equation():
    bars, delta = example()
    c1, c2 = 0.7, -1.2
    nodes, mu, Bv = inc.solve_dense(bars, delta, c1, c2)
    assert abs(Bv.sum()) < 1e-12 and abs(mu.sum()) < 1e-10  # B's range is zero-sum
    centres = [(x, y) for x in range(-6, 8) for y in range(-4, 9)] + [(40, -35), (-120, 90)]
    pts = sorted({(x + dx, y + dy) for x, y in centres for dx, dy in [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]}
                 | {tuple(p) for p in nodes})
    for sign in (+1.0, -1.0):
        u = inc.potential(nodes, sign * mu, Bv, c1, c2, np.array(pts))
        u_of = {p: val for p, val in zip(pts, u)}
        worst = max(abs(residual(u_of, bars, delta, m)) for m in centres)
        if sign > 0:
            assert worst < 1e-10, worst
        else:
            assert worst > 1e-3, worst
    # far away, u approaches v
    far = np.array([[3000, 0], [0, -3000]])
    u = inc.potential(nodes, mu, Bv, c1, c2, far)
    assert np.abs(u - (c1 * far[:, 0] + c2 * far[:, 1])).max() < 1e-2


def test_no_change_gives_the_linear_field():
    bars = np.array([[0, 0, 1, 0]], dtype=np.int64)
    nodes, mu, Bv = inc.solve_dense(bars, np.array([0.0]), 1.0, 2.0)
    assert np.all(mu == 0) and np.all(Bv == 0)
    t = np.array([[5, 7], [-3, 2]])
    assert np.allclose(inc.potential(nodes, mu, Bv, 1.0, 2.0, t), t[:, 0] + 2.0 * t[:, 1])
