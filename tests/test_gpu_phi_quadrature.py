"""The GPU quadrature of Sec. 3.2 for phi near the origin (lfmm_phi_quadrature), for the
5-point operator against the oracle's exact table, and for operators with no closed
recurrence (anisotropic bars, next-nearest-neighbour bars, triangular lattices) against
the defining equation A phi = delta_0 with phi(0) = 0 and the symmetry phi(m) = phi(-m)."""
import numpy as np
import pytest

import oracle
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


def test_five_point_matches_exact_table(lfmm):
    R = 20
    tab = lfmm.lfmm_phi_quadrature([[1, 0], [0, 1]], [1.0, 1.0], R)
    ys, xs = np.mgrid[-R:R + 1, -R:R + 1]
    ref = oracle.phi(np.stack([xs.ravel(), ys.ravel()], axis=1)).reshape(tab.shape)
    assert np.abs(tab - ref).max() <= 1e-12, np.abs(tab - ref).max()
    assert tab[R, R] == 0.0
    assert abs(tab[R, R + 1] + 0.25) <= 1e-13 and abs(tab[R + 1, R + 1] + 1.0 / np.pi) <= 1e-13


@pytest.mark.parametrize("offsets,weights", [
    ([[1, 0], [0, 1]], [1.0, 2.5]),                          # anisotropic conductivities
    ([[1, 0], [0, 1], [1, 1], [1, -1]], [1.0, 1.0, 0.5, 0.5]),  # next-nearest-neighbour bars
    ([[1, 0], [0, 1], [1, 1]], [0.7, 1.3, 0.4]),             # a triangular lattice
    ([[1, 0], [0, 1]], [1.0, 20.0]),                         # strongly anisotropic (split 3 x 3)
    ([[1, 0], [0, 1], [1, 1]], [0.1, 0.1, 3.0]),             # nearly degenerate along (1, 1)
])
def test_general_operator_satisfies_its_equation(lfmm, offsets, weights):
    R = 16
    tab = lfmm.lfmm_phi_quadrature(offsets, weights, R)
    assert tab[R, R] == 0.0
    assert np.abs(tab - tab[::-1, ::-1]).max() <= 1e-13  # phi(m) = phi(-m)

    def at(x, y):
        return tab[y + R, x + R]

    worst = 0.0
    reach = max(max(abs(a), abs(b)) for a, b in offsets)
    for y in range(-R + reach, R - reach + 1):
        for x in range(-R + reach, R - reach + 1):
            a = sum(w * (2 * at(x, y) - at(x + dx, y + dy) - at(x - dx, y - dy))
                    for (dx, dy), w in zip(offsets, weights))
            worst = max(worst, abs(a - (1.0 if (x, y) == (0, 0) else 0.0)))
    # an entry error e gives a residual of at most 4 e sum(w); the 5-point table is
    # exact to ~1e-15
    assert worst <= 1e-13 * 4 * sum(weights), worst


def test_invalid_stencils_rejected(lfmm):
    with pytest.raises(lfmm.LfmmError):
        lfmm.lfmm_phi_quadrature([[2, 0], [0, 2]], [1.0, 1.0], 4)  # does not connect the lattice
    with pytest.raises(lfmm.LfmmError):
        lfmm.lfmm_phi_quadrature([[1, 0], [0, 1]], [1.0, -1.0], 4)
    with pytest.raises(lfmm.LfmmError):
        lfmm.lfmm_phi_quadrature([[1, 0], [0, 1]], [1.0, 1000.0], 4)  # too anisotropic
