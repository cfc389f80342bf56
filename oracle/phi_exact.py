"""Exact lattice fundamental solution on a finite octant (oracle; test infrastructure).

The oracle is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library.

phi is the fundamental solution of the 5-point discrete Laplacian (Sec. 1,
eq. 1.2) normalised by the Fourier integral of eq. 1.8, hence

    phi(0) = 0,   (A phi)(m) = delta_{m,0}.

Every value lies in Q + Q/pi.  This module computes the octant
0 <= n <= m <= R exactly, as phi(m, n) = a/4 + b/(D pi) with integers a, b and
D = lcm(1, 3, 5, ..., 2R-1), and rounds each value to binary64 once.

Steps (the classical lattice Green's function recursion; not a formula of the
paper, whose own evaluation routes are quadrature, Sec. 3.2 / Remark 3.1):

  1. diagonal:        phi(k, k) = -(1/pi) * sum_{j=1..k} 1/(2j-1)
  2. first neighbour: phi(1, 0) = -1/4       (A phi = delta at 0 + D4 symmetry)
  3. off-diagonal d = m - n = 1:  phi(k+1, k) = 2 phi(k, k) - phi(k, k-1)
                                   ((A phi)(k, k) = 0 and phi(m, n) = phi(n, m))
  4. d >= 2: (A phi)(m-1, n) = 0 solved for phi(m, n):
        phi(m, n) = 4 phi(m-1, n) - phi(m-2, n) - phi(m-1, n+1) - phi(m-1, n-1)
     with phi(m, -1) = phi(m, 1).

The recursion is exact (integer arithmetic); it loses ~0.8 decimal digits per
lattice step in floating point, which is why nothing here is floating point
until the final rounding.  Pins (tests/test_oracle_phi.py): the closed forms of
phi(e1), phi(1,1), phi(2,0); eq. 1.8 by 2-D quadrature; Remark 3.1's 1-D
integral; the asymptotic expansion eq. 3.1 at large |m|.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import gcd

import numpy as np


def _lcm_odd(R: int) -> int:
    D = 1
    for j in range(1, R + 1):
        q = 2 * j - 1
        D = D * q // gcd(D, q)
    return D


def _pi_fraction(bits: int) -> Fraction:
    """pi to ~2^-bits by Machin's formula pi = 16 atan(1/5) - 4 atan(1/239),
    evaluated in integer fixed point with 32 guard bits."""
    scale_bits = bits + 32
    one = 1 << scale_bits

    def atan_inv(x: int) -> int:
        x2 = x * x
        term = one // x
        total = term
        k = 1
        sign = -1
        while term:
            term //= x2
            total += sign * (term // (2 * k + 1))
            sign = -sign
            k += 1
        return total

    return Fraction(16 * atan_inv(5) - 4 * atan_inv(239), one)


def octant_index(hi: int, lo: int) -> int:
    """Index of phi(hi, lo), 0 <= lo <= hi, in the packed octant array."""
    return hi * (hi + 1) // 2 + lo


@lru_cache(maxsize=None)
def exact_octant(R: int):
    """Integer pairs (a, b) with phi(m, n) = a/4 + b/(D*pi) for 0 <= n <= m <= R.

    Returns (a_list, b_list, D) in packed octant order (octant_index)."""
    if R < 1:
        raise ValueError("R must be >= 1")
    D = _lcm_odd(R)
    size = octant_index(R, R) + 1
    A = [0] * size
    B = [0] * size
    idx = octant_index

    def get(m: int, n: int):
        m, n = abs(m), abs(n)
        if n > m:
            m, n = n, m
        k = idx(m, n)
        return A[k], B[k]

    # 1. diagonal closed form
    harm = 0
    for k in range(1, R + 1):
        harm += D // (2 * k - 1)
        A[idx(k, k)] = 0
        B[idx(k, k)] = -harm
    # 2. phi(1, 0) = -1/4
    A[idx(1, 0)] = -1
    B[idx(1, 0)] = 0
    # 3. first off-diagonal
    for k in range(1, R):
        a1, b1 = get(k, k)
        a0, b0 = get(k, k - 1)
        A[idx(k + 1, k)] = 2 * a1 - a0
        B[idx(k + 1, k)] = 2 * b1 - b0
    # 4. remaining off-diagonals, d = m - n >= 2, increasing n within a diagonal
    for d in range(2, R + 1):
        for n in range(0, R - d + 1):
            m = n + d
            a1, b1 = get(m - 1, n)
            a2, b2 = get(m - 2, n)
            a3, b3 = get(m - 1, n + 1)
            a4, b4 = get(m - 1, n - 1)
            A[idx(m, n)] = 4 * a1 - a2 - a3 - a4
            B[idx(m, n)] = 4 * b1 - b2 - b3 - b4
    return tuple(A), tuple(B), D


def exact_value(a: int, b: int, D: int, inv_pi: Fraction) -> Fraction:
    return Fraction(a, 4) + Fraction(b, D) * inv_pi


@lru_cache(maxsize=None)
def phi_octant(R: int = 128) -> np.ndarray:
    """binary64 phi on the packed octant 0 <= lo <= hi <= R (correctly rounded)."""
    A, B, D = exact_octant(R)
    mag = max(max(abs(x) for x in A).bit_length(), max(abs(x) for x in B).bit_length())
    inv_pi = 1 / _pi_fraction(mag + D.bit_length() + 128)
    out = np.empty(len(A), dtype=np.float64)
    for k in range(len(A)):
        out[k] = float(exact_value(A[k], B[k], D, inv_pi))
    out.setflags(write=False)
    return out


def phi_exact_fraction(m: int, n: int, R: int | None = None):
    """(a/4, b/D) as Fractions such that phi(m, n) = a/4 + (b/D)/pi, exactly."""
    m, n = abs(m), abs(n)
    if n > m:
        m, n = n, m
    R = max(m, 1) if R is None else R
    A, B, D = exact_octant(R)
    k = octant_index(m, n)
    return Fraction(A[k], 4), Fraction(B[k], D)
