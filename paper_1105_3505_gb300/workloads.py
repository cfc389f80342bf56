"""Seeded synthetic inputs for the lattice sum (shared by tests, bench and oracle runs).

This module holds input generation only, none of the method's arithmetic, so
that the CUDA path and the CPU oracle can be fed identical inputs.  All draws use
numpy's PCG64 ``default_rng(seed)``.

Workload recipes (the paper's experiments, Sec. 9, are synthetic too: uniform
random loads, loads on a curve, dense loads):

  uniform_4k     4,096 distinct points drawn without replacement from [0,256)^2,
                 targets = sources, seed 0.
  uniform_1m     2^20 distinct sources uniform in [0,4096)^2 and 2^20 distinct
                 targets drawn independently in the same box, seed 1.
  clustered_4m   4,194,304 distinct points: 41,943 on 16 segments of length
                 4,000 (centres uniform in [0,65536)^2, angle uniform in [0,pi),
                 parameter uniform along the segment, rounded) and the rest in 64
                 Gaussian clusters (sigma = 200, centres uniform in [0,65536)^2,
                 rounded, not clipped), targets = sources, seed 2.
  forest_4096    4,096 independent problems, N log-uniform in [512, 8192],
                 distinct points uniform in a box of side ceil(4 sqrt(N)),
                 targets = sources, seed 3.
  serve_stream   Poisson arrivals at a given rate; per request N_src log-uniform
                 in [1e3, 1e6] (uniform, or 4 Gaussian clusters of sigma side/16),
                 box side ceil(4 sqrt(N_src)), N_tgt = N_src/4 random lattice
                 points in the box, tolerance 1e-6 or 1e-10 with equal odds,
                 seed 4.

Charges f ~ N(0,1) (U(-1,1) for clustered_4m) are shifted to sum to zero: the
mean is subtracted and the last entry is then set to minus the exactly rounded
sum (math.fsum) of the others.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def zero_sum(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    f = f - f.mean()
    f[-1] = -math.fsum(f[:-1])
    return f


def distinct_in_box(rng: np.random.Generator, n: int, side: int, x0: int = 0, y0: int = 0) -> np.ndarray:
    """n distinct lattice points uniform in [x0, x0+side) x [y0, y0+side), as int32 (n, 2)."""
    cells = side * side
    if n > cells:
        raise ValueError("more points than lattice cells")
    idx = rng.choice(cells, size=n, replace=False)
    pts = np.empty((n, 2), dtype=np.int32)
    pts[:, 0] = x0 + idx % side
    pts[:, 1] = y0 + idx // side
    return pts


def _take_new(cand: np.ndarray, seen: set, need: int) -> np.ndarray:
    """Up to `need` candidates not drawn before, in draw order; records them in `seen`."""
    key = (cand[:, 0].astype(np.int64) << 32) ^ (cand[:, 1].astype(np.int64) & 0xFFFFFFFF)
    _, first = np.unique(key, return_index=True)
    first.sort()
    cand, key = cand[first], key[first]
    keep = np.fromiter((k not in seen for k in key.tolist()), dtype=bool, count=key.shape[0])
    cand, key = cand[keep][:need], key[keep][:need]
    seen.update(key.tolist())
    return cand


@dataclass
class Problem:
    name: str
    src: np.ndarray      # (n_src, 2) int32
    tgt: np.ndarray      # (n_tgt, 2) int32
    f: np.ndarray        # (n_src,) float64, sums to zero
    same_points: bool    # targets are the sources

    @property
    def n_points(self) -> int:
        return int(self.src.shape[0] + self.tgt.shape[0])


def uniform_4k(seed: int = 0) -> Problem:
    rng = np.random.default_rng(seed)
    src = distinct_in_box(rng, 4096, 256)
    f = zero_sum(rng.standard_normal(4096))
    return Problem("uniform_4k", src, src.copy(), f, True)


def uniform_box(n_src: int, n_tgt: int, side: int, seed: int, name: str = "uniform_box",
                same_points: bool = False) -> Problem:
    rng = np.random.default_rng(seed)
    src = distinct_in_box(rng, n_src, side)
    f = zero_sum(rng.standard_normal(n_src))
    tgt = src.copy() if same_points else distinct_in_box(rng, n_tgt, side)
    return Problem(name, src, tgt, f, same_points)


def uniform_1m(seed: int = 1, n: int = 1 << 20, side: int = 4096) -> Problem:
    return uniform_box(n, n, side, seed, name="uniform_1m")


def clustered_4m(seed: int = 2, n_total: int = 4_194_304, n_clusters: int = 64,
                 sigma: float = 200.0, n_segments: int = 16, seg_len: float = 4000.0,
                 frac_lines: float = 0.01, domain: int = 65536) -> Problem:
    rng = np.random.default_rng(seed)
    n_lines = int(round(frac_lines * n_total)) if frac_lines > 0 else 0
    n_lines = min(n_lines, n_total)
    n_clu = n_total - n_lines
    seen: set = set()
    parts = []
    # segments
    centres = rng.uniform(0, domain, size=(n_segments, 2))
    angles = rng.uniform(0, np.pi, size=n_segments)
    per_seg = [n_lines // n_segments + (1 if i < n_lines % n_segments else 0) for i in range(n_segments)]
    for c, a, k in zip(centres, angles, per_seg):
        got = np.empty((0, 2), dtype=np.int32)
        while got.shape[0] < k:
            t = rng.uniform(-0.5, 0.5, size=2 * (k - got.shape[0]) + 16) * seg_len
            cand = np.rint(np.stack([c[0] + t * np.cos(a), c[1] + t * np.sin(a)], 1)).astype(np.int32)
            got = np.concatenate([got, _take_new(cand, seen, k - got.shape[0])])
        parts.append(got)
    # clusters
    centres = rng.uniform(0, domain, size=(n_clusters, 2))
    per_clu = [n_clu // n_clusters + (1 if i < n_clu % n_clusters else 0) for i in range(n_clusters)]
    for c, k in zip(centres, per_clu):
        got = np.empty((0, 2), dtype=np.int32)
        while got.shape[0] < k:
            need = k - got.shape[0]
            cand = np.rint(rng.normal(loc=c, scale=sigma, size=(need + need // 8 + 16, 2))).astype(np.int32)
            got = np.concatenate([got, _take_new(cand, seen, need)])
        parts.append(got)
    src = np.ascontiguousarray(np.concatenate(parts).astype(np.int32))
    f = zero_sum(rng.uniform(-1.0, 1.0, size=src.shape[0]))
    return Problem("clustered_4m", src, src.copy(), f, True)


def forest_sizes(seed: int = 3, n_problems: int = 4096, n_min: int = 512, n_max: int = 8192) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_problems))).astype(np.int64)


def forest_4096(seed: int = 3, n_problems: int = 4096, n_min: int = 512, n_max: int = 8192) -> list[Problem]:
    sizes = forest_sizes(seed, n_problems, n_min, n_max)
    ss = np.random.SeedSequence(seed).spawn(n_problems)
    out = []
    for i, (n, s) in enumerate(zip(sizes.tolist(), ss)):
        rng = np.random.default_rng(s)
        side = int(math.ceil(4.0 * math.sqrt(n)))
        src = distinct_in_box(rng, n, side)
        f = zero_sum(rng.standard_normal(n))
        out.append(Problem(f"forest_{i}", src, src.copy(), f, True))
    return out


@dataclass
class Request:
    index: int
    arrival_s: float
    tol: float
    problem: Problem


def serve_schedule(seed: int = 4, n_requests: int = 20_000, rate_per_s: float = 2000.0,
                   n_min: float = 1e3, n_max: float = 1e6) -> dict:
    """Arrival times (Poisson at rate_per_s), sizes (log-uniform N_src), point-set kinds
    (0 uniform, 1 four clusters) and tolerances (1e-6 or 1e-10) of the serving stream.
    Each array comes from its own generator, so the schedule of the first n requests
    is a prefix of the schedule of any longer stream."""
    g_arr, g_size, g_kind, g_tol = (np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(4))
    gaps = g_arr.exponential(1.0 / rate_per_s, size=n_requests)
    return {"seed": seed,
            "arrival_s": np.cumsum(gaps),
            "n_src": np.rint(np.exp(g_size.uniform(np.log(n_min), np.log(n_max), size=n_requests))).astype(np.int64),
            "kind": g_kind.integers(0, 2, size=n_requests),
            "tol": np.where(g_tol.integers(0, 2, size=n_requests) == 0, 1e-6, 1e-10)}


def serve_request(schedule: dict, i: int) -> Request:
    """Request i of a schedule; independent of the others (its own seed), so requests can
    be generated in any order or in parallel."""
    seed = schedule["seed"]
    rng = np.random.default_rng(np.random.SeedSequence([seed + 1_000_003, i]))
    n = int(schedule["n_src"][i])
    side = int(math.ceil(4.0 * math.sqrt(n)))
    if int(schedule["kind"][i]) == 0:
        src = distinct_in_box(rng, n, side)
    else:
        seen: set = set()
        centres = rng.uniform(0, side, size=(4, 2))
        per = [n // 4 + (1 if j < n % 4 else 0) for j in range(4)]
        parts = []
        for c, k in zip(centres, per):
            got = np.empty((0, 2), dtype=np.int32)
            while got.shape[0] < k:
                need = k - got.shape[0]
                cand = np.rint(rng.normal(c, side / 16.0, size=(need + need // 8 + 16, 2))).astype(np.int32)
                got = np.concatenate([got, _take_new(cand, seen, need)])
            parts.append(got)
        src = np.ascontiguousarray(np.concatenate(parts))
    n_t = max(1, n // 4)
    tgt = np.empty((n_t, 2), dtype=np.int32)
    tgt[:, 0] = rng.integers(0, side, size=n_t)
    tgt[:, 1] = rng.integers(0, side, size=n_t)
    f = zero_sum(rng.standard_normal(n))
    return Request(i, float(schedule["arrival_s"][i]), float(schedule["tol"][i]),
                   Problem(f"req_{i}", src, tgt, f, False))


def serve_stream(seed: int = 4, n_requests: int = 20_000, rate_per_s: float = 2000.0,
                 n_min: float = 1e3, n_max: float = 1e6):
    """Yields the Requests of the serving stream lazily (all of them do not fit in host
    memory at once)."""
    sch = serve_schedule(seed, n_requests, rate_per_s, n_min, n_max)
    for i in range(n_requests):
        yield serve_request(sch, i)


WORKLOADS = {
    "uniform_4k": uniform_4k,
    "uniform_1m": uniform_1m,
    "clustered_4m": clustered_4m,
}
