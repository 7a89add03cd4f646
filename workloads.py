"""Seeded synthetic particle sets for the adaptive 2-D FMM.

This module only draws random inputs.  It holds none of the method's
arithmetic, so both the CPU oracle (tests, CPU baseline) and the CUDA path
(tests, bench) can take their inputs from it.

Shapes follow the point distributions used in the paper's adaptivity study
(Sec. 5.5, Fig. "adaptivity": uniform, normal clusters, a thin layer) and the
benchmark configurations of this project:

* ``uniform``   -- iid uniform in the unit square.
* ``clusters``  -- 16 Gaussian clusters, centres uniform in the unit square,
                   sigma log-uniform in [1e-3, 1e-1], equal weight, plus 10 %
                   uniform background; points outside the unit square are
                   redrawn (rejection), as the paper does for its normal set.
* ``curve``     -- (0.5, 0.5) + r(t)(cos t, sin t), r = 0.4 + 0.1 cos 7t,
                   t ~ U[0, 2pi), plus isotropic Gaussian jitter sigma = 1e-4.
* ``normal``    -- the paper's normal set: N((0.5, 0.5), sigma^2 I), sigma = 0.1
                   (variance 1/100) unless given, rejected into the unit square.
* ``layer``     -- the paper's "layer": x uniform, y ~ N(0.5, sigma^2), rejected
                   into the unit square.

Strengths are complex (re, im iid U[-1, 1]) or real N(0, 1) stored as complex
with zero imaginary part.  Arrays are float64, positions interleaved (x, y),
strengths interleaved (re, im).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 12054611

DISTRIBUTIONS = ("uniform", "clusters", "curve")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_points(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.random((n, 2))


def cluster_points(n: int, rng: np.random.Generator, n_clusters: int = 16,
                   background: float = 0.1) -> np.ndarray:
    centres = rng.random((n_clusters, 2))
    sigmas = 10.0 ** rng.uniform(-3.0, -1.0, size=n_clusters)
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    which = rng.integers(0, n_clusters, size=n_cl)
    pts = np.empty((n, 2))
    pts[:n_bg] = rng.random((n_bg, 2))
    cl = centres[which] + sigmas[which, None] * rng.standard_normal((n_cl, 2))
    # rejection into the unit square: redraw only the offending points
    bad = np.nonzero(((cl < 0.0) | (cl > 1.0)).any(axis=1))[0]
    while bad.size:
        w = which[bad]
        cl[bad] = centres[w] + sigmas[w, None] * rng.standard_normal((bad.size, 2))
        bad = bad[((cl[bad] < 0.0) | (cl[bad] > 1.0)).any(axis=1)]
    pts[n_bg:] = cl
    return pts[rng.permutation(n)]


def curve_points(n: int, rng: np.random.Generator, jitter: float = 1e-4) -> np.ndarray:
    t = rng.uniform(0.0, 2.0 * np.pi, size=n)
    r = 0.4 + 0.1 * np.cos(7.0 * t)
    pts = np.stack([0.5 + r * np.cos(t), 0.5 + r * np.sin(t)], axis=1)
    return pts + jitter * rng.standard_normal((n, 2))


def _reject_normal(n: int, rng: np.random.Generator, sigma: float, layer: bool) -> np.ndarray:
    """Normal about 0.5 in y (and in x unless `layer`), redrawn until inside [0, 1]^2."""
    def draw(k):
        y = 0.5 + sigma * rng.standard_normal(k)
        x = rng.random(k) if layer else 0.5 + sigma * rng.standard_normal(k)
        return np.stack([x, y], axis=1)
    pts = draw(n)
    bad = np.nonzero(((pts < 0.0) | (pts > 1.0)).any(axis=1))[0]
    while bad.size:
        pts[bad] = draw(bad.size)
        bad = bad[((pts[bad] < 0.0) | (pts[bad] > 1.0)).any(axis=1)]
    return pts


def points(dist: str, n: int, rng: np.random.Generator, sigma: float = 0.1) -> np.ndarray:
    if dist == "uniform":
        return uniform_points(n, rng)
    if dist == "clusters":
        return cluster_points(n, rng)
    if dist == "curve":
        return curve_points(n, rng)
    if dist == "normal":
        return _reject_normal(n, rng, sigma, layer=False)
    if dist == "layer":
        return _reject_normal(n, rng, sigma, layer=True)
    raise ValueError(f"unknown distribution {dist!r}")


def complex_strengths(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=(n, 2))


def real_strengths(n: int, rng: np.random.Generator) -> np.ndarray:
    q = np.zeros((n, 2))
    q[:, 0] = rng.standard_normal(n)
    return q


def problem(dist: str, n: int, seed: int, real_q: bool = False,
            tgt_dist: str | None = None, m: int = 0, sigma: float = 0.1):
    """Return (src_xy[n,2], q[n,2], tgt_xy[m,2] or None), all float64, C-contiguous."""
    rng = _rng(seed)
    src = np.ascontiguousarray(points(dist, n, rng, sigma))
    q = real_strengths(n, rng) if real_q else complex_strengths(n, rng)
    tgt = None
    if tgt_dist is not None:
        tgt = np.ascontiguousarray(points(tgt_dist, m, rng))
    return src, np.ascontiguousarray(q), tgt


# The five benchmark workloads (sizes as named; seeds BASE_SEED + index).
WORKLOADS = {
    "uniform_1e4": dict(dist="uniform", n=10_000, p=20, leaf=40, seed=BASE_SEED + 0),
    "clusters_1e6": dict(dist="clusters", n=1_000_000, p=24, leaf=64, seed=BASE_SEED + 1),
    "curve_4e6": dict(dist="curve", n=4_000_000, p=24, leaf=64, seed=BASE_SEED + 2, real_q=True),
    "batched_512": dict(n_inst=512, p=20, seed=BASE_SEED + 3),
    "clusters_1p6e7_targets": dict(dist="clusters", n=16_000_000, p=30, leaf=64,
                                   seed=BASE_SEED + 4, tgt_dist="uniform", m=16_000_000),
    # the case of the paper's time breakdown (Sec. 5.1): N = 45 * 2^16 uniform
    # points, 45 per leaf, p = 17 (tolerance ~1e-6), harmonic kernel
    "uniform_45x2p16": dict(dist="uniform", n=45 * 2 ** 16, p=17, leaf=45, seed=BASE_SEED + 5),
}


def make(name: str, scale: float = 1.0):
    """Build a named workload, optionally scaled down in N (and M)."""
    w = dict(WORKLOADS[name])
    n = max(1, int(round(w["n"] * scale)))
    m = max(1, int(round(w.get("m", 0) * scale))) if w.get("tgt_dist") else 0
    return problem(w["dist"], n, w["seed"], real_q=w.get("real_q", False),
                   tgt_dist=w.get("tgt_dist"), m=m)


def batched_instances(n_inst: int = 512, seed: int = BASE_SEED + 3,
                      log_lo: float = 3.0, log_hi: float = 5.0):
    """Independent instances with N_i = floor(10**U[log_lo, log_hi]) and a
    distribution drawn per instance; returns a list of (dist, src, q)."""
    rng = _rng(seed)
    sizes = np.floor(10.0 ** rng.uniform(log_lo, log_hi, size=n_inst)).astype(np.int64)
    kinds = rng.integers(0, len(DISTRIBUTIONS), size=n_inst)
    out = []
    for i in range(n_inst):
        r = _rng(seed * 1000 + i)
        dist = DISTRIBUTIONS[kinds[i]]
        src = np.ascontiguousarray(points(dist, int(sizes[i]), r))
        q = np.ascontiguousarray(complex_strengths(int(sizes[i]), r))
        out.append((dist, src, q))
    return out
