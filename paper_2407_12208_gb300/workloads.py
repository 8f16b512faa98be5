"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers: it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle consume the fp32 arrays
it returns.  Every generator takes an explicit seed (numpy PCG64).

Workloads (the paper's data are not available here; these stand in for them):

* ``blobs``            isotropic Gaussian blobs (Section 6.2.1 experiments):
                       centres uniform in [-box, box]^d, each point picks a
                       blob uniformly, additive N(0, std^2).
* ``uniform_pairs``    X ~ U[0,1)^(n x d), C = k distinct rows of X ("far"
                       data of Table 6.1's random-points scenario).
* ``cancellation``     X = offset * 1 + N(0, sigma^2), C = k distinct rows of X:
                       all pairs nearly coincide far from the origin, the
                       cancellation-prone regime of Section 4 (Table 6.1's
                       near-points scenario, Eq. (quantis-necess-cond)).
* ``gaussian_mixture`` centre coordinates N(0, 25), per-cluster std
                       log-uniform in [0.1, 2], uniform cluster choice.
* ``voronoi_image``    an H x W image of ``sites`` constant-colour Voronoi
                       regions plus N(0, 0.02^2) noise clipped to [0, 1];
                       features (R, G, B, x/(W-1), y/(H-1)) as in Section 6.2.2.
* ``near_far``         Table 6.2's stress data: C = P + eps N(0, I) for a
                       fraction of rows, fresh random rows otherwise.
* ``serving_jobs``     the job mix of a served stream (sizes only).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def init_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct seeded indices in [0, n): 'k centers uniformly from the data'."""
    return np.sort(_rng(seed).choice(n, size=k, replace=False)).astype(np.int64)


def seed_uniforms(k: int, seed: int) -> np.ndarray:
    """k seeded draws in [0, 1) for D^2-sampling seeding (the method's random
    numbers are inputs, the same for the library and the oracle)."""
    return _rng(seed).random(k)


def blobs(n: int, d: int, k: int, seed: int, box: float = 10.0, std: float = 1.0, with_labels: bool = False):
    """Isotropic Gaussian blobs: k centres uniform in [-box, box]^d, each
    point picks a blob uniformly, noise N(0, std^2 I); init = k seeded
    distinct points.  with_labels: also the blob of every point."""
    r = _rng(seed)
    centres = r.uniform(-box, box, size=(k, d))
    lab = r.integers(0, k, size=n)
    X = centres[lab] + r.normal(0.0, std, size=(n, d))
    X = X.astype(np.float32)
    C0 = X[init_indices(n, k, seed + 1)].copy()
    if with_labels:
        return X, C0, lab.astype(np.int32)
    return X, C0


def uniform_pairs(n: int, d: int, k: int, seed: int):
    r = _rng(seed)
    X = r.random((n, d), dtype=np.float32)
    C = X[init_indices(n, k, seed + 1)].copy()
    return X, C


def cancellation(n: int, d: int, k: int, seed: int, offset: float = 1e3, sigma: float = 1e-2):
    r = _rng(seed)
    X = (offset + r.normal(0.0, sigma, size=(n, d))).astype(np.float32)
    C = X[init_indices(n, k, seed + 1)].copy()
    return X, C


def gaussian_mixture(n: int, d: int, k: int, seed: int, centre_std: float = 5.0,
                     std_lo: float = 0.1, std_hi: float = 2.0, chunk: int = 1 << 20):
    r = _rng(seed)
    centres = r.normal(0.0, centre_std, size=(k, d))
    stds = np.exp(r.uniform(np.log(std_lo), np.log(std_hi), size=k))
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = r.integers(0, k, size=e - s)
        X[s:e] = (centres[lab] + r.normal(0.0, 1.0, size=(e - s, d)) * stds[lab, None]).astype(np.float32)
    C0 = X[init_indices(n, k, seed + 1)].copy()
    return X, C0


def voronoi_image(H: int, W: int, sites: int, k: int, seed: int, noise: float = 0.02):
    """Returns (features n x 5 fp32, initial centres k x 5)."""
    r = _rng(seed)
    sx = r.uniform(0, W, size=sites)
    sy = r.uniform(0, H, size=sites)
    colours = r.random((sites, 3))
    X = np.empty((H * W, 5), dtype=np.float32)
    xs = np.arange(W, dtype=np.float64)
    for y0 in range(0, H, 256):
        y1 = min(H, y0 + 256)
        yy, xx = np.meshgrid(np.arange(y0, y1, dtype=np.float64), xs, indexing="ij")
        dist = (xx[..., None] - sx) ** 2 + (yy[..., None] - sy) ** 2
        reg = np.argmin(dist, axis=-1)
        rgb = colours[reg] + r.normal(0.0, noise, size=reg.shape + (3,))
        rgb = np.clip(rgb, 0.0, 1.0)
        rows = slice(y0 * W, y1 * W)
        X[rows, 0:3] = rgb.reshape(-1, 3)
        X[rows, 3] = (xx / max(W - 1, 1)).reshape(-1)
        X[rows, 4] = (yy / max(H - 1, 1)).reshape(-1)
    C0 = X[init_indices(H * W, k, seed + 1)].copy()
    return X, C0


def near_far(n: int, d: int, frac_near: float, seed: int, eps: float = 1e-4):
    """Table 6.2's hybrid data: P random (N(0,1)), C = P + eps N(0, I) on a
    fraction of rows, fresh random rows otherwise."""
    r = _rng(seed)
    P = r.normal(0.0, 1.0, size=(n, d))
    C = r.normal(0.0, 1.0, size=(n, d))
    m = int(round(frac_near * n))
    C[:m] = P[:m] + eps * r.normal(0.0, 1.0, size=(m, d))
    return P.astype(np.float32), C.astype(np.float32)


def serving_jobs(num: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e6,
                 ds=(2, 8, 32, 128, 256), k_lo: float = 4, k_hi: float = 1024):
    """Job sizes of a served stream: n log-uniform, d uniform over ds,
    k log-uniform (rounded, at most n)."""
    r = _rng(seed)
    n = np.exp(r.uniform(np.log(n_lo), np.log(n_hi), size=num)).astype(np.int64)
    d = r.choice(np.asarray(ds), size=num)
    k = np.rint(np.exp(r.uniform(np.log(k_lo), np.log(k_hi), size=num))).astype(np.int64)
    k = np.minimum(k, n)
    return [dict(n=int(a), d=int(b), k=int(c)) for a, b, c in zip(n, d, k)]


def poisson_arrivals(num: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    r = _rng(seed)
    return np.cumsum(r.exponential(1.0 / rate_per_s, size=num))
