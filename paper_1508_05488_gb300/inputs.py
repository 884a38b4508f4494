"""Seeded synthetic point sets.

The paper measures on uniformly random points in a square (generated with
Qhull's ``rbox``) and on 3D scan models projected onto the XY plane
(Sec. 3, Tables 2-5).  The scan models are not available here; the uniform
square, disk, Gaussian, circle and degenerate sets below stand in for them.
This module only draws numbers: it holds none of the hull method's arithmetic
and is the one module shared by the CUDA path's tests and the oracle's.
"""
from __future__ import annotations

import numpy as np

GRID = 2.0 ** -20  # rounding grid of the degenerate workload


def square_i32(n: int, seed: int = 1, hi: int = 2 ** 29) -> np.ndarray:
    """n points, int32 coordinates uniform in [0, hi)^2."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(n, 2), dtype=np.int64).astype(np.int32)


def disk_i32(n: int, seed: int, center: int = 2 ** 28, radius: int = 2 ** 28 - 1) -> np.ndarray:
    """n points, int32 coordinates uniform in a disk (rejection sampling)."""
    rng = np.random.default_rng(seed)
    out = np.empty((0, 2), dtype=np.int64)
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.35) + 16
        p = rng.integers(center - radius, center + radius + 1, size=(m, 2), dtype=np.int64)
        d = p - center
        p = p[d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] <= radius * radius]
        out = np.concatenate([out, p])
    return out[:n].astype(np.int32)


def square_f64(n: int, seed: int = 2) -> np.ndarray:
    """n points uniform in the unit square [0, 1)^2."""
    return np.random.default_rng(seed).random((n, 2))


def disk_f64(n: int, seed: int = 3, radius: float = 1.0) -> np.ndarray:
    """n points uniform in the disk of the given radius: r = R sqrt(U), theta = 2 pi U."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.random(n))
    t = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def gauss_f64(n: int, seed: int = 4) -> np.ndarray:
    """n points from an isotropic Gaussian, sigma = 1."""
    return np.random.default_rng(seed).standard_normal((n, 2))


def shell_f64(n: int, seed: int, r0: float = 0.99, r1: float = 1.0) -> np.ndarray:
    """n points uniform in the annulus r0 <= r <= r1."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(r0 * r0 + (r1 * r1 - r0 * r0) * rng.random(n))
    t = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def circle_f64(n: int, seed: int = 6) -> np.ndarray:
    """n points at angles 2 pi k / n on the unit circle, shuffled: every
    point is a hull vertex (the limitation case of Sec. 4.3)."""
    t = 2.0 * np.pi * np.arange(n) / n
    p = np.stack([np.cos(t), np.sin(t)], axis=1)
    return p[np.random.default_rng(seed).permutation(n)]


def degenerate_f64(n: int = 20_000_000, seed: int = 5) -> np.ndarray:
    """Degenerate stress set: n/5 points at random angles on the unit circle
    and 4n/5 uniform in the disk of radius 1 - 2^-10, all rounded to the
    2^-20 grid (collinear runs, coincident points), then 1% of the rows
    overwritten by copies of other rows (half of them circle points) and the
    whole set shuffled."""
    rng = np.random.default_rng(seed)
    nc = n // 5
    t = 2.0 * np.pi * rng.random(nc)
    circ = np.stack([np.cos(t), np.sin(t)], axis=1)
    ni = n - nc
    r = (1.0 - 2.0 ** -10) * np.sqrt(rng.random(ni))
    t = 2.0 * np.pi * rng.random(ni)
    inner = np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    p = np.concatenate([circ, inner])
    p = np.round(p / GRID) * GRID
    nd = n // 100
    dst = rng.choice(n, size=nd, replace=False)
    src = np.where(np.arange(nd) % 2 == 0, rng.integers(0, nc, nd), rng.integers(0, n, nd))
    p[dst] = p[src]
    return p[rng.permutation(n)]


# ---------------------------------------------------------------- workloads

def headline_f64(kind: str, n: int = 20_000_000) -> np.ndarray:
    """The 20M-point float64 workloads: 'square' (seed 2), 'disk' (seed 3),
    'gauss' (seed 4)."""
    if kind == "square":
        return square_f64(n, 2)
    if kind == "disk":
        return disk_f64(n, 3)
    if kind == "gauss":
        return gauss_f64(n, 4)
    raise ValueError(kind)


def batched_sizes(nsets: int = 4096, seed: int = 7, lo: int = 256, hi: int = 2 ** 20) -> np.ndarray:
    """Set sizes floor(exp(U(ln lo, ln hi)))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), nsets))).astype(np.int64)


def batched_i32(nsets: int = 4096, seed: int = 7, lo: int = 256, hi: int = 2 ** 20):
    """Many independent int32 sets of log-uniform size, each a uniform
    square [0, 2^29)^2 or a disk (centre 2^28, radius 2^28 - 1) by a fair
    coin.  Returns (points [N, 2] int32, offsets int64[nsets + 1])."""
    sizes = batched_sizes(nsets, seed, lo, hi)
    rng = np.random.default_rng(seed + 1000)
    coins = rng.random(nsets) < 0.5
    parts = []
    for s in range(nsets):
        sub = int(rng.integers(0, 2 ** 31))
        n = int(sizes[s])
        parts.append(square_i32(n, sub) if coins[s] else disk_i32(n, sub))
    off = np.zeros(nsets + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return np.concatenate(parts), off


SERVE_KINDS = ("square", "disk", "gauss", "shell")


def serve_request(i: int, seed: int = 8, lo: float = 1e3, hi: float = 2e7) -> np.ndarray:
    """Request i of the serving stream: log-uniform size in [lo, hi), kind
    uniform over square / disk / Gaussian / shell, float64."""
    rng = np.random.default_rng([seed, i])
    n = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
    kind = SERVE_KINDS[int(rng.integers(0, 4))]
    sub = int(rng.integers(0, 2 ** 31))
    if kind == "square":
        return square_f64(n, sub)
    if kind == "disk":
        return disk_f64(n, sub)
    if kind == "gauss":
        return gauss_f64(n, sub)
    return shell_f64(n, sub)


def serve_request_meta(i: int, seed: int = 8, lo: float = 1e3, hi: float = 2e7):
    """Size, kind and sub-seed of request i of the serving stream (the same
    draws as serve_request)."""
    rng = np.random.default_rng([seed, i])
    n = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
    kind = SERVE_KINDS[int(rng.integers(0, 4))]
    sub = int(rng.integers(0, 2 ** 31))
    return n, kind, sub


def serve_request_device(i: int, device, seed: int = 8):
    """Request i of the serving stream drawn directly in device memory (a
    seeded torch generator on the device; the same size and kind as
    serve_request, other coordinates): float64 [n, 2] uniform in the unit
    square, the unit disk, Gaussian sigma 1, or the shell 0.99 <= r <= 1."""
    import torch
    n, kind, sub = serve_request_meta(i, seed)
    g = torch.Generator(device=device)
    g.manual_seed(sub)
    f64 = torch.float64
    if kind == "square":
        return torch.rand((n, 2), dtype=f64, device=device, generator=g)
    if kind == "gauss":
        return torch.randn((n, 2), dtype=f64, device=device, generator=g)
    u = torch.rand((n, 2), dtype=f64, device=device, generator=g)
    if kind == "disk":
        r = torch.sqrt(u[:, 0])
    else:
        r = torch.sqrt(0.99 ** 2 + u[:, 0] * (1.0 - 0.99 ** 2))
    t = 2.0 * np.pi * u[:, 1]
    return torch.stack([r * torch.cos(t), r * torch.sin(t)], dim=1).contiguous()


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 8) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed + 77)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


# ------------------------------------------------------ small adversarial sets

def small_cases(seed: int):
    """Small sets rich in collinear and duplicate points, for exhaustive
    cross-checks: int32 grids, float64 dyadic grids and plain random sets."""
    rng = np.random.default_rng(seed)
    kind = seed % 4
    n = int(rng.integers(1, 26))
    if kind == 0:
        k = int(rng.integers(1, 6))
        return rng.integers(-k, k + 1, size=(n, 2)).astype(np.int32)
    if kind == 1:
        k = int(rng.integers(1, 5))
        return (rng.integers(-k, k + 1, size=(n, 2)) / 4.0).astype(np.float64)
    if kind == 2:
        p = rng.random((n, 2))
        if n > 3:
            m = int(rng.integers(1, n))
            p[rng.integers(0, n, m)] = p[rng.integers(0, n, m)]
        return p
    big = 2 ** 31 - 1
    return rng.integers(-big - 1, big + 1, size=(n, 2), dtype=np.int64).astype(np.int32)
