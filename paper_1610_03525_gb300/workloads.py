"""Seeded synthetic workloads: field descriptions, sample subsets, chunk
batches and request streams.  Pure input recipes -- no noise arithmetic --
shared by the GPU path's tests and benchmark and by the oracle checks.

The paper's own workloads are 2D maps with R = 1024 and N <= 9 octaves and
S = 512 maps (Thorimbert & Chopard, arXiv:1610.03525, Sec. 5.2, 5.3); the
configurations below bracket them (256^2 to 8192^2, 3D volumes, chunk
batches) and stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

# name -> dict(dims, size, spc, octaves, smoothness, origin, dtype(s), seeds)
CONFIGS = {
    # 2D 256^2, C1, 6 octaves, base lattice 4x4 (spc 64), seed 0, FP32
    "2d_256_c1_n6": dict(dims=2, size=(256, 256), spc=64, octaves=6, origin=(0, 0, 0), seeds=(0,)),
    # 2D 8192^2, 12 octaves, base lattice 8x8 (spc 1024), C1/C2, seeds 0..3
    "2d_8192_n12": dict(dims=2, size=(8192, 8192), spc=1024, octaves=12, origin=(0, 0, 0),
                             seeds=(0, 1, 2, 3)),
    # 3D 512^3, 8 octaves, base lattice 4^3 (spc 128), C1, FP16, world offset
    "3d_512_n8": dict(dims=3, size=(512, 512, 512), spc=128, octaves=8, origin=(1 << 20, 1 << 20, 0),
                           seeds=(0,)),
}


def total_amplitude(octaves: int, persistence: float = 0.5) -> float:
    """Sum of the octave amplitudes p^i, i < N (the tolerance scale)."""
    return sum(persistence ** i for i in range(octaves))


def grid_indices_2d(w: int, h: int) -> np.ndarray:
    """All (x, y) sample indices of a w x h field, row-major."""
    ys, xs = np.meshgrid(np.arange(h, dtype=np.int64), np.arange(w, dtype=np.int64), indexing="ij")
    return np.stack([xs.ravel(), ys.ravel()], 1)


def grid_indices_3d(w: int, h: int, d: int) -> np.ndarray:
    zs, ys, xs = np.meshgrid(np.arange(d, dtype=np.int64), np.arange(h, dtype=np.int64),
                             np.arange(w, dtype=np.int64), indexing="ij")
    return np.stack([xs.ravel(), ys.ravel(), zs.ravel()], 1)


def subsample(size, every: int, n_random: int, seed: int = 12345, lattice_spc: int = 0) -> np.ndarray:
    """Deterministic parity subset of a large field: every `every`-th row
    (2D) or plane (3D) in full, plus n_random uniformly drawn samples, plus
    (lattice_spc > 0) the samples on the base lattice's lines: every column
    x = 0 mod lattice_spc in 2D, every line along z at x, y = 0 mod
    lattice_spc in 3D."""
    dims = len(size)
    rng = np.random.default_rng(seed)
    parts = []
    if dims == 2:
        w, h = size
        for y in range(0, h, every):
            parts.append(np.stack([np.arange(w, dtype=np.int64), np.full(w, y, np.int64)], 1))
        if lattice_spc > 0:
            for x in range(0, w, lattice_spc):
                parts.append(np.stack([np.full(h, x, np.int64), np.arange(h, dtype=np.int64)], 1))
    else:
        w, h, d = size
        for z in range(0, d, every):
            ys, xs = np.meshgrid(np.arange(h, dtype=np.int64), np.arange(w, dtype=np.int64), indexing="ij")
            parts.append(np.stack([xs.ravel(), ys.ravel(), np.full(xs.size, z, np.int64)], 1))
        if lattice_spc > 0:
            for y in range(0, h, lattice_spc):
                for x in range(0, w, lattice_spc):
                    parts.append(np.stack([np.full(d, x, np.int64), np.full(d, y, np.int64),
                                           np.arange(d, dtype=np.int64)], 1))
    rnd = np.stack([rng.integers(0, size[k], n_random, dtype=np.int64) for k in range(dims)], 1)
    parts.append(rnd)
    return np.concatenate(parts, 0)


def chunk_batch(n: int = 4096, seed: int = 12345, spc: int = 1024):
    """Batched workload: n 2D chunks, side log-uniform in [64, 1024] rounded
    to a multiple of 64, octaves uniform in 4..12, C1/C2 50/50, seed = chunk
    id, integer origins uniform in [-2^20, 2^20] base cells."""
    rng = np.random.default_rng(seed)
    out = []
    for cid in range(n):
        side = int(round(math.exp(rng.uniform(math.log(64), math.log(1024))) / 64.0)) * 64
        side = min(max(side, 64), 1024)
        octaves = int(rng.integers(4, 13))
        smooth = 1 if rng.random() < 0.5 else 2
        origin = (int(rng.integers(-(1 << 20), (1 << 20) + 1)), int(rng.integers(-(1 << 20), (1 << 20) + 1)), 0)
        out.append(dict(dims=2, size=(side, side), spc=spc, octaves=octaves, smoothness=smooth, seed=cid,
                        origin=origin))
    return out


def request_stream(rate_hz: float = 20000.0, duration_s: float = 1.0, seed: int = 12345):
    """Serving workload: Poisson arrivals; 80% 2D chunks with side
    log-uniform in [128, 2048] (spc 1024), 20% 3D with side log-uniform in
    [32, 256] (spc 128); octaves 4..12; C1/C2 50/50.  Sides are rounded to the
    tile (64 in 2D, 32 in 3D)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        octaves = int(rng.integers(4, 13))
        smooth = 1 if rng.random() < 0.5 else 2
        if rng.random() < 0.8:
            side = int(round(math.exp(rng.uniform(math.log(128), math.log(2048))) / 64.0)) * 64
            reqs.append(dict(t=t, dims=2, size=(side, side), spc=1024, octaves=octaves, smoothness=smooth,
                             seed=rid % (1 << 24), origin=(rid, 0, 0)))
        else:
            side = int(round(math.exp(rng.uniform(math.log(32), math.log(256))) / 32.0)) * 32
            reqs.append(dict(t=t, dims=3, size=(side, side, side), spc=128, octaves=octaves, smoothness=smooth,
                             seed=rid % (1 << 24), origin=(rid, 0, 0)))
        rid += 1
    return reqs
