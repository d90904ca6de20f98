"""Seeded synthetic scalar fields shaped like the paper's HPC datasets.

This module only makes inputs.  It holds none of the compressor's
arithmetic and is shared by the tests, the benchmark and the CPU oracle's
callers, so both sides of every parity check see the same bytes.

The paper evaluates on SDRBench fields (Table 1: CESM 1800x3600, Nyx 512^3,
...) that are not available here; these seeded fields stand in for them with
the same shapes and a comparable smoothness:

* ``bumps3d``  -- 64^3 sum of 32 Gaussian bumps + N(0, 1e-3) noise (seed 1)
* ``climate2d`` -- 1800x3600 Gaussian random field, power ~ k^-3, mean 280,
  std 15 (seed 2; stands in for CESM's 2-D climate fields)
* ``cosmo3d`` -- 512^3 Gaussian random field g with power ~ k^-11/3, unit
  std, field = exp(0.5 g) (seed 3; a lognormal density like Nyx's baryon
  density)
* ``grf`` -- any shape and spectral slope, used for ragged and batched cases
* ``particles1d`` -- particle velocities in particle order (seed 5; stands
  in for HACC's 1-D velocity arrays, which the paper compresses
  log-transformed with a point-wise relative bound)

Arrays are returned in numpy C order indexed [z, y, x] (x fastest), i.e. the
layout the C ABI expects with dims given fastest-first.
"""
from __future__ import annotations

import numpy as np

try:  # scipy's FFT works in single precision and threads; numpy is fallback
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None


def _rfftn(a):
    if _sfft is not None:
        return _sfft.rfftn(a, workers=-1)
    return np.fft.rfftn(a)


def _irfftn(a, shape):
    if _sfft is not None:
        return _sfft.irfftn(a, s=shape, workers=-1)
    return np.fft.irfftn(a, s=shape, axes=tuple(range(len(shape))))


def grf(shape, beta: float, seed: int, single: bool | None = None) -> np.ndarray:
    """Zero-mean, unit-std Gaussian random field with power spectrum ~ |k|^beta.

    White noise is filtered in Fourier space by |k|^(beta/2), the k = 0 mode
    is removed, and the result is normalised.  ``shape`` is numpy order.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    if single is None:
        single = n > (1 << 24)
    rng = np.random.default_rng(seed)
    dt = np.float32 if single else np.float64
    w = rng.standard_normal(shape, dtype=dt)
    F = _rfftn(w)
    del w
    # |k|^2 built one axis at a time to keep memory at one complex volume
    k2 = None
    for ax, s in enumerate(shape):
        if ax == len(shape) - 1:
            k = np.fft.rfftfreq(s) * s
        else:
            k = np.fft.fftfreq(s) * s
        k = k.astype(dt)
        sh = [1] * len(shape)
        sh[ax] = k.size
        kk = (k * k).reshape(sh)
        k2 = kk if k2 is None else k2 + kk
    k2 = np.broadcast_to(k2, F.shape).copy()
    k2.flat[0] = 1.0
    F *= (k2 ** dt(beta / 4.0)).astype(dt)
    del k2
    F.flat[0] = 0.0
    g = _irfftn(F, shape)
    del F
    g = g.astype(dt, copy=False)
    g -= g.mean(dtype=np.float64)
    g /= g.std(dtype=np.float64)
    return g


def bumps3d(n: int = 64, nbumps: int = 32, seed: int = 1) -> np.ndarray:
    """Sum of Gaussian bumps (amplitude N(0,1), width U[4,16] voxels) plus
    N(0, 1e-3) noise on an n^3 grid, float32, [z, y, x]."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, n, size=(nbumps, 3))
    amps = rng.standard_normal(nbumps)
    sig = rng.uniform(4, 16, size=nbumps)
    ax = np.arange(n, dtype=np.float64)
    f = np.zeros((n, n, n), np.float64)
    for c, a, s in zip(centers, amps, sig):
        gz = np.exp(-((ax - c[2]) ** 2) / (2 * s * s))
        gy = np.exp(-((ax - c[1]) ** 2) / (2 * s * s))
        gx = np.exp(-((ax - c[0]) ** 2) / (2 * s * s))
        f += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    f += rng.normal(0.0, 1e-3, size=f.shape)
    return f.astype(np.float32)


def climate2d(ny: int = 1800, nx: int = 3600, seed: int = 2) -> np.ndarray:
    """k^-3 Gaussian random field, mean 280, std 15, float32 [y, x]."""
    g = grf((ny, nx), -3.0, seed, single=False)
    return (280.0 + 15.0 * g).astype(np.float32)


def cosmo3d(n: int = 512, seed: int = 3) -> np.ndarray:
    """exp(0.5 g), g a unit-std k^-11/3 Gaussian random field, float32."""
    g = grf((n, n, n), -11.0 / 3.0, seed)
    np.multiply(g, 0.5, out=g)
    np.exp(g, out=g)
    return g.astype(np.float32, copy=False)


def batch_shapes(count: int = 256, seed: int = 4, lo: int = 64 << 10,
                 hi: int = 64 << 20):
    """(shape, ndim, beta, rel_eb) for a batch of uneven fields: byte sizes
    log-uniform on [lo, hi], 2-D/3-D half and half, near-square/cubic
    shapes, spectral slope U[-4, -2], relative bound from {1e-2,1e-3,1e-4}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nbytes = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        n = max(16, int(nbytes / 4))
        ndim = 2 if rng.uniform() < 0.5 else 3
        if ndim == 2:
            ny = int(round(np.sqrt(n) * rng.uniform(0.7, 1.4)))
            ny = max(4, ny)
            nx = max(4, n // ny)
            shape = (ny, nx)
        else:
            a = n ** (1.0 / 3.0)
            nz = max(4, int(round(a * rng.uniform(0.7, 1.4))))
            ny = max(4, int(round(a * rng.uniform(0.7, 1.4))))
            nx = max(4, n // (nz * ny))
            shape = (nz, ny, nx)
        beta = float(rng.uniform(-4.0, -2.0))
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))
        out.append((shape, ndim, beta, eb))
    return out


def particles1d(n: int = 1 << 24, seed: int = 5, zero_frac: float = 1e-4) -> np.ndarray:
    """Particle velocities, float32, in particle order: groups of particles
    (halos of 64 to 4096 members) share a bulk velocity, members scatter
    around it (normal, 20% of the bulk spread); signs mix; a fraction of
    exact zeros.  Neighbouring values are related as in a sorted particle
    file, and magnitudes span several decades."""
    rng = np.random.default_rng(seed)
    sizes = []
    tot = 0
    while tot < n:
        s = int(rng.integers(64, 4097))
        sizes.append(s)
        tot += s
    sizes = np.asarray(sizes)
    bulk = rng.normal(0.0, 300.0, sizes.size)
    v = np.repeat(bulk, sizes)[:n] + rng.normal(0.0, 60.0, n)
    v = v.astype(np.float32)
    z = rng.random(n) < zero_frac
    v[z] = 0.0
    return v


def dense_sparse(ndim: int, seed: int) -> np.ndarray:
    """A smooth field (sums of sines) with uniform noise of amplitude 200 in
    one band of every four: 3-D (80, 512, 512), the noise on planes z with
    (z // 2) % 4 == 0; 2-D (4096, 4800), on rows y with (y // 32) % 4 == 0.
    At an absolute bound of 0.05 the noisy bands make nearly all bit-plane
    blocks of their tiles nonzero and the smooth bands few, so dense and
    sparse tiles alternate through a field of about 10,000 tiles, float32."""
    rng = np.random.default_rng(seed)
    if ndim == 3:
        shape = (80, 512, 512)
        z = np.arange(shape[0], dtype=np.float32)[:, None, None]
        y = np.arange(shape[1], dtype=np.float32)[None, :, None]
        x = np.arange(shape[2], dtype=np.float32)[None, None, :]
        base = np.sin(0.011 * x) + np.cos(0.017 * y) + 0.5 * np.sin(0.023 * z)
        noisy = (np.arange(shape[0]) // 2) % 4 == 0
        out = np.broadcast_to(base, shape).astype(np.float32)
        for k in np.flatnonzero(noisy):
            out[k] += rng.uniform(-200.0, 200.0, shape[1:]).astype(np.float32)
    else:
        shape = (4096, 4800)
        y = np.arange(shape[0], dtype=np.float32)[:, None]
        x = np.arange(shape[1], dtype=np.float32)[None, :]
        out = (np.sin(0.011 * x) + np.cos(0.017 * y)).astype(np.float32)
        noisy = (np.arange(shape[0]) // 32) % 4 == 0
        rows = np.flatnonzero(noisy)
        out[rows] += rng.uniform(-200.0, 200.0, (rows.size, shape[1])).astype(np.float32)
    return out


def small_cases():
    """Small ragged shapes (numpy order) spanning several tiles/chunks."""
    return [
        ((5,), 1), ((2048,), 1), ((8193,), 1), ((30001,), 1),
        ((3, 7), 2), ((129, 65), 2), ((200, 130), 2), ((257, 300), 2),
        ((2, 2, 2), 3), ((9, 33, 31), 3), ((17, 40, 70), 3), ((20, 64, 96), 3),
    ]
