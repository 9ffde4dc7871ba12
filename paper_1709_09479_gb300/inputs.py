"""Seeded synthetic inputs shaped like the workloads of arXiv 1709.09479 (Sec. 4.1).

The paper evaluates on photo collections (fruit, city, house) and a colour video. None of these is
available here, so every input is synthesised from a seed:

* ``sparse_synthetic``: images built as a sum of random unit-norm filters convolved with
  Bernoulli-Gaussian sparse maps, plus white noise. This is the generative model of Eq. 1.
* ``powerlaw_field``: Gaussian random fields with a 1/f^2 power spectrum (natural-image
  statistics), contrast-normalised per image to zero mean and unit variance (Sec. 4.1 applies
  contrast normalisation without defining it).
* ``unit_filters``: a seeded Gaussian dictionary with every filter scaled to unit norm over all
  of its channels and taps (the constraint set of Eq. 1).
* ``uneven_sizes``: per-image side lengths drawn uniformly from an integer range.

This module is shared by the tests, the benchmark and the CPU oracle's callers. It holds only data
synthesis: none of the coding or learning arithmetic of the method lives here. Everything is
generated in float64 with numpy's PCG64 ``default_rng`` and cast by the caller.
"""
from __future__ import annotations

import numpy as np

__all__ = ["unit_filters", "sparse_synthetic", "powerlaw_field", "uneven_sizes", "filter_offsets"]


def filter_offsets(f: int) -> int:
    """Index of the origin tap of a support of length ``f``: tap ``a`` sits at offset ``a - (f-1)//2``."""
    return (f - 1) // 2


def unit_filters(seed: int, K: int, J: int, fs) -> np.ndarray:
    """K filters of J channels and support ``fs`` drawn N(0,1), each scaled to unit l2 norm.

    Returns float64 of shape (K, J, *fs).
    """
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((K, J) + tuple(fs))
    norms = np.sqrt((d.reshape(K, -1) ** 2).sum(axis=1))
    return d / norms.reshape((K,) + (1,) * (d.ndim - 1))


def _shift_add(out: np.ndarray, d: np.ndarray, z: np.ndarray) -> None:
    """out += circular sum over taps of d[q] * z shifted by the tap offset (data synthesis only)."""
    fs = d.shape
    for idx in np.ndindex(*fs):
        w = d[idx]
        if w == 0.0:
            continue
        shift = [a - filter_offsets(f) for a, f in zip(idx, fs)]
        out += w * np.roll(z, shift=shift, axis=tuple(range(z.ndim)))


def sparse_synthetic(seed: int = 0, N: int = 10, dims=(100, 100), K: int = 16, s: int = 11,
                     density: float = 0.01, noise: float = 0.01):
    """Images x_n = sum_k d_k * z_nk + N(0, noise^2), with d_k ~ unit-norm Gaussian s x s filters and
    z_nk ~ Bernoulli(density) x N(0,1) per pixel (the model of Eq. 1, circular boundary).

    Returns dict with x (N, 1, *dims), d_true (K, 1, s, s), z_true (N, K, *dims); all float64.
    """
    rng = np.random.default_rng(seed)
    dims = tuple(dims)
    fs = (s,) * len(dims)
    d = rng.standard_normal((K, 1) + fs)
    d /= np.sqrt((d.reshape(K, -1) ** 2).sum(axis=1)).reshape((K, 1) + (1,) * len(fs))
    mask = rng.random((N, K) + dims) < density
    z = np.where(mask, rng.standard_normal((N, K) + dims), 0.0)
    x = np.zeros((N, 1) + dims)
    for n in range(N):
        for k in range(K):
            if mask[n, k].any():
                _shift_add(x[n, 0], d[k, 0], z[n, k])
    x += noise * rng.standard_normal(x.shape)
    return {"x": x, "d_true": d, "z_true": z}


def powerlaw_field(seed: int, N: int, J: int, dims, normalise: bool = True) -> np.ndarray:
    """Gaussian fields whose power spectrum falls as 1/|f|^2 over all axes of ``dims``.

    White N(0,1) noise is transformed, its amplitude multiplied by 1/|f| with f in cycles per sample
    (signed), the mean component set to 0, and transformed back. With ``normalise`` each (image,
    channel) is then shifted and scaled to zero mean and unit variance.
    Returns float64 of shape (N, J, *dims).
    """
    rng = np.random.default_rng(seed)
    dims = tuple(dims)
    white = rng.standard_normal((N, J) + dims)
    axes = tuple(range(2, 2 + len(dims)))
    spec = np.fft.rfftn(white, axes=axes)
    grids = []
    for i, n in enumerate(dims):
        f = np.fft.rfftfreq(n) if i == len(dims) - 1 else np.fft.fftfreq(n)
        shape = [1] * len(dims)
        shape[i] = f.size
        grids.append(f.reshape(shape))
    fmag2 = sum(g * g for g in grids)
    amp = np.zeros_like(fmag2)
    nz = fmag2 > 0
    amp[nz] = 1.0 / np.sqrt(fmag2[nz])
    field = np.fft.irfftn(spec * amp, s=dims, axes=axes)
    if normalise:
        red = tuple(range(2, field.ndim))
        field = field - field.mean(axis=red, keepdims=True)
        field = field / field.std(axis=red, keepdims=True)
    return field


def uneven_sizes(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """(n, 2) int array of (H, W), each side uniform on the integers [lo, hi], drawn independently."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n, 2))
