"""Pins for the symmetric-boundary (DCT) variant the paper mentions at the start of Sec. 3.

* convolution with reflected boundaries, written as tap-by-tap loops over the reflected image, equals
  circular convolution on the half-sample symmetric extension, cropped;
* for a filter symmetric about its centre it is diagonal in the orthonormal type-II DCT with the
  cosine eigenvalues of dct_eigenvalues;
* the dual ADMM run in the DCT domain (code_admm_dct) and the extended-grid ADMM (code_admm_symmetric,
  the GPU path's definition) reach the same codes on the image, and the extended codes are mirror
  symmetric: two independent computations of the same iteration.
"""
import itertools

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import csc_oracle as O


def reflect(i, n):
    i = i % (2 * n)
    return i if i < n else 2 * n - 1 - i


def brute_reflected_conv(e, z):
    """(e * z)(p) = sum_a e[a] z_refl(p - (a - c)) with z_refl the half-sample reflection of z."""
    H, W = z.shape
    out = np.zeros(z.shape)
    for a, b in itertools.product(range(e.shape[0]), range(e.shape[1])):
        oa, ob = a - (e.shape[0] - 1) // 2, b - (e.shape[1] - 1) // 2
        for h, w in itertools.product(range(H), range(W)):
            out[h, w] += e[a, b] * z[reflect(h - oa, H), reflect(w - ob, W)]
    return out


def symmetric_filter(rng, f):
    e = rng.standard_normal((f, f))
    return 0.25 * (e + e[::-1, :] + e[:, ::-1] + e[::-1, ::-1])


@pytest.mark.parametrize("dims,f", [((7, 9), 3), ((8, 6), 5)])
def test_reflected_convolution_is_extension_convolution_and_dct_diagonal(dims, f):
    rng = np.random.default_rng(80)
    z = rng.standard_normal(dims)
    e = rng.standard_normal((f, f))
    want = brute_reflected_conv(e, z)
    ext = O.synthesize(e[None, None], O.symmetric_extend(z)[None, None])[0, 0]
    np.testing.assert_allclose(ext[: dims[0], : dims[1]], want, atol=1e-12)
    es = symmetric_filter(rng, f)
    want_s = brute_reflected_conv(es, z)
    delta = O.dct_eigenvalues(es[None], dims)[0]
    got = sfft.idctn(delta * sfft.dctn(z, type=2, norm="ortho"), type=2, norm="ortho")
    np.testing.assert_allclose(got, want_s, atol=1e-12)


def test_dct_admm_equals_extended_grid_admm_for_symmetric_filters():
    rng = np.random.default_rng(81)
    N, K, dims, f, beta, rho, iters = 2, 3, (10, 12), 3, 0.2, 1.5, 15
    x = rng.standard_normal((N, 1) + dims)
    d = np.stack([symmetric_filter(rng, f) for _ in range(K)])[:, None]
    d /= np.sqrt((d ** 2).sum(axis=(1, 2, 3), keepdims=True))
    v_dct, z_dct = O.code_admm_dct(x, d, beta, rho, iters)
    v_ext, z_ext = O.code_admm_symmetric(x, d, beta, rho, iters)
    H, W = dims
    np.testing.assert_allclose(z_ext[..., :H, :W], z_dct, atol=1e-10)
    np.testing.assert_allclose(v_ext[..., :H, :W], v_dct, atol=1e-10)
    np.testing.assert_allclose(z_ext, O.symmetric_extend(z_ext[..., :H, :W]), atol=1e-10)
    assert np.abs(z_dct).max() > 0
