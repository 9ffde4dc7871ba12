"""Direct pins for the oracle's learning operators Z_k and Z_k^T (Sec. 3.2, learning subproblem).

Every learning pin and the full-size GPU learning checks apply these two operators, so they are
pinned here against tap-by-tap loops that share nothing with the oracle's DFT route:

* Z_k with a filter-support map e_k: (Z e)_n = sum_k z_nk * S^T e_k is the circular convolution of
  Eq. 1 with the taps of e_k at their centred offsets (the model x ~ sum_k d_k * z_k with the roles of
  code and filter exchanged);
* S Z_k^T g: tap o of filter k is sum_n sum_p z_nk(p) g_n(p + o), the correlation of each image's
  code with the image-domain vector, summed over the images that share the dictionary;
* the adjoint identity <Z e, g> = <e, Z^T g> to rounding.

A conjugate on the wrong spectrum (correlation in place of convolution) or a sign flip of the tap
offsets fails the first two checks: the codes and maps are random and not symmetric.
"""
import itertools

import numpy as np
import pytest

from oracle import csc_oracle as O


def brute_conv_taps(e, z):
    """(e * z)(p) = sum_a e[a] z[(p - (a - c)) mod dims] with c = (f - 1) // 2, by explicit loops."""
    out = np.zeros(z.shape)
    dims = z.shape
    for a in itertools.product(*[range(f) for f in e.shape]):
        off = [ai - (f - 1) // 2 for ai, f in zip(a, e.shape)]
        for p in itertools.product(*[range(n) for n in dims]):
            q = tuple((pi - oi) % n for pi, oi, n in zip(p, off, dims))
            out[p] += e[a] * z[q]
    return out


def brute_corr_taps(z, g, fs):
    """t[a] = sum_p z(p) g((p + (a - c)) mod dims) for the taps a of support fs, by explicit loops."""
    dims = z.shape
    t = np.zeros(fs)
    for a in itertools.product(*[range(f) for f in fs]):
        off = [ai - (f - 1) // 2 for ai, f in zip(a, fs)]
        s = 0.0
        for p in itertools.product(*[range(n) for n in dims]):
            q = tuple((pi + oi) % n for pi, oi, n in zip(p, off, dims))
            s += z[p] * g[q]
        t[a] = s
    return t


CASES = [((6, 7), (3, 3)), ((5, 8), (3, 5)), ((4, 5, 6), (3, 3, 3))]


@pytest.mark.parametrize("dims,fs", CASES)
def test_Z_of_support_map_is_brute_force_convolution(dims, fs):
    rng = np.random.default_rng(71)
    N, K = 2, 3
    z = rng.standard_normal((N, K) + dims)
    e = rng.standard_normal((K,) + fs)
    got = O.LearningOperators(z).Z(O.pad_support(e, dims))
    for n in range(N):
        want = sum(brute_conv_taps(e[k], z[n, k]) for k in range(K))
        np.testing.assert_allclose(got[n], want, atol=1e-12)


@pytest.mark.parametrize("dims,fs", CASES)
def test_cropped_ZT_is_brute_force_correlation_summed_over_images(dims, fs):
    rng = np.random.default_rng(72)
    N, K = 3, 2
    z = rng.standard_normal((N, K) + dims)
    g = rng.standard_normal((N,) + dims)
    got = O.crop_support(O.LearningOperators(z).ZT(g), fs)
    for k in range(K):
        want = sum(brute_corr_taps(z[n, k], g[n], fs) for n in range(N))
        np.testing.assert_allclose(got[k], want, atol=1e-12)


@pytest.mark.parametrize("dims", [(6, 7), (4, 5, 6)])
def test_Z_and_ZT_are_adjoint(dims):
    rng = np.random.default_rng(73)
    N, K = 3, 4
    ops = O.LearningOperators(rng.standard_normal((N, K) + dims))
    e = rng.standard_normal((K,) + dims)
    g = rng.standard_normal((N,) + dims)
    lhs = float(np.sum(ops.Z(e) * g))
    rhs = float(np.sum(e * ops.ZT(g)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_Z_matches_the_coding_model_with_roles_exchanged():
    # Z_k S^T d_k summed over k is D z of Eq. 1: the learning model and the coding model agree
    rng = np.random.default_rng(74)
    N, K, dims, fs = 2, 3, (7, 6), (3, 3)
    z = rng.standard_normal((N, K) + dims)
    d = rng.standard_normal((K, 1) + fs)
    via_z = O.LearningOperators(z).Z(O.pad_support(d[:, 0], dims))
    np.testing.assert_allclose(via_z, O.synthesize(d, z)[:, 0], atol=1e-12)
