"""Pins for the oracle's grid operators, per-frequency solve and objective (Sec. 3.1-3.2).

Every check compares the oracle with something other than itself: brute-force circular loops,
explicit dense matrices solved with numpy.linalg, or exact identities.
"""
import itertools

import numpy as np
import pytest

from oracle import csc_oracle as O


def brute_conv(d, z):
    """(d*z)(p) = sum_a d[a] z[(p - (a - c)) mod dims], c = (f-1)//2, by explicit loops."""
    out = np.zeros(z.shape)
    dims = z.shape
    for a in itertools.product(*[range(f) for f in d.shape]):
        off = [ai - (f - 1) // 2 for ai, f in zip(a, d.shape)]
        for p in itertools.product(*[range(n) for n in dims]):
            q = tuple((pi - oi) % n for pi, oi, n in zip(p, off, dims))
            out[p] += d[a] * z[q]
    return out


def brute_corr(d, lam):
    """(d ⋆ lam)(p) = sum_a d[a] lam[(p + (a - c)) mod dims]."""
    out = np.zeros(lam.shape)
    dims = lam.shape
    for a in itertools.product(*[range(f) for f in d.shape]):
        off = [ai - (f - 1) // 2 for ai, f in zip(a, d.shape)]
        for p in itertools.product(*[range(n) for n in dims]):
            q = tuple((pi + oi) % n for pi, oi, n in zip(p, off, dims))
            out[p] += d[a] * lam[q]
    return out


def dense_D(d, dims):
    """Explicit (J*D) x (K*D) matrix of z -> Dz built from brute_conv of unit impulses."""
    K, J = d.shape[:2]
    Dn = int(np.prod(dims))
    M = np.zeros((J * Dn, K * Dn))
    for k in range(K):
        for i in range(Dn):
            e = np.zeros(dims)
            e.reshape(-1)[i] = 1.0
            for j in range(J):
                M[j * Dn:(j + 1) * Dn, k * Dn + i] = brute_conv(d[k, j], e).reshape(-1)
    return M


@pytest.mark.parametrize("dims,fs", [((6, 7), (3, 3)), ((5, 8), (3, 5)), ((4, 6, 5), (3, 3, 3))])
def test_synthesize_matches_brute_force(dims, fs):
    rng = np.random.default_rng(1)
    K, J, N = 3, 2, 2
    d = rng.standard_normal((K, J) + fs)
    z = rng.standard_normal((N, K) + dims)
    got = O.synthesize(d, z)
    for n in range(N):
        for j in range(J):
            want = sum(brute_conv(d[k, j], z[n, k]) for k in range(K))
            np.testing.assert_allclose(got[n, j], want, atol=1e-12)


@pytest.mark.parametrize("dims,fs", [((6, 7), (3, 3)), ((4, 6, 5), (3, 3, 3))])
def test_correlate_matches_brute_force_and_is_adjoint(dims, fs):
    rng = np.random.default_rng(2)
    K, J, N = 3, 2, 2
    d = rng.standard_normal((K, J) + fs)
    lam = rng.standard_normal((N, J) + dims)
    got = O.correlate(d, lam)
    for n in range(N):
        for k in range(K):
            want = sum(brute_corr(d[k, j], lam[n, j]) for j in range(J))
            np.testing.assert_allclose(got[n, k], want, atol=1e-12)
    z = rng.standard_normal((N, K) + dims)
    lhs = np.sum(O.synthesize(d, z) * lam)
    rhs = np.sum(z * O.correlate(d, lam))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_pad_crop_place_taps_at_centred_offsets():
    d = np.arange(1.0, 10.0).reshape(3, 3)
    g = O.pad_support(d, (5, 6))
    # centre tap (1,1) -> origin; tap (0,0) -> offset (-1,-1) -> (4,5)
    assert g[0, 0] == d[1, 1] and g[4, 5] == d[0, 0] and g[1, 1] == d[2, 2] and g[0, 1] == d[1, 2]
    assert np.count_nonzero(g) == 9
    np.testing.assert_array_equal(O.crop_support(g, (3, 3)), d)


@pytest.mark.parametrize("J", [1, 3])
def test_per_frequency_solve_equals_dense_solve(J):
    """(D D^T + I/rho)^{-1} rhs via an explicit dense matrix equals the per-frequency closed form."""
    rng = np.random.default_rng(3)
    dims, fs, K, rho = (4, 5), (3, 3), 3, 0.7
    d = rng.standard_normal((K, J) + fs)
    rhs = rng.standard_normal((1, J) + dims)
    Dm = dense_D(d, dims)
    want = np.linalg.solve(Dm @ Dm.T + np.eye(Dm.shape[0]) / rho, rhs.reshape(-1))
    dh = O.filter_spectra(d, dims)
    got = O.irdft(O.solve_per_frequency(dh, rho, O.rdft(rhs, 2)), dims)
    np.testing.assert_allclose(got.reshape(-1), want, atol=1e-11)


def test_objective_matches_dense():
    rng = np.random.default_rng(4)
    dims, fs, K, J = (5, 4), (3, 3), 2, 2
    d = rng.standard_normal((K, J) + fs)
    z = rng.standard_normal((1, K) + dims)
    x = rng.standard_normal((1, J) + dims)
    Dm = dense_D(d, dims)
    r = x.reshape(-1) - Dm @ z.reshape(-1)
    want = 0.5 * r @ r + 0.3 * np.abs(z).sum()
    assert abs(O.objective(x, d, z, 0.3) - want) <= 1e-11 * want


def test_lipschitz_is_largest_singular_value_squared():
    rng = np.random.default_rng(5)
    dims, fs, K, J = (5, 6), (3, 3), 3, 2
    d = rng.standard_normal((K, J) + fs)
    Dm = dense_D(d, dims)
    want = np.linalg.norm(Dm, 2) ** 2
    assert abs(O.lipschitz(d, dims) - want) <= 1e-10 * want
