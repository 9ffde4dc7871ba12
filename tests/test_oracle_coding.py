"""Pins for the oracle's coding subproblem (Sec. 3.2, Eq. Inference_solution).

* the v-state form equals the three-variable form of the paper step by step;
* the multiplier update is the l1 soft-threshold (Moreau identity);
* run to convergence, ADMM reaches the lasso optimum found by FISTA, with a vanishing duality gap
  and the KKT conditions of Eq. 2;
* closed-form special cases: beta >= ||D^T x||_inf gives z = 0; a 1x1 filter gives scalar lasso.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O


def tiny(seed, dims=(10, 12), K=3, J=1, s=3, N=2):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((K, J) + (s,) * len(dims))
    d /= np.sqrt((d.reshape(K, -1) ** 2).sum(1)).reshape((K,) + (1,) * (d.ndim - 1))
    x = rng.standard_normal((N, J) + dims)
    return x, d


@pytest.mark.parametrize("J,dims", [(1, (10, 12)), (3, (6, 8)), (2, (4, 6, 5))])
def test_vform_equals_textbook_form(J, dims):
    x, d = tiny(10 + J, dims=dims, J=J)
    beta, rho = 0.4, 1.7
    for iters in (1, 2, 7):
        v, z = O.code_admm(x, d, beta, rho, iters)
        zt, theta, _ = O.code_admm_textbook(x, d, beta, rho, iters)
        np.testing.assert_allclose(z, zt, atol=1e-12 * max(1.0, np.abs(zt).max()))
        np.testing.assert_allclose(np.clip(v, -beta, beta), theta, atol=1e-12)


def test_multiplier_update_is_soft_threshold():
    rng = np.random.default_rng(0)
    v = 3.0 * rng.standard_normal(1000)
    beta, rho = 0.8, 2.5
    z = rho * (np.clip(v, -beta, beta) - v)
    soft = np.sign(v) * np.maximum(np.abs(v) - beta, 0.0)
    np.testing.assert_allclose(z, -rho * soft, atol=1e-14)
    # and z^{i+1} = soft_{rho beta}(z^i - rho D^T lam): here z^i - rho D^T lam = -rho v
    a = -rho * v
    np.testing.assert_allclose(z, np.sign(a) * np.maximum(np.abs(a) - rho * beta, 0.0), atol=1e-13)
    assert np.all(z[np.abs(v) <= beta] == 0.0)


def test_admm_reaches_fista_optimum_with_zero_gap():
    x, d = tiny(20, dims=(8, 9), K=2, s=3, N=1)
    beta, rho = 0.3, 1.0
    _, z_admm = O.code_admm(x, d, beta, rho, 8000)
    z_fista = O.fista_code(x, d, beta, 30000)
    f_admm = O.objective(x, d, z_admm, beta)
    f_fista = O.objective(x, d, z_fista, beta)
    assert abs(f_admm - f_fista) <= 1e-9 * f_fista
    np.testing.assert_allclose(z_admm, z_fista, atol=1e-8)
    gap, primal = O.duality_gap(x, d, z_admm, beta)
    assert 0.0 <= gap <= 1e-9 * primal
    # KKT of Eq. 2: |D^T(Dz - x)| <= beta, and = -beta sign(z) on the support
    g = O.correlate(d, O.synthesize(d, z_admm) - x)
    assert np.max(np.abs(g)) <= beta * (1 + 1e-7)
    supp = np.abs(z_admm) > 1e-8
    np.testing.assert_allclose(g[supp], -beta * np.sign(z_admm[supp]), atol=1e-7)


def test_duality_gap_positive_away_from_optimum():
    x, d = tiny(21, dims=(8, 9), K=2, s=3, N=1)
    _, z = O.code_admm(x, d, 0.3, 1.0, 3)
    gap, _ = O.duality_gap(x, d, z, 0.3)
    assert gap > 1e-3


def test_large_beta_gives_zero_codes():
    x, d = tiny(22)
    beta = 1.01 * float(np.max(np.abs(O.correlate(d, x))))
    _, z = O.code_admm(x, d, beta, 2.0, 300)
    assert np.all(z == 0.0)


def test_scalar_filter_is_elementwise_lasso():
    rng = np.random.default_rng(23)
    dval, beta = 1.7, 0.5
    d = np.full((1, 1, 1, 1), dval)
    x = 2.0 * rng.standard_normal((1, 1, 6, 7))
    _, z = O.code_admm(x, d, beta, 1.3, 3000)
    dx = dval * x[:, 0]
    want = np.sign(dx) * np.maximum(np.abs(dx) - beta, 0.0) / dval ** 2
    np.testing.assert_allclose(z[:, 0], want, atol=1e-10)


def test_planted_sign_error_in_multiplier_is_caught(monkeypatch):
    """A plausible mistake (z = rho (v - clamp v)) breaks the two-form equality pin."""
    x, d = tiny(24)
    zt, _, _ = O.code_admm_textbook(x, d, 0.4, 1.7, 5)
    real_clip = np.clip
    v, z = O.code_admm(x, d, 0.4, 1.7, 5)
    bad = 1.7 * (v - real_clip(v, -0.4, 0.4))
    assert np.max(np.abs(bad - zt)) > 1e-3


def test_coding_is_separable_per_image_and_odd_sizes_are_exact_dfts():
    """The coding of a batch is the coding of each image alone (Eq. Inference_solution couples only
    the K maps of one image): the sampled-image parity checks at full size rest on this. On an odd,
    prime-sized grid the oracle's transforms are exact H x W DFTs: its data term equals the spatial
    circular convolution computed tap by tap."""
    x, d = tiny(77, dims=(13, 11), K=3, N=3)
    beta, rho = 0.3, 1.3
    v, z = O.code_admm(x, d, beta, rho, 4)
    for n in range(3):
        vn, zn = O.code_admm(x[n:n + 1], d, beta, rho, 4)
        np.testing.assert_allclose(v[n:n + 1], vn, atol=1e-13)
        np.testing.assert_allclose(z[n:n + 1], zn, atol=1e-13)
    # spatial check of the objective's data term on the prime-sized grid
    K, J, s = d.shape[0], d.shape[1], d.shape[-1]
    c = (s - 1) // 2
    H, W = x.shape[-2:]
    rec = np.zeros_like(x)
    for k in range(K):
        for j in range(J):
            for ta in range(s):
                for tb in range(s):
                    rec[:, j] += d[k, j, ta, tb] * np.roll(z[:, k], (ta - c, tb - c), axis=(-2, -1))
    data = 0.5 * ((rec - x) ** 2).sum()
    reg = beta * np.abs(z).sum()
    assert abs(O.objective(x, d, z, beta) - (data + reg)) <= 1e-10 * (data + reg)
