"""Pins for the oracle's learning subproblem (Sec. 3.2, Eqs. Learning_gamma, Learning_Solution, mu_update)
and the alternating loop (Algorithm 1).

* for fixed mu, the dual gamma route equals a dense solve of the primal normal equations;
* N = K = 1 with z a unit impulse: d* = S x / max(1, ||S x||) in closed form;
* run to convergence, the mu fixed point reaches the constrained optimum found by projected gradient;
* with converged subproblems the joint objective decreases monotonically (Sec. 3.2, Coordinate Descent).
"""
import numpy as np
import pytest

from oracle import csc_oracle as O


def codes(seed, N, K, dims, density=0.2):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((N, K) + dims) < density, rng.standard_normal((N, K) + dims), 0.0)


@pytest.mark.parametrize("J", [1, 2])
def test_gamma_route_equals_dense_normal_equations(J):
    rng = np.random.default_rng(30 + J)
    N, K, dims, fs = 2, 3, (7, 8), (3, 3)
    z = codes(31, N, K, dims)
    x = rng.standard_normal((N, J) + dims)
    mu = np.array([0.3, 0.7, 1.9])
    d0 = rng.standard_normal((K, J) + fs)
    # one step without the final projection: compare d(mu) only
    ops = O.LearningOperators(z)
    want = O.learn_normal_equations(x, z, d0.shape, mu)
    scale = 1.0 / (2.0 * mu)

    def apply(g):
        e = O.pad_support(O.crop_support(ops.ZT(g), fs), dims) * scale[:, None, None]
        return g + ops.Z(e)

    for j in range(J):
        g, _ = O.conjugate_gradient(apply, -x[:, j], np.zeros((N,) + dims), 1e-13, 1000)
        got = -O.crop_support(ops.ZT(g), fs) * scale[:, None, None]
        np.testing.assert_allclose(got, want[:, j], atol=1e-10)


def test_impulse_code_gives_projected_crop():
    rng = np.random.default_rng(40)
    dims, fs = (9, 10), (3, 3)
    z = np.zeros((1, 1) + dims)
    z[0, 0, 0, 0] = 1.0
    for scale in (0.1, 5.0):   # inside and outside the unit ball
        x = scale * rng.standard_normal((1, 1) + dims)
        d, mu, _, _ = O.learn_paper(x, z, np.ones((1, 1) + fs) / 3.0, np.array([0.5]),
                                    np.zeros_like(x), steps=200)
        sx = O.crop_support(x[0, 0], fs)
        want = sx / max(1.0, np.linalg.norm(sx))
        np.testing.assert_allclose(d[0, 0], want, atol=1e-7)


def projected_gradient_learning(x, z, d0, iters):
    """Projected gradient on 1/2||x - Z S^T d||^2 over the product of unit balls (exact projection)."""
    fs = d0.shape[2:]
    K, J = d0.shape[:2]
    ops = O.LearningOperators(z)
    dims = ops.dims
    # Lipschitz bound: power iteration on S Z^T Z S^T
    e = np.random.default_rng(0).standard_normal((K,) + fs)
    for _ in range(200):
        e = O.crop_support(ops.ZT(ops.Z(O.pad_support(e, dims))), fs)
        L = np.linalg.norm(e)
        e /= L
    d = d0.copy()
    for _ in range(iters):
        for j in range(J):
            r = ops.Z(O.pad_support(d[:, j], dims)) - x[:, j]
            d[:, j] -= O.crop_support(ops.ZT(r), fs) / L
        d = O.project_unit_ball(d)
    return d


def test_mu_fixed_point_reaches_constrained_optimum():
    rng = np.random.default_rng(50)
    N, K, dims, fs = 2, 2, (8, 8), (3, 3)
    z = codes(51, N, K, dims, density=0.3)
    x = 3.0 * rng.standard_normal((N, 1) + dims)   # large data: constraint active
    d0 = rng.standard_normal((K, 1) + fs)
    d0 = O.project_unit_ball(d0)
    d, mu, _, _ = O.learn_paper(x, z, d0, np.full(K, 0.5), np.zeros_like(x), steps=300)
    d_pg = projected_gradient_learning(x, z, d0, 20000)
    f = lambda dd: 0.5 * np.sum((x - O.synthesize(dd, z)) ** 2)
    assert abs(f(d) - f(d_pg)) <= 1e-7 * f(d_pg)
    np.testing.assert_allclose(d, d_pg, atol=1e-5)
    norms = np.sqrt((d.reshape(K, -1) ** 2).sum(1))
    np.testing.assert_allclose(norms, 1.0, atol=1e-8)      # active constraints, mu_k > 0


def test_inactive_filter_keeps_d_and_mu():
    rng = np.random.default_rng(60)
    N, K, dims, fs = 2, 3, (7, 7), (3, 3)
    z = codes(61, N, K, dims)
    z[:, 1] = 0.0
    x = rng.standard_normal((N, 1) + dims)
    d0 = O.project_unit_ball(rng.standard_normal((K, 1) + fs))
    d, mu, _, _ = O.learn_paper(x, z, d0, np.full(K, 0.5), np.zeros_like(x), steps=3)
    np.testing.assert_array_equal(d[1], d0[1])
    assert mu[1] == 0.5


def test_alternation_is_monotone_with_converged_subproblems():
    from paper_1709_09479_gb300 import inputs
    data = inputs.sparse_synthetic(seed=7, N=2, dims=(16, 16), K=3, s=3, density=0.05)
    x = data["x"]
    d0 = inputs.unit_filters(8, 3, 1, (3, 3))
    out = O.csc_alternate(x, d0, beta=0.1, rho=1.0, n_outer=4, n_code=600, n_learn=60)
    seq = []
    for h in out["history"]:
        seq += [h["f_code"], h["f_learn"]]
    for a, b in zip(seq, seq[1:]):
        assert b <= a * (1 + 1e-6), seq
