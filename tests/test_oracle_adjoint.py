"""Pins for the oracle's reverse mode through T unrolled coding iterations: central finite
differences in float64 on tiny instances, away from the clamp kinks."""
import numpy as np
import pytest

from oracle import csc_oracle as O


def kink_margin(x, d, beta, rho, T):
    v = np.zeros((x.shape[0], d.shape[0]) + x.shape[2:])
    m = np.inf
    for _ in range(T + 1):
        m = min(m, float(np.min(np.abs(np.abs(v) - beta))))
        v, _ = O.code_admm(x, d, beta, rho, 1, v)
    return m


@pytest.mark.parametrize("J,dims", [(1, (6, 7)), (2, (5, 6))])
def test_unrolled_gradient_matches_finite_differences(J, dims):
    rng = np.random.default_rng(70 + J)
    N, K, fs, T, beta, rho = 2, 2, (3, 3), 4, 0.35, 1.3
    x = rng.standard_normal((N, J) + dims)
    d = rng.standard_normal((K, J) + fs) * 0.6
    y = rng.standard_normal((N, J) + dims)
    assert kink_margin(x, d, beta, rho, T) > 2e-5   # FD step 1e-6 stays clear of every clamp kink
    loss, gx, gd = O.unrolled_loss_and_grad(x, d, y, beta, rho, T)
    h = 1e-6

    def _loss(xx, dd):
        _, z = O.code_admm(xx, dd, beta, rho, T)
        r = O.synthesize(dd, z) - y
        return float(np.sum(r * r)) / r.size

    assert abs(_loss(x, d) - loss) <= 1e-12 * loss
    for idx in [(0, 0, 1, 2), (1, J - 1, 3, 4), (0, 0, 0, 0)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (_loss(x + e, d) - _loss(x - e, d)) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (idx, fd, gx[idx])
    for idx in [(0, 0, 1, 1), (1, J - 1, 0, 2), (0, 0, 2, 0)]:
        e = np.zeros_like(d)
        e[idx] = h
        fd = (_loss(x, d + e) - _loss(x, d - e)) / (2 * h)
        assert abs(fd - gd[idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (idx, fd, gd[idx])
