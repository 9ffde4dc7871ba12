"""GPU parity of the symmetric-boundary (DCT) variant the paper mentions at the start of Sec. 3:
CSC_FLAG_SYMMETRIC_BOUNDARY codes the half-sample symmetric extension of the caller's H x W images.

* centre-symmetric filters: the codes equal the float64 oracle's dual ADMM run in the type-II DCT
  domain of the H x W images, and the GPU's extended codes are mirror symmetric;
* general filters: the codes equal the oracle's extended-grid ADMM (both through the fused 128 x 128
  sweep, from 64 x 64 images, and through the run-time geometry);
* learning on such a context equals the oracle's learning on the extended images and codes.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, make_problem, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def centre_symmetric(d):
    return 0.25 * (d + d[..., ::-1, :] + d[..., :, ::-1] + d[..., ::-1, ::-1])


def gpu_code_sym(csc, x, d, beta, rho, iters, host=False):
    import torch
    N, K = x.shape[0], d.shape[0]
    H, W = x.shape[2:]
    s = d.shape[2:]
    with csc.Solver(J=1, K=K, fs=s, dims=(H, W), n_images=N, beta=beta, rho=rho,
                    flags=csc.CSC_FLAG_SYMMETRIC_BOUNDARY) as sv:
        if host:
            v = np.zeros((N, K, 2 * H, 2 * W), dtype=np.float32)
            z = np.zeros_like(v)
            sv.code(f32(x), f32(d), v, z, iters)
            return v.astype(np.float64), z.astype(np.float64)
        v = torch.zeros((N, K, 2 * H, 2 * W), device="cuda")
        z = torch.empty_like(v)
        sv.code(to_cuda(x), to_cuda(d), v, z, iters)
        obj = sv.objective(to_cuda(x), to_cuda(d), z)
        return to_np(v), to_np(z), obj


@pytest.mark.parametrize("dims,s", [((64, 64), 5), ((50, 48), 3)])
def test_symmetric_filters_match_dct_domain_admm(csc, dims, s):
    N, K, beta, rho, iters = 2, 6, 0.1, 1.0, 12
    x, d = make_problem(500, N, K, 1, dims, s)
    d = f32(centre_symmetric(d)).astype(np.float64)
    v, z, obj = gpu_code_sym(csc, x, d, beta, rho, iters)
    H, W = dims
    _, z_dct = O.code_admm_dct(x, d, beta, rho, iters)
    assert np.abs(z_dct).max() > 0
    assert rel(z[..., :H, :W], z_dct) <= REL_TOL
    assert maxrel(z[..., :H, :W], z_dct) <= REL_TOL
    # mirror symmetric extended codes
    assert maxrel(z, O.symmetric_extend(z[..., :H, :W])) <= REL_TOL
    # the objective of the extended problem
    f_ref = O.objective(O.symmetric_extend(x), d, f32(z).astype(np.float64), beta)
    assert abs(obj - f_ref) <= 1e-5 * f_ref


@pytest.mark.parametrize("dims,s,host", [((64, 64), 11, False), ((50, 48), 5, True)])
def test_general_filters_match_extended_grid_admm(csc, dims, s, host):
    N, K, beta, rho, iters = 2, 5, 0.15, 1.0, 10
    x, d = make_problem(501, N, K, 1, dims, s)
    out = gpu_code_sym(csc, x, d, beta, rho, iters, host=host)
    v, z = out[0], out[1]
    v_o, z_o = O.code_admm_symmetric(x, d, beta, rho, iters)
    assert rel(v, v_o) <= REL_TOL and maxrel(v, v_o) <= REL_TOL
    assert rel(z, z_o) <= REL_TOL


def test_learning_on_a_symmetric_boundary_context(csc):
    import torch
    N, K, dims, s, beta, rho = 2, 4, (32, 32), 5, 0.2, 1.0
    x, d = make_problem(502, N, K, 1, dims, s)
    _, z = O.code_admm_symmetric(x, d, beta, rho, 15)
    z = f32(z).astype(np.float64)
    mu0 = np.full(K, 0.5)
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho, cg_max=400, cg_tol=1e-6,
                    flags=csc.CSC_FLAG_SYMMETRIC_BOUNDARY) as sv:
        dv = to_cuda(d)
        mu = torch.tensor(mu0, device="cuda")
        sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
    d_o, mu_o, _, _ = O.learn_paper(O.symmetric_extend(x), z, d, mu0, np.zeros((N, 1) + (64, 64)), 2)
    assert rel(to_np(dv), d_o) <= REL_TOL
    np.testing.assert_allclose(mu.cpu().numpy(), mu_o, rtol=REL_TOL)
