"""GPU parity of video coding (the higher-order extension of Sec. 3.3 with a time axis, 3-D DFTs):
the CUDA path through csc_init_video / csc_code / csc_objective against the float64 oracle, which
runs the same dual ADMM (Eq. Inference_solution) with n-dimensional transforms.

Cases: grey and colour (J = 1, 3), odd and even frame counts, time supports 1, 3 and 5, a warm
start, host-pointer arguments, and the objective of Eq. 1.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

CASES = [
    # (N, K, J, T, ft, s, beta, rho, iters)
    (1, 4, 3, 8, 3, 5, 0.5, 1.0, 6),
    (2, 3, 1, 5, 5, 3, 0.3, 0.5, 5),
    (1, 2, 1, 4, 1, 7, 0.2, 2.0, 4),
]


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def problem(seed, N, K, J, T, ft, s):
    from paper_1709_09479_gb300 import inputs
    x = f32(inputs.powerlaw_field(seed, N, J, (T, 128, 128))).astype(np.float64)
    d = f32(inputs.unit_filters(seed + 1, K, J, (ft, s, s))).astype(np.float64)
    return x, d


def run_gpu(csc, x, d, beta, rho, iters, v0=None, host=False):
    import torch
    N, J, T = x.shape[:3]
    K, ft, s = d.shape[0], d.shape[2], d.shape[3]
    sv = csc.Solver(J=J, K=K, fs=(s, s), ft=ft, dims=(T, 128, 128), n_images=N, beta=beta, rho=rho)
    shape = (N, K, T, 128, 128)
    if host:
        v = np.zeros(shape, np.float32) if v0 is None else f32(v0)
        z = np.zeros_like(v)
        sv.code(f32(x), f32(d), v, z, iters)
        out = v.astype(np.float64), z.astype(np.float64)
    else:
        v = torch.zeros(shape, device="cuda") if v0 is None else to_cuda(v0)
        z = torch.empty_like(v)
        sv.code(to_cuda(x), to_cuda(d), v, z, iters)
        torch.cuda.synchronize()
        out = to_np(v), to_np(z)
    sv.close()
    return out


@pytest.mark.parametrize("N,K,J,T,ft,s,beta,rho,iters", CASES)
def test_video_coding_matches_oracle(csc, N, K, J, T, ft, s, beta, rho, iters):
    x, d = problem(70 + T, N, K, J, T, ft, s)
    v_o, z_o = O.code_admm(x, d, beta, rho, iters)
    v_g, z_g = run_gpu(csc, x, d, beta, rho, iters)
    assert np.count_nonzero(z_o) > 0
    assert rel(v_g, v_o) <= REL_TOL
    assert rel(z_g, z_o) <= REL_TOL
    assert maxrel(v_g, v_o) <= REL_TOL


def test_video_warm_start_and_host_pointers(csc):
    N, K, J, T, ft, s, beta, rho = 1, 3, 3, 6, 3, 5, 0.4, 1.0
    x, d = problem(90, N, K, J, T, ft, s)
    v1, _ = O.code_admm(x, d, beta, rho, 3)
    v_o, z_o = O.code_admm(x, d, beta, rho, 4, v0=v1)
    v_g, z_g = run_gpu(csc, x, d, beta, rho, 4, v0=v1, host=True)
    assert rel(v_g, v_o) <= REL_TOL
    assert rel(z_g, z_o) <= REL_TOL


def test_video_objective_matches_oracle(csc):
    import torch
    N, K, J, T, ft, s, beta, rho = 1, 4, 3, 8, 3, 5, 0.5, 1.0
    x, d = problem(95, N, K, J, T, ft, s)
    _, z_o = O.code_admm(x, d, beta, rho, 5)
    zf = f32(z_o).astype(np.float64)
    f_o = O.objective(x, d, zf, beta)
    sv = csc.Solver(J=J, K=K, fs=(s, s), ft=ft, dims=(T, 128, 128), n_images=N, beta=beta, rho=rho)
    f_g = sv.objective(to_cuda(x), to_cuda(d), to_cuda(zf))
    sv.close()
    assert abs(f_g - f_o) <= 1e-5 * abs(f_o)


def test_video_rejects_unsupported_shapes(csc):
    with pytest.raises(csc.CscError):
        csc.Solver(J=1, K=2, fs=(3, 3), ft=3, dims=(8, 64, 64), n_images=1, beta=0.5, rho=1.0)
    with pytest.raises(csc.CscError):
        csc.Solver(J=1, K=2, fs=(3, 3), ft=4, dims=(8, 128, 128), n_images=1, beta=0.5, rho=1.0)
    sv = csc.Solver(J=1, K=2, fs=(3, 3), ft=3, dims=(8, 128, 128), n_images=1, beta=0.5, rho=1.0)
    with pytest.raises(csc.CscError) as e:
        sv.learn(np.zeros((1, 1, 8, 128, 128), np.float32), np.zeros((1, 2, 8, 128, 128), np.float32),
                 np.zeros((2, 1, 3, 3, 3), np.float32), np.full(2, 0.5), 1)
    assert e.value.status == 8
    sv.close()


def test_video_full_size_matches_oracle(csc):
    """The RGB video workload's full size (3 x 32 x 128 x 128, K = 64 filters 5 x 11 x 11), two ADMM
    iterations, element by element against the oracle."""
    N, K, J, T, ft, s, beta, rho = 1, 64, 3, 32, 5, 11, 0.5, 0.1
    x, d = problem(4, N, K, J, T, ft, s)
    v_o, z_o = O.code_admm(x, d, beta, rho, 2)
    v_g, z_g = run_gpu(csc, x, d, beta, rho, 2)
    assert np.count_nonzero(z_o) > 0
    assert rel(v_g, v_o) <= REL_TOL
    assert rel(z_g, z_o) <= REL_TOL
