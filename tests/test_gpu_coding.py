"""GPU parity of the coding subproblem (Sec. 3.2, Eq. Inference_solution) and the objective (Eq. 1):
the CUDA path through the C ABI against the float64 oracle, element by element, on seeded inputs.

Cases span the fixed-size FFT instantiations (64x64, 100x100, 128x128) and the run-time one,
J = 1 and J = 3 (Sec. 3.3), map counts below, at and above the number of SMs (so a CTA's range of
maps spans image boundaries), warm starts, and host-pointer arguments.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, make_problem, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

CASES = [
    # (N, K, J, dims, s, beta, rho, iters)
    (2, 3, 1, (64, 64), 5, 0.2, 1.0, 7),        # fixed-size 64 x 64
    (2, 4, 1, (48, 40), 5, 0.3, 2.0, 5),        # run-time geometry (48 = 16*3, 20 = 4*5)
    (2, 3, 3, (24, 32), 3, 0.25, 1.5, 4),       # J = 3: per-frequency 3 x 3 solve, run-time geometry
    (3, 5, 1, (100, 100), 11, 1.0, 10.0, 3),    # 100 x 100 (the 10-image sparse workload's size)
    (1, 2, 1, (128, 128), 11, 1.0, 10.0, 2),    # 128 x 128
    (7, 50, 1, (64, 64), 5, 0.5, 1.0, 3),       # 350 maps: CTAs cover several images each
    (1, 1, 1, (8, 8), 1, 0.1, 1.0, 2),          # smallest grid, 1 x 1 filter
]


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def run_gpu(csc, x, d, beta, rho, iters, v0=None, host=False):
    N, J = x.shape[:2]
    K = d.shape[0]
    dims = x.shape[2:]
    s = d.shape[2:]
    solver = csc.Solver(J=J, K=K, fs=s, dims=dims, n_images=N, beta=beta, rho=rho)
    if host:
        xv, dv = f32(x), f32(d)
        v = np.zeros((N, K) + dims, np.float32) if v0 is None else f32(v0)
        z = np.zeros_like(v)
        solver.code(xv, dv, v, z, iters)
        out = v.astype(np.float64), z.astype(np.float64)
    else:
        import torch
        xv, dv = to_cuda(x), to_cuda(d)
        v = torch.zeros((N, K) + dims, device="cuda") if v0 is None else to_cuda(v0)
        z = torch.empty_like(v)
        solver.code(xv, dv, v, z, iters)
        torch.cuda.synchronize()
        out = to_np(v), to_np(z)
    solver.close()
    return out


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}K{c[1]}J{c[2]}_{c[3][0]}x{c[3][1]}_s{c[4]}")
def test_coding_matches_oracle(csc, case):
    N, K, J, dims, s, beta, rho, iters = case
    x, d = make_problem(11 + K, N, K, J, dims, s)
    v, z = run_gpu(csc, x, d, beta, rho, iters)
    vo, zo = O.code_admm(x, d, beta, rho, iters)
    assert rel(v, vo) <= REL_TOL, rel(v, vo)
    assert maxrel(v, vo) <= REL_TOL
    if np.any(zo != 0):
        assert rel(z, zo) <= REL_TOL, rel(z, zo)
        assert maxrel(z, zo) <= REL_TOL


def test_warm_start_and_split_calls_equal_one_call(csc):
    """Algorithm 1 warm-starts the ADMM state: 3 + 4 iterations equal 7, and equal the oracle."""
    N, K, J, dims, s, beta, rho = 2, 6, 1, (64, 64), 5, 0.3, 1.0
    x, d = make_problem(5, N, K, J, dims, s)
    v1, _ = run_gpu(csc, x, d, beta, rho, 3)
    v2, z2 = run_gpu(csc, x, d, beta, rho, 4, v0=v1)
    v7, z7 = run_gpu(csc, x, d, beta, rho, 7)
    vo, zo = O.code_admm(x, d, beta, rho, 7)
    assert maxrel(v2, v7) <= 1e-5
    assert rel(z2, zo) <= REL_TOL and rel(z7, zo) <= REL_TOL


def test_host_pointers_give_the_device_result(csc):
    N, K, J, dims, s, beta, rho = 2, 4, 1, (48, 40), 5, 0.3, 2.0
    x, d = make_problem(6, N, K, J, dims, s)
    vd, zd = run_gpu(csc, x, d, beta, rho, 3)
    vh, zh = run_gpu(csc, x, d, beta, rho, 3, host=True)
    np.testing.assert_array_equal(vh, vd)
    np.testing.assert_array_equal(zh, zd)


def test_zero_iterations_only_maps_state_to_codes(csc):
    import torch
    N, K, dims = 2, 3, (64, 64)
    x, d = make_problem(7, N, K, 1, dims, 5)
    v0 = np.random.default_rng(0).standard_normal((N, K) + dims)
    v, z = run_gpu(csc, x, d, 0.4, 3.0, 0, v0=v0)
    want = 3.0 * (np.clip(f32(v0), -0.4, 0.4) - f32(v0))
    np.testing.assert_allclose(z, want, rtol=1e-6, atol=1e-6)


def test_large_beta_gives_exact_zero_codes(csc):
    N, K, dims, s = 2, 3, (64, 64), 5
    x, d = make_problem(8, N, K, 1, dims, s)
    beta = 1.5 * float(np.max(np.abs(O.correlate(d, x))))
    _, z = run_gpu(csc, x, d, beta, 1.0, 30)
    assert np.all(z == 0.0)


@pytest.mark.parametrize("case", [(3, 5, 1, (100, 100), 11), (2, 3, 3, (24, 32), 3), (7, 50, 1, (64, 64), 5)])
def test_objective_matches_oracle(csc, case):
    N, K, J, dims, s = case
    x, d = make_problem(21, N, K, J, dims, s)
    rng = np.random.default_rng(3)
    z = f32(np.where(rng.random((N, K) + dims) < 0.05, rng.standard_normal((N, K) + dims), 0.0)).astype(np.float64)
    solver = csc.Solver(J=J, K=K, fs=(s, s), dims=dims, n_images=N, beta=0.7, rho=1.0)
    f = solver.objective(to_cuda(x), to_cuda(d), to_cuda(z))
    fh = solver.objective(f32(x), f32(d), f32(z))
    solver.close()
    fo = O.objective(x, d, z, 0.7)
    assert abs(f - fo) <= 1e-5 * fo, (f, fo)
    assert abs(fh - f) <= 1e-12 * fo
