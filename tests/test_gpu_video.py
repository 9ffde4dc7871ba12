"""GPU parity of video coding and learning (the higher-order extension of Sec. 3.3 with a time axis,
3-D DFTs): the CUDA path through csc_init_video / csc_code / csc_objective / csc_learn against the
float64 oracle, which runs the same dual ADMM (Eq. Inference_solution) and learning (Sec. 3.2) with
n-dimensional transforms.

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
    sv = csc.Solver(J=1, K=2, fs=(13, 13), ft=3, dims=(8, 128, 128), n_images=1, beta=0.5, rho=1.0)
    with pytest.raises(csc.CscError) as e:   # a 25-tap lag window per axis: beyond the learning kernels
        sv.learn(np.zeros((1, 1, 8, 128, 128), np.float32), np.zeros((1, 2, 8, 128, 128), np.float32),
                 np.zeros((2, 1, 3, 13, 13), np.float32), np.full(2, 0.5), 1)
    assert e.value.status == 2
    sv.close()


LEARN_CASES = [
    # (N, K, J, T, ft, s, steps); N <= 2 forms the per-frequency products inside the lag window's
    # partial DFTs, N = 3 goes through the materialised tensor-core Gram
    (1, 3, 1, 6, 3, 5, 2),
    (1, 4, 3, 4, 3, 5, 2),
    (2, 3, 3, 4, 3, 5, 2),
    (3, 2, 1, 4, 3, 5, 2),
]


@pytest.mark.parametrize("N,K,J,T,ft,s,steps", LEARN_CASES)
def test_video_learning_matches_oracle(csc, N, K, J, T, ft, s, steps):
    """Learning on video tensors (Sec. 3.2 with 3-D DFTs, Sec. 3.3's channels): the GPU's
    filter-space normal equations against the oracle's dual gamma route, element by element."""
    import torch
    from paper_1709_09479_gb300 import inputs
    x = f32(inputs.powerlaw_field(80 + T, N, J, (T, 128, 128))).astype(np.float64)
    d = f32(inputs.unit_filters(81 + T, K, J, (ft, s, s))).astype(np.float64)
    _, z = O.code_admm(x, d, 0.3, 1.0, 20)
    z = f32(z).astype(np.float64)
    mu0 = np.full(K, 0.5)
    d_o, mu_o, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), steps)
    sv = csc.Solver(J=J, K=K, fs=(s, s), ft=ft, dims=(T, 128, 128), n_images=N, beta=0.3, rho=1.0,
                    cg_tol=1e-7, cg_max=400)
    dv = to_cuda(d)
    mu = torch.tensor(mu0, device="cuda")
    its = sv.learn(to_cuda(x), to_cuda(z), dv, mu, steps)
    sv.close()
    d_g, mu_g = to_np(dv), mu.cpu().numpy()
    print(f"video learning: CG iterations {its}, filters rel err {rel(d_g, d_o):.2e}")
    assert len(its) == steps and all(0 < i <= 400 for i in its)
    assert rel(d_g, d_o) <= REL_TOL
    assert maxrel(d_g, d_o) <= 3 * REL_TOL
    np.testing.assert_allclose(mu_g, mu_o, rtol=REL_TOL)


def test_video_learning_full_size_normal_equations(csc):
    """The RGB video workload's full size (3 x 32 x 128 x 128, K = 64 colour filters 5 x 11 x 11): one
    learning step's filters against the normal equations (S Z^T Z S^T + 2 diag mu) d_j = S Z^T x_j, with
    Z and Z^T applied by the oracle's float64 3-D operators; the codes are the GPU's own."""
    import torch
    N, K, J, T, ft, s, beta, rho = 1, 64, 3, 32, 5, 11, 0.5, 0.1
    x, d = problem(4, N, K, J, T, ft, s)
    sv = csc.Solver(J=J, K=K, fs=(s, s), ft=ft, dims=(T, 128, 128), n_images=N, beta=beta, rho=rho,
                    cg_tol=1e-6, cg_max=400)
    v = torch.zeros((N, K, T, 128, 128), device="cuda")
    zt = torch.empty_like(v)
    sv.code(to_cuda(x), to_cuda(d), v, zt, 10)
    mu0 = np.full(K, 0.5)
    dv = to_cuda(d)
    mu = torch.tensor(mu0, device="cuda")
    its = sv.learn(to_cuda(x), zt, dv, mu, 1)
    sv.close()
    z = to_np(zt)
    d_out, mu1 = to_np(dv), mu.cpu().numpy()
    assert 0 < its[0] <= 400
    active = np.array([np.any(z[:, k] != 0) for k in range(K)])
    ok = active & (mu1 > 10 * O.MU_FLOOR)
    assert ok.sum() >= K // 2
    d_pre = d_out * np.maximum(1.0, mu1 / mu0)[:, None, None, None, None]
    ops = O.LearningOperators(z)
    fs = (ft, s, s)
    res_num = res_den = 0.0
    for j in range(J):
        lhs = O.crop_support(ops.ZT(ops.Z(O.pad_support(d_pre[:, j], ops.dims))), fs) \
            + 2.0 * mu0[:, None, None, None] * d_pre[:, j]
        rhs = O.crop_support(ops.ZT(x[:, j]), fs)
        res_num += np.sum((lhs - rhs)[ok] ** 2)
        res_den += np.sum(rhs[ok] ** 2)
    res = np.sqrt(res_num / res_den)
    print(f"full-size video learning: CG iterations {its[0]}, normal-equation residual {res:.2e}")
    assert res <= 1e-4
    assert np.all(np.sqrt((d_out.reshape(K, -1) ** 2).sum(1)) <= 1 + 1e-5)


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


def video_learn_case():
    """A small video learning problem (N=1, K=3 grey filters 3 x 5 x 5, 6 frames) and its oracle codes."""
    from paper_1709_09479_gb300 import inputs
    N, K, J, T, ft, s = 1, 3, 1, 6, 3, 5
    x = f32(inputs.powerlaw_field(86, N, J, (T, 128, 128))).astype(np.float64)
    d = f32(inputs.unit_filters(87, K, J, (ft, s, s))).astype(np.float64)
    _, z = O.code_admm(x, d, 0.3, 1.0, 20)
    return x, f32(z).astype(np.float64), d


def video_solver(csc, x, d, **kw):
    N, J, T = x.shape[:3]
    K, ft, s = d.shape[0], d.shape[2], d.shape[3]
    args = dict(J=J, K=K, fs=(s, s), ft=ft, dims=(T, 128, 128), n_images=N, beta=0.3, rho=1.0, cg_tol=1e-7,
                cg_max=400)
    args.update(kw)
    return csc.Solver(**args)


def test_video_cg_wait_limit_times_out_then_context_learns_normally(csc):
    """The persistent video CG's exchange waits honour csc_set_wait_limit: with a one-clock bound a
    wait gives up, every CTA returns and csc_learn reports CSC_ERR_TIMEOUT; the same context then
    learns normally and matches the oracle."""
    import torch
    x, z, d = video_learn_case()
    K = d.shape[0]
    mu0 = np.full(K, 0.5)
    d_o, mu_o, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), 2)
    with video_solver(csc, x, d) as sv:
        sv.set_wait_limit(1)
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(z), to_cuda(d), torch.tensor(mu0, device="cuda"), 2)
        assert e.value.status == 7
        sv.set_wait_limit(0)
        dv, mu = to_cuda(d), torch.tensor(mu0, device="cuda")
        sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
        assert rel(to_np(dv), d_o) <= REL_TOL
        np.testing.assert_allclose(mu.cpu().numpy(), mu_o, rtol=REL_TOL)


def test_video_nan_codes_stop_the_cg_with_nonfinite(csc):
    import torch
    x, z, d = video_learn_case()
    zb = z.copy()
    zb[0, 1, 2, 5, 5] = np.nan
    with video_solver(csc, x, d) as sv:
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(zb), to_cuda(d), torch.full((d.shape[0],), 0.5, dtype=torch.float64,
                                                                        device="cuda"), 2)
        assert e.value.status == 5


def test_video_cg_stopped_at_its_cap(csc):
    """cg_max = 1: one CG iteration per learning step is reported; with CSC_FLAG_CG_STRICT the call
    returns CSC_ERR_NOT_CONVERGED."""
    import torch
    x, z, d = video_learn_case()
    mu = lambda: torch.full((d.shape[0],), 0.5, dtype=torch.float64, device="cuda")
    with video_solver(csc, x, d, cg_max=1, cg_tol=1e-9) as sv:
        assert sv.learn(to_cuda(x), to_cuda(z), to_cuda(d), mu(), 3) == [1, 1, 1]
    with video_solver(csc, x, d, cg_max=1, cg_tol=1e-9, flags=csc.CSC_FLAG_CG_STRICT) as sv:
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(z), to_cuda(d), mu(), 3)
        assert e.value.status == 6
