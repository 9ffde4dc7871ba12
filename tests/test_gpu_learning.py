"""GPU parity of the learning subproblem (Sec. 3.2, Eqs. Learning_new .. mu_update) and of
Algorithm 1: the CUDA path through the C ABI against the float64 oracle (which follows the paper's
dual gamma route), element by element on the filters and multipliers.

The GPU solves the filter-space normal equations by float32 CG to a relative residual of 1e-6;
the oracle solves the gamma system to 1e-12. For fixed mu both give the same d (strong duality),
so the filters agree to the CG tolerance times the system's conditioning.
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


def codes_for(x, d, beta, rho, iters):
    _, z = O.code_admm(x, d, beta, rho, iters)
    return f32(z).astype(np.float64)


def gpu_learn(csc, x, z, d, mu, steps, host=False, cg_tol=1e-6, cg_max=400):
    N, J = x.shape[:2]
    K = d.shape[0]
    solver = csc.Solver(J=J, K=K, fs=d.shape[2:], dims=x.shape[2:], n_images=N, beta=1.0, rho=1.0,
                        cg_tol=cg_tol, cg_max=cg_max)
    if host:
        dv = f32(d)
        muv = np.array(mu, dtype=np.float64)
        its = solver.learn(f32(x), f32(z), dv, muv, steps)
        out = dv.astype(np.float64), muv, its
    else:
        import torch
        dv = to_cuda(d)
        muv = torch.tensor(np.asarray(mu, dtype=np.float64), device="cuda")
        its = solver.learn(to_cuda(x), to_cuda(z), dv, muv, steps)
        out = to_np(dv), muv.cpu().numpy(), its
    solver.close()
    return out


LEARN_CASES = [
    # (N, K, J, dims, s, code_beta, steps)
    (2, 3, 1, (32, 32), 5, 0.2, 3),
    (3, 6, 1, (64, 64), 5, 0.3, 4),
    (2, 3, 3, (24, 32), 3, 0.2, 3),
    (4, 8, 1, (100, 100), 11, 0.5, 2),
    # Gram coverage: three image chunks with a ragged tail, colour with three chunks, K + J = 128
    # (the largest tensor-core tile), and K + J > 128 (the CUDA-core Gram) in grey and colour. The
    # many-filter cases have few codes per filter and a CG bound 1e-7, which keeps the CG error
    # (about cond x tolerance) inside the parity bar.
    (37, 20, 1, (32, 32), 5, 0.3, 2),
    (40, 12, 3, (24, 24), 3, 0.3, 2),
    (3, 125, 3, (16, 16), 3, 0.3, 2, 1e-7),
    (3, 128, 1, (16, 16), 3, 0.3, 2, 1e-7),
    (4, 130, 1, (16, 16), 3, 0.3, 2, 2e-8),
    (3, 126, 3, (16, 16), 3, 0.3, 2, 1e-7),
]


@pytest.mark.parametrize("case", LEARN_CASES, ids=lambda c: f"N{c[0]}K{c[1]}J{c[2]}_{c[3][0]}x{c[3][1]}_s{c[4]}")
def test_learning_matches_oracle(csc, case):
    N, K, J, dims, s, beta, steps = case[:7]
    cg_tol = case[7] if len(case) > 7 else 1e-6
    x, d = make_problem(31 + K, N, K, J, dims, s)
    z = codes_for(x, d, beta, 1.0, 30)
    mu0 = np.full(K, 0.5)
    d_gpu, mu_gpu, its = gpu_learn(csc, x, z, d, mu0, steps, cg_tol=cg_tol)
    d_o, mu_o, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), steps)
    assert rel(d_gpu, d_o) <= REL_TOL, rel(d_gpu, d_o)
    assert maxrel(d_gpu, d_o) <= 3 * REL_TOL
    np.testing.assert_allclose(mu_gpu, mu_o, rtol=REL_TOL)
    assert len(its) == steps and all(0 <= i <= 400 for i in its)
    norms = np.sqrt((d_gpu.reshape(K, -1) ** 2).sum(1))
    assert np.all(norms <= 1 + 1e-6)


def test_learning_host_pointers_and_inactive_filter(csc):
    N, K, J, dims, s = 2, 4, 1, (32, 32), 5
    x, d = make_problem(40, N, K, J, dims, s)
    z = codes_for(x, d, 0.2, 1.0, 20)
    z[:, 2] = 0.0                       # filter 2 has no codes: keeps d_2 and mu_2
    mu0 = np.array([0.5, 0.4, 0.3, 0.6])
    d_dev, mu_dev, _ = gpu_learn(csc, x, z, d, mu0, 3)
    d_host, mu_host, _ = gpu_learn(csc, x, z, d, mu0, 3, host=True)
    np.testing.assert_array_equal(d_dev, d_host)
    np.testing.assert_array_equal(mu_dev, mu_host)
    d_o, mu_o, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), 3)
    np.testing.assert_array_equal(d_dev[2], f32(O.project_unit_ball(d)[2]))
    assert mu_dev[2] == 0.3
    assert rel(d_dev, d_o) <= REL_TOL


def test_alternation_matches_oracle(csc):
    """Algorithm 1 with warm-started coding state: 3 outer rounds of 10 coding + 4 learning steps."""
    import torch
    N, K, J, dims, s = 2, 4, 1, (32, 32), 5
    beta, rho = 0.2, 1.0
    from paper_1709_09479_gb300 import inputs
    x = f32(inputs.powerlaw_field(50, N, J, dims)).astype(np.float64)
    d0 = f32(inputs.unit_filters(51, K, J, (s, s))).astype(np.float64)
    ref = O.csc_alternate(x, d0, beta, rho, n_outer=3, n_code=10, n_learn=4)
    solver = csc.Solver(J=J, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho, cg_tol=1e-6, cg_max=400)
    xv, dv = to_cuda(x), to_cuda(d0)
    v = torch.zeros((N, K) + dims, device="cuda")
    z = torch.empty_like(v)
    mu = torch.full((K,), 0.5, dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(3):
        solver.code(xv, dv, v, z, 10)
        f_code = solver.objective(xv, dv, z)
        solver.learn(xv, z, dv, mu, 4)
        hist.append((f_code, solver.objective(xv, dv, z)))
    solver.close()
    for (fc, fl), h in zip(hist, ref["history"]):
        assert abs(fc - h["f_code"]) <= 1e-4 * h["f_code"]
        assert abs(fl - h["f_learn"]) <= 1e-4 * h["f_learn"]
    assert rel(to_np(dv), ref["d"]) <= 3 * REL_TOL
    assert rel(to_np(z), ref["z"]) <= 3 * REL_TOL
