"""The mixed-precision modes (CSC_MIXED_BF16, and CSC_MIXED_TF32 at the end of the file): per-frequency contractions with bfloat16 operands and
float32 accumulation — the coding sweep's sum_k d_hat_k u_hat_k and conj(d_hat_k) lambda_hat on the
CUDA cores, and the learning step's code Gram Z(w)^H Z(w) on the tensor cores (tcgen05) — against
the float64 oracle. bfloat16 keeps 8 significant bits (unit roundoff 2^-9 ~ 2e-3), so the errors
are stated, measured bounds rather than the float32 bar; a layout or sign error in the tensor-core
Gram would show as an O(1) error in the learned filters."""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import f32, make_problem, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

#: measured on GB300 and printed by the tests; bounds leave a factor of ~3
CODE_BF16_TOL = 1e-2
LEARN_BF16_TOL = 3e-2


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


@pytest.mark.parametrize("case", [(3, 5, (100, 100), 11, 1.0, 0.1, 10), (4, 40, (64, 64), 5, 0.3, 1.0, 8),
                                  (2, 24, (128, 128), 11, 0.3, 1.0, 8)])
def test_bf16_coding_error_against_oracle(csc, case):
    """bf16 contraction operands in the generic sweep (100 x 100, 64 x 64) and the fused 128 x 128 one."""
    import torch
    N, K, dims, s, beta, rho, iters = case
    x, d = make_problem(110 + K, N, K, 1, dims, s)
    _, zo = O.code_admm(x, d, beta, rho, iters)
    out = {}
    for prec in (csc.CSC_FP32, csc.CSC_MIXED_BF16):
        with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho, precision=prec) as sv:
            v = torch.zeros((N, K) + dims, device="cuda")
            z = torch.empty_like(v)
            sv.code(to_cuda(x), to_cuda(d), v, z, iters)
            torch.cuda.synchronize()
            out[prec] = to_np(z)
    e32, e16 = rel(out[csc.CSC_FP32], zo), rel(out[csc.CSC_MIXED_BF16], zo)
    print(f"coding rel err vs oracle: fp32 {e32:.2e}  bf16 {e16:.2e}")
    assert e32 <= 1e-4
    assert e16 <= CODE_BF16_TOL


@pytest.mark.parametrize("case", [(3, 6, (64, 64), 5, 0.3), (16, 100, (64, 64), 5, 0.3), (4, 8, (100, 100), 11, 0.5),
                                  (45, 20, (32, 32), 5, 0.3)])
def test_tensor_core_gram_learning_against_oracle(csc, case):
    import torch
    N, K, dims, s, beta = case
    x, d = make_problem(120 + K, N, K, 1, dims, s)
    _, z = O.code_admm(x, d, beta, 1.0, 30)
    z = f32(z).astype(np.float64)
    mu0 = np.full(K, 0.5)
    do, muo, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), 2)
    res = {}
    for prec in (csc.CSC_FP32, csc.CSC_MIXED_BF16):
        with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=1.0, precision=prec,
                        cg_tol=1e-6, cg_max=400) as sv:
            dv = to_cuda(d)
            mu = torch.tensor(mu0, device="cuda")
            sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
            torch.cuda.synchronize()
            res[prec] = (to_np(dv), mu.cpu().numpy())
    e32 = rel(res[csc.CSC_FP32][0], do)
    e16 = rel(res[csc.CSC_MIXED_BF16][0], do)
    m16 = float(np.max(np.abs(res[csc.CSC_MIXED_BF16][1] - muo) / muo))
    print(f"learned filters rel err vs oracle: fp32 {e32:.2e}  bf16 tensor-core Gram {e16:.2e}  (mu {m16:.2e})")
    assert e32 <= 1e-4
    assert e16 <= LEARN_BF16_TOL
    assert m16 <= LEARN_BF16_TOL


def test_objective_stays_float32_in_mixed_mode(csc):
    N, K, dims, s = 3, 5, (100, 100), 11
    x, d = make_problem(130, N, K, 1, dims, s)
    rng = np.random.default_rng(9)
    z = f32(np.where(rng.random((N, K) + dims) < 0.05, rng.standard_normal((N, K) + dims), 0.0)).astype(np.float64)
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=0.7, rho=1.0,
                    precision=csc.CSC_MIXED_BF16) as sv:
        f = sv.objective(to_cuda(x), to_cuda(d), to_cuda(z))
    fo = O.objective(x, d, z, 0.7)
    assert abs(f - fo) <= 1e-5 * fo


#: CSC_MIXED_TF32 (10 explicit mantissa bits, unit roundoff 2^-11 ~ 4.9e-4): measured on GB300 and
#: printed by the tests; bounds leave a factor of ~3
CODE_TF32_TOL = 3e-3
LEARN_TF32_TOL = 2e-3


@pytest.mark.parametrize("case", [(3, 5, (100, 100), 11, 1.0, 0.1, 10), (4, 40, (64, 64), 5, 0.3, 1.0, 8),
                                  (2, 24, (128, 128), 11, 0.3, 1.0, 8)])
def test_tf32_coding_error_against_oracle(csc, case):
    """TF32 contraction operands in the generic sweep (100 x 100, 64 x 64) and the fused 128 x 128 one."""
    import torch
    N, K, dims, s, beta, rho, iters = case
    x, d = make_problem(140 + K, N, K, 1, dims, s)
    _, zo = O.code_admm(x, d, beta, rho, iters)
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho,
                    precision=csc.CSC_MIXED_TF32) as sv:
        v = torch.zeros((N, K) + dims, device="cuda")
        z = torch.empty_like(v)
        sv.code(to_cuda(x), to_cuda(d), v, z, iters)
        torch.cuda.synchronize()
    e = rel(to_np(z), zo)
    print(f"coding rel err vs oracle: tf32 {e:.2e}")
    assert np.abs(zo).max() > 0
    assert e <= CODE_TF32_TOL


@pytest.mark.parametrize("case", [(3, 6, (64, 64), 5, 0.3), (16, 100, (64, 64), 5, 0.3)])
def test_tf32_tensor_core_gram_learning_against_oracle(csc, case):
    import torch
    N, K, dims, s, beta = case
    x, d = make_problem(150 + K, N, K, 1, dims, s)
    _, z = O.code_admm(x, d, beta, 1.0, 30)
    z = f32(z).astype(np.float64)
    mu0 = np.full(K, 0.5)
    do, muo, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), 2)
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=1.0,
                    precision=csc.CSC_MIXED_TF32, cg_tol=1e-6, cg_max=400) as sv:
        dv = to_cuda(d)
        mu = torch.tensor(mu0, device="cuda")
        sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
        torch.cuda.synchronize()
    e = rel(to_np(dv), do)
    m = float(np.max(np.abs(mu.cpu().numpy() - muo) / muo))
    print(f"learned filters rel err vs oracle: tf32 tensor-core Gram {e:.2e} (mu {m:.2e})")
    assert e <= LEARN_TF32_TOL
    assert m <= LEARN_TF32_TOL
