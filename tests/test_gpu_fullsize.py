"""Parity at the benchmark workload's full size (powerlaw128: N = 100 grey 1/f^2 fields 128 x 128,
K = 100 filters 11 x 11, beta = 1, rho = 0.1), in the launch configuration bench.py times.

Coding is separable per image (the dual ADMM of Eq. Inference_solution couples only the K maps of
one image), so the GPU run over all 100 images is checked element by element on sampled images
that the float64 oracle codes one by one.

Learning couples all images; at this size the oracle's dual route is too slow for a test, so the
GPU's learned filters are checked against a property that fixes them: after one learning step they
solve the filter-space normal equations (S Z^T Z S^T + 2 diag(mu)) d = S Z^T x of Eq. Learning_new
for the multipliers mu the step started from, with Z and Z^T applied by the oracle's own
(float64, FFT-based) operators.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

N, K, H, S = 100, 100, 128, 11
BETA, RHO, ITERS = 1.0, 0.1, 20


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


@pytest.fixture(scope="module")
def workload():
    from paper_1709_09479_gb300 import inputs
    x = f32(inputs.powerlaw_field(2, N, 1, (H, H))).astype(np.float64)
    d = f32(inputs.unit_filters(21, K, 1, (S, S))).astype(np.float64)
    return x, d


@pytest.fixture(scope="module")
def gpu_codes(csc, workload):
    import torch
    x, d = workload
    sv = csc.Solver(J=1, K=K, fs=(S, S), dims=(H, H), n_images=N, beta=BETA, rho=RHO)
    v = torch.zeros((N, K, H, H), device="cuda")
    z = torch.empty_like(v)
    sv.code(to_cuda(x), to_cuda(d), v, z, ITERS)
    torch.cuda.synchronize()
    sv.close()
    return to_np(v), to_np(z)


@pytest.mark.parametrize("n", [0, 41, 99])
def test_full_size_coding_sampled_images(workload, gpu_codes, n):
    x, d = workload
    v_g, z_g = gpu_codes
    v_o, z_o = O.code_admm(x[n:n + 1], d, BETA, RHO, ITERS)
    assert np.count_nonzero(z_o) > 0
    assert rel(v_g[n], v_o[0]) <= REL_TOL
    assert rel(z_g[n], z_o[0]) <= REL_TOL
    assert maxrel(v_g[n], v_o[0]) <= REL_TOL


def test_full_size_learning_solves_normal_equations(csc, workload, gpu_codes):
    import torch
    x, d = workload
    z = gpu_codes[1]
    mu0 = np.full(K, 0.5)
    sv = csc.Solver(J=1, K=K, fs=(S, S), dims=(H, H), n_images=N, beta=BETA, rho=RHO, cg_tol=1e-6, cg_max=400)
    dv = to_cuda(d)
    mu = torch.tensor(mu0, device="cuda")
    its = sv.learn(to_cuda(x), to_cuda(z), dv, mu, 1)
    sv.close()
    d_out, mu1 = to_np(dv), mu.cpu().numpy()
    assert 0 < its[0] <= 400
    # the step's solve, before the unit-norm projection: ||d_k|| = mu1_k / mu0_k (Eq. mu_update)
    z64 = z.astype(np.float64)
    active = np.array([np.any(z64[:, k] != 0) for k in range(K)])
    ok = active & (mu1 > 10 * O.MU_FLOOR)
    assert ok.sum() >= K // 2
    norms = mu1 / mu0
    d_pre = d_out.reshape(K, S, S) * np.maximum(1.0, norms)[:, None, None]
    ops = O.LearningOperators(z64)
    lhs = O.crop_support(ops.ZT(ops.Z(O.pad_support(d_pre, ops.dims))), (S, S)) + 2.0 * mu0[:, None, None] * d_pre
    rhs = O.crop_support(ops.ZT(x[:, 0]), (S, S))
    res = np.linalg.norm((lhs - rhs)[ok]) / np.linalg.norm(rhs[ok])
    print(f"full-size learning: CG iterations {its[0]}, normal-equation residual {res:.2e}")
    assert res <= 1e-4
    # the projection: every filter ends inside the unit ball
    assert np.all(np.sqrt((d_out.reshape(K, -1) ** 2).sum(1)) <= 1 + 1e-5)


# ---- uneven256 at full size: 256 images, H and W uniform in [64, 512] (seed 3), K = 64, 11 x 11,
# beta = 1, rho = 0.1, in bench.py's launch configuration (CSC_FLAG_GRAPH). Images are coded
# independently, so sampled images are checked element by element against the oracle.
@pytest.fixture(scope="module")
def uneven_workload():
    from paper_1709_09479_gb300 import inputs
    rng = np.random.default_rng(3)
    sizes = [(int(rng.integers(64, 513)), int(rng.integers(64, 513))) for _ in range(256)]
    xs = [f32(inputs.powerlaw_field(1000 + i, 1, 1, hw)) for i, hw in enumerate(sizes)]
    d = f32(inputs.unit_filters(30, 64, 1, (S, S)))
    return sizes, xs, d


def _sampled(sizes):
    px = [h * w for h, w in sizes]
    primes = [i for i, (h, w) in enumerate(sizes) if all(h % p for p in range(2, h)) and h > 7]
    return sorted({int(np.argmin(px)), int(np.argmax(px)), primes[0] if primes else 1})


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_full_size_uneven256_sampled_images(csc, uneven_workload, precision):
    import torch
    from tests.test_gpu_precision import CODE_BF16_TOL
    sizes, xs, d = uneven_workload
    Ku, iters = 64, 5
    prec = csc.CSC_FP32 if precision == "fp32" else csc.CSC_MIXED_BF16
    x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in xs])).cuda()
    dd = torch.from_numpy(d.reshape(-1).copy()).cuda()
    npx = sum(h * w for h, w in sizes)
    v = torch.zeros(Ku * npx, device="cuda")
    z = torch.empty_like(v)
    with csc.Solver(J=1, K=Ku, fs=(S, S), dims_list=sizes, beta=BETA, rho=RHO, precision=prec,
                    flags=csc.CSC_FLAG_GRAPH) as sv:
        sv.code(x, dd, v, z, iters)
        torch.cuda.synchronize()
    offs = np.cumsum([0] + [Ku * h * w for h, w in sizes])
    tol = REL_TOL if precision == "fp32" else CODE_BF16_TOL
    for n in _sampled(sizes):
        h, w = sizes[n]
        vg = v[offs[n]:offs[n + 1]].cpu().numpy().astype(np.float64).reshape(1, Ku, h, w)
        zg = z[offs[n]:offs[n + 1]].cpu().numpy().astype(np.float64).reshape(1, Ku, h, w)
        vo, zo = O.code_admm(xs[n].astype(np.float64), d.astype(np.float64), BETA, RHO, iters)
        assert rel(vg, vo) <= tol, (n, sizes[n], rel(vg, vo))
        if np.any(zo != 0):
            assert rel(zg, zo) <= tol, (n, sizes[n], rel(zg, zo))
        if precision == "fp32":
            assert maxrel(vg, vo) <= REL_TOL
