"""Failure detection through the C ABI, with no GPU fault: non-finite inputs, a CG exchange wait that
runs out on purpose, and a CG that stops at its iteration cap.

* a NaN or Inf anywhere in x, d or v reaches the dual variable lambda_hat within one ADMM iteration
  (Eq. Inference_solution sums every map of an image into it); the sweeps raise a device flag there,
  which a synchronous csc_code (host arrays, or CSC_FLAG_CHECK_FINITE) returns as CSC_ERR_NONFINITE and
  csc_check reports for an asynchronous one;
* the learning CG checks its residual and step scalars (the same totals in every CTA) and stops with
  CSC_ERR_NONFINITE;
* csc_set_wait_limit bounds the CG's grid-exchange waits to a few SM clocks, so a wait gives up, every
  CTA returns and csc_learn returns CSC_ERR_TIMEOUT; the same context then learns normally and matches
  the oracle (the context stays usable);
* cg_max = 1 with CSC_FLAG_CG_STRICT returns CSC_ERR_NOT_CONVERGED, and without the flag reports one
  CG iteration per step.
After every failure the test makes a normal call on the same context and checks it against the oracle.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, make_problem, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def code_ref(x, d, beta, rho, iters):
    v, z = O.code_admm(x, d, beta, rho, iters)
    return v, z


@pytest.mark.parametrize("dims,s", [((128, 128), 11), ((48, 40), 5)])
def test_nan_image_is_reported_and_context_stays_usable(csc, dims, s):
    import torch
    N, K, beta, rho, iters = 2, 6, 0.2, 1.0, 4
    x, d = make_problem(300, N, K, 1, dims, s)
    bad = x.copy()
    bad[1, 0, 5, 7] = np.nan
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho,
                    flags=csc.CSC_FLAG_CHECK_FINITE) as sv:
        v = torch.zeros((N, K) + dims, device="cuda")
        with pytest.raises(csc.CscError) as e:
            sv.code(to_cuda(bad), to_cuda(d), v, None, iters)
        assert e.value.status == 5
        # the same context on clean inputs
        v.zero_()
        z = torch.empty_like(v)
        sv.code(to_cuda(x), to_cuda(d), v, z, iters)
        _, zr = code_ref(x, d, beta, rho, iters)
        assert rel(to_np(z), zr) <= REL_TOL


def test_nan_state_on_host_arrays_and_csc_check(csc):
    import torch
    N, K, dims, s, beta, rho, iters = 2, 5, (64, 64), 5, 0.2, 1.0, 3
    x, d = make_problem(301, N, K, 1, dims, s)
    with csc.Solver(J=1, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho) as sv:
        # host arrays: the call is synchronous and reports the flag itself
        v = np.zeros((N, K) + dims, dtype=np.float32)
        v[0, 3, 10, 10] = np.inf
        with pytest.raises(csc.CscError) as e:
            sv.code(f32(x), f32(d), v, None, iters)
        assert e.value.status == 5
        # device arrays without the flag: asynchronous, reported by csc_check
        vd = torch.zeros((N, K) + dims, device="cuda")
        vd[1, 0, 3, 3] = float("nan")
        sv.code(to_cuda(x), to_cuda(d), vd, None, iters)
        with pytest.raises(csc.CscError) as e:
            sv.check()
        assert e.value.status == 5
        # a clean call clears the flag
        vd.zero_()
        z = torch.empty_like(vd)
        sv.code(to_cuda(x), to_cuda(d), vd, z, iters)
        sv.check()
        _, zr = code_ref(x, d, beta, rho, iters)
        assert rel(to_np(z), zr) <= REL_TOL


def learn_case():
    N, K, dims, s = 3, 6, (64, 64), 5
    x, d = make_problem(302, N, K, 1, dims, s)
    _, z = O.code_admm(x, d, 0.3, 1.0, 10)
    z = f32(z).astype(np.float64)
    return x, z, d


def test_nan_codes_stop_the_cg_with_nonfinite(csc):
    import torch
    x, z, d = learn_case()
    K = d.shape[0]
    zb = z.copy()
    zb[0, 2, 4, 4] = np.nan
    with csc.Solver(J=1, K=K, fs=d.shape[2:], dims=x.shape[2:], n_images=x.shape[0], beta=1.0, rho=1.0,
                    cg_max=200, cg_tol=1e-6) as sv:
        dv = to_cuda(d)
        mu = torch.full((K,), 0.5, dtype=torch.float64, device="cuda")
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(zb), dv, mu, 2)
        assert e.value.status == 5


def test_cg_wait_limit_times_out_then_context_learns_normally(csc):
    import torch
    x, z, d = learn_case()
    K = d.shape[0]
    mu0 = np.full(K, 0.5)
    d_ref, mu_ref, _, _ = O.learn_paper(x, z, d, mu0, np.zeros_like(x), 2)
    with csc.Solver(J=1, K=K, fs=d.shape[2:], dims=x.shape[2:], n_images=x.shape[0], beta=1.0, rho=1.0,
                    cg_max=400, cg_tol=1e-6) as sv:
        sv.set_wait_limit(1)          # one SM clock: the first exchange that is not complete gives up
        dv = to_cuda(d)
        mu = torch.tensor(mu0, device="cuda")
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
        assert e.value.status == 7
        sv.set_wait_limit(0)          # the default bound again; same context
        dv = to_cuda(d)
        mu = torch.tensor(mu0, device="cuda")
        sv.learn(to_cuda(x), to_cuda(z), dv, mu, 2)
        assert rel(to_np(dv), d_ref) <= REL_TOL
        np.testing.assert_allclose(mu.cpu().numpy(), mu_ref, rtol=REL_TOL)


def test_cg_stopped_at_its_cap(csc):
    import torch
    x, z, d = learn_case()
    K = d.shape[0]
    args = dict(J=1, K=K, fs=d.shape[2:], dims=x.shape[2:], n_images=x.shape[0], beta=1.0, rho=1.0,
                cg_max=1, cg_tol=1e-9)
    with csc.Solver(**args) as sv:
        its = sv.learn(to_cuda(x), to_cuda(z), to_cuda(d), torch.full((K,), 0.5, dtype=torch.float64,
                                                                        device="cuda"), 3)
        assert its == [1, 1, 1]
    with csc.Solver(flags=csc.CSC_FLAG_CG_STRICT, **args) as sv:
        with pytest.raises(csc.CscError) as e:
            sv.learn(to_cuda(x), to_cuda(z), to_cuda(d), torch.full((K,), 0.5, dtype=torch.float64,
                                                                      device="cuda"), 3)
        assert e.value.status == 6
