"""The allocation-free coding entry point (csc_code_noalloc) against the context entry point.

Callers that cannot allocate device memory where they code images (under a framework whose caching
allocator owns the device pool, plugins handed only a stream and device pointers, latency-bound
paths that cannot take cudaMalloc's implicit synchronisation) use csc_code_noalloc, whose workspace
is a fixed file-scope device array. At 128 x 128 it runs the generic sweep while csc_code runs the
dedicated 128 x 128 one, so that case also checks the two sweeps against each other. Here it must give what
csc_init + csc_code give, on two calls in a row (the second warm-started, reusing the scratch the
first one left behind), and refuse problems larger than its scratch. Collected last on purpose.
"""
import numpy as np
import pytest

from tests.gpu_common import REL_TOL, make_problem, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def test_noalloc_matches_context_call_on_two_calls_in_a_row(csc):
    import torch
    for (N, K, J, dims, s, beta, rho) in [(7, 50, 1, (64, 64), 5, 0.5, 1.0), (2, 3, 3, (24, 32), 3, 0.25, 1.5),
                                         (2, 8, 1, (128, 128), 11, 0.05, 1.0)]:
        x, d = make_problem(90 + K, N, K, J, dims, s)
        xv, dv = to_cuda(x), to_cuda(d)
        v_ref = torch.zeros((N, K) + dims, device="cuda")
        z_ref = torch.empty_like(v_ref)
        v_na = torch.zeros_like(v_ref)
        z_na = torch.full_like(v_ref, 7.0)
        with csc.Solver(J=J, K=K, fs=(s, s), dims=dims, n_images=N, beta=beta, rho=rho) as sv:
            for iters in (4, 3):                       # two calls in a row, the second warm-started
                sv.code(xv, dv, v_ref, z_ref, iters)
                csc.csc_code_noalloc(J, K, (s, s), dims, N, beta, rho, xv, dv, v_na, z_na, iters)
                torch.cuda.synchronize()
                assert rel(to_np(v_na), to_np(v_ref)) <= REL_TOL
                assert maxrel(to_np(v_na), to_np(v_ref)) <= REL_TOL
                if float(z_ref.abs().max()) > 0:
                    assert rel(to_np(z_na), to_np(z_ref)) <= REL_TOL
                else:
                    assert float(z_na.abs().max()) == 0.0


def test_noalloc_rejects_problems_beyond_its_scratch(csc):
    import torch
    N, K, dims = 400, 100, (128, 128)   # ~120 MB of workspace > 64 MiB
    x = torch.zeros((1,), device="cuda")
    with pytest.raises(csc.CscError) as e:
        csc.csc_code_noalloc(1, K, (11, 11), dims, N, 1.0, 10.0, x, x, x, None, 2)
    assert e.value.status == 2 and "64 MiB" in str(e.value)
