"""GPU parity of the direct spatial route (CSC_FLAG_SPATIAL): the coding iteration of
Eq. Inference_solution with D and D^T applied as convolutions on the pixel grid by the tensor cores
(tcgen05, float32 operands as two TF32 parts, three products per pair) and only the one-channel solve
for lambda in the Fourier domain. It is the same iteration as the Fourier-domain sweep (convolution
theorem), so it is checked element by element against the float64 oracle at the float32 bar, and
against the Fourier route on the same context shape.

Cases cover filter counts and tap counts that are not multiples of the 16-element operand chunks,
rectangular supports, a 1 x 1 filter, CTAs whose rows span several images (so the convolution's
halo rows cross image boundaries), warm starts, determinism, the TF32 mode's stated bound, the full
benchmark size on sampled images, unsupported shapes, and a wait that gives up.
"""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, maxrel, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

H = 128
CASES = [
    # (N, K, (fh, fw), beta, rho, iters)
    (2, 12, (11, 11), 0.5, 1.0, 6),     # 121 taps -> 128, K = 12 -> 16
    (1, 16, (5, 5), 0.3, 2.0, 8),       # 25 taps -> 32
    (3, 100, (11, 11), 1.0, 10.0, 3),   # the benchmark's K; 384 rows over the SMs: segments cross images
    (2, 7, (7, 3), 0.2, 1.0, 5),        # rectangular support
    (1, 1, (1, 1), 0.1, 1.0, 4),        # one filter, one tap
    (5, 33, (9, 9), 0.4, 3.0, 4),       # 81 taps -> 96, K = 33 -> 48
    (1, 128, (11, 11), 0.5, 1.0, 3),    # K = 128: the largest filter operand, two A stages
]


def make_problem(seed, N, K, fs):
    """Seeded 1/f^2 fields (float32-representable) and unit-norm fh x fw filters, as float64."""
    from paper_1709_09479_gb300 import inputs
    x = inputs.powerlaw_field(seed, N, 1, (H, H))
    d = inputs.unit_filters(seed + 100, K, 1, tuple(fs))
    return f32(x).astype(np.float64), f32(d).astype(np.float64)


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def code(csc, x, d, beta, rho, iters, v0=None, flags=None, precision=None):
    import torch
    N, K = x.shape[0], d.shape[0]
    kw = {} if precision is None else {"precision": precision}
    sv = csc.Solver(J=1, K=K, fs=d.shape[2:], dims=(H, H), n_images=N, beta=beta, rho=rho,
                    flags=csc.CSC_FLAG_SPATIAL if flags is None else flags, **kw)
    v = torch.zeros((N, K, H, H), device="cuda") if v0 is None else to_cuda(v0)
    z = torch.empty_like(v)
    sv.code(to_cuda(x), to_cuda(d), v, z, iters)
    torch.cuda.synchronize()
    sv.close()
    return to_np(v), to_np(z)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}K{c[1]}_{c[2][0]}x{c[2][1]}")
def test_spatial_coding_matches_oracle(csc, case):
    N, K, fs, beta, rho, iters = case
    x, d = make_problem(31 + K, N, K, fs)
    v, z = code(csc, x, d, beta, rho, iters)
    vo, zo = O.code_admm(x, d, beta, rho, iters)
    assert rel(v, vo) <= REL_TOL, rel(v, vo)
    assert maxrel(v, vo) <= REL_TOL, maxrel(v, vo)
    if np.any(zo != 0):
        assert rel(z, zo) <= REL_TOL, rel(z, zo)
        assert maxrel(z, zo) <= REL_TOL


def test_spatial_route_equals_fourier_route(csc):
    """Both routes compute the iteration of Eq. Inference_solution in float32."""
    N, K, fs, beta, rho, iters = 4, 100, (11, 11), 1.0, 0.1, 8
    x, d = make_problem(7, N, K, fs)
    vs, zs = code(csc, x, d, beta, rho, iters)
    vf, zf = code(csc, x, d, beta, rho, iters, flags=0)
    assert rel(vs, vf) <= 2e-5, rel(vs, vf)
    assert rel(zs, zf) <= 2e-5, rel(zs, zf)


def test_spatial_split_calls_and_repeats_are_bitwise(csc):
    """Every sum runs in a fixed order (no atomics on data): a call repeated gives the same bits, and
    3 + 4 warm-started iterations give the bits of 7 (the state is the whole ADMM state)."""
    N, K, fs, beta, rho = 2, 20, (11, 11), 0.3, 1.0
    x, d = make_problem(5, N, K, fs)
    v7, z7 = code(csc, x, d, beta, rho, 7)
    v7b, z7b = code(csc, x, d, beta, rho, 7)
    np.testing.assert_array_equal(v7, v7b)
    np.testing.assert_array_equal(z7, z7b)
    v3, _ = code(csc, x, d, beta, rho, 3)
    v34, z34 = code(csc, x, d, beta, rho, 4, v0=v3)
    np.testing.assert_array_equal(v34, v7)
    np.testing.assert_array_equal(z34, z7)


def test_spatial_tf32_mode_within_its_bound(csc):
    """CSC_MIXED_TF32 takes one TF32 product per operand pair (10 explicit mantissa bits): the
    measured error against the float64 oracle after 10 iterations is stated here as its bound."""
    N, K, fs, beta, rho, iters = 2, 40, (11, 11), 1.0, 1.0, 10
    x, d = make_problem(9, N, K, fs)
    v, z = code(csc, x, d, beta, rho, iters, precision=csc.CSC_MIXED_TF32)
    vo, zo = O.code_admm(x, d, beta, rho, iters)
    assert rel(v, vo) <= 1e-2, rel(v, vo)
    assert rel(z, zo) <= 3e-2, rel(z, zo)


def test_spatial_full_size_sampled_images(csc):
    """powerlaw128 at full size (N = 100, K = 100, 11 x 11, beta = 1, rho = 0.1, 20 iterations), the
    launch configuration the benchmark times; coding is separable per image, so sampled images are
    checked element by element against the oracle."""
    from paper_1709_09479_gb300 import inputs
    N, K, S, beta, rho, iters = 100, 100, 11, 1.0, 0.1, 20
    x = f32(inputs.powerlaw_field(2, N, 1, (H, H))).astype(np.float64)
    d = f32(inputs.unit_filters(21, K, 1, (S, S))).astype(np.float64)
    v, z = code(csc, x, d, beta, rho, iters)
    for n in (0, 57, 99):
        vo, zo = O.code_admm(x[n:n + 1], d, beta, rho, iters)
        assert np.count_nonzero(zo) > 0
        assert rel(v[n], vo[0]) <= REL_TOL
        assert maxrel(v[n], vo[0]) <= REL_TOL
        assert rel(z[n], zo[0]) <= REL_TOL


@pytest.mark.parametrize("kw", [
    dict(J=3, K=4, fs=(5, 5), dims=(32, 32)),          # colour images (128 x 128 colour exceeds csc_init)
    dict(J=1, K=4, fs=(5, 5), dims=(64, 64)),          # another size
    dict(J=1, K=130, fs=(5, 5), dims=(H, H)),          # K above one MMA tile
    dict(J=1, K=4, fs=(13, 13), dims=(H, H)),          # 169 taps
    dict(J=1, K=4, fs=(5, 5), dims=(H, H), precision=1),   # CSC_MIXED_BF16
])
def test_spatial_unsupported_shapes_are_refused(csc, kw):
    with pytest.raises(csc.CscError) as e:
        csc.Solver(n_images=1, beta=1.0, rho=1.0, flags=csc.CSC_FLAG_SPATIAL, **kw)
    assert e.value.status == 8


def test_spatial_wait_limit_times_out_then_codes_normally(csc):
    """A wait limit of one SM clock makes the tensor-core kernels' first pending mbarrier wait give up:
    the CTA stops issuing work, drains its MMAs under the default bound, frees its TMEM, and the
    synchronous call returns CSC_ERR_TIMEOUT. The same context then codes normally."""
    N, K, fs, beta, rho, iters = 2, 24, (11, 11), 0.5, 1.0, 4
    x, d = make_problem(3, N, K, fs)
    vo, zo = O.code_admm(x, d, beta, rho, iters)
    with csc.Solver(J=1, K=K, fs=fs, dims=(H, H), n_images=N, beta=beta, rho=rho,
                    flags=csc.CSC_FLAG_SPATIAL) as sv:
        sv.set_wait_limit(1)
        v = np.zeros((N, K, H, H), np.float32)
        z = np.zeros_like(v)
        with pytest.raises(csc.CscError) as e:
            sv.code(f32(x), f32(d), v, z, iters)   # host arrays: the call synchronises and checks
        assert e.value.status == 7
        sv.set_wait_limit(0)
        v = np.zeros((N, K, H, H), np.float32)
        sv.code(f32(x), f32(d), v, z, iters)
        assert rel(v, vo) <= REL_TOL
        assert rel(z, zo) <= REL_TOL


def test_spatial_needs_an_aligned_state(csc):
    """The state's rows are moved by TMA bulk copies (16-byte aligned addresses): a v that starts 4
    bytes into an allocation is refused before any launch."""
    import torch
    N, K, fs = 1, 4, (5, 5)
    x, d = make_problem(1, N, K, fs)
    with csc.Solver(J=1, K=K, fs=fs, dims=(H, H), n_images=N, beta=0.5, rho=1.0,
                    flags=csc.CSC_FLAG_SPATIAL) as sv:
        buf = torch.zeros(N * K * H * H + 1, device="cuda")
        v = buf[1:].view(N, K, H, H)
        with pytest.raises(csc.CscError) as e:
            sv.code(to_cuda(x), to_cuda(d), v, None, 2)
        assert e.value.status == 1
