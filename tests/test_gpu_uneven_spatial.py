"""GPU parity of the direct spatial route on uneven batches (CSC_FLAG_SPATIAL on csc_init_uneven):
the coding iteration of Eq. Inference_solution with D and D^T taken as circular convolutions on each
image's own H x W grid (CUDA cores, filters zero-padded to 11 x 11 about their centre) and only the
one-channel solve for lambda in the Fourier domain (the multi-pass engine's transforms, Bluestein for
sides with large prime factors). By the convolution theorem it is the iteration of the Fourier route,
so it is checked element by element against the float64 oracle run image by image at the float32 bar,
and against the Fourier route on the same batch.

Cases: odd, prime and rectangular sides (ragged output tiles of 32 x 64, images smaller than one
tile), filter supports from 1 x 1 to 11 x 11 including rectangular ones, warm starts and split calls
(bitwise), the objective on such a context, refused shapes, and sampled images of the full 256-image
batch (sides uniform in [64, 512], K = 64, 11 x 11)."""
import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, maxrel, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def batch(seed, sizes, K, fs):
    from paper_1709_09479_gb300 import inputs
    xs = [f32(inputs.powerlaw_field(seed + i, 1, 1, hw)).astype(np.float64) for i, hw in enumerate(sizes)]
    d = f32(inputs.unit_filters(seed + 99, K, 1, tuple(fs))).astype(np.float64)
    return xs, d


def flat(arrs):
    import torch
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrs]).astype(np.float32)).cuda()


def split(t, sizes, per):
    out, off = [], 0
    a = t.detach().cpu().numpy().astype(np.float64)
    for (H, W) in sizes:
        n = per * H * W
        out.append(a[off:off + n].reshape((1, per, H, W)))
        off += n
    return out


def code(csc, xs, d, sizes, beta, rho, iters, flags, v0=None):
    import torch
    K = d.shape[0]
    n_v = sum(K * H * W for H, W in sizes)
    with csc.Solver(J=1, K=K, fs=d.shape[2:], dims_list=sizes, beta=beta, rho=rho, flags=flags) as sv:
        v = torch.zeros(n_v, device="cuda") if v0 is None else v0.clone()
        z = torch.empty_like(v)
        sv.code(flat(xs), flat([d]), v, z, iters)
        torch.cuda.synchronize()
    return v, z


SIZES = [(67, 131), (64, 64), (37, 53), (100, 100), (24, 32), (129, 70), (8, 9), (97, 33)]
CASES = [
    # (K, (fh, fw), beta, rho, iters)
    (12, (11, 11), 0.3, 1.0, 5),
    (5, (5, 5), 0.5, 2.0, 4),
    (7, (3, 7), 0.2, 1.0, 3),    # rectangular support
    (3, (1, 1), 0.1, 1.0, 3),    # one tap
    (33, (9, 11), 0.4, 3.0, 3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"K{c[0]}_{c[1][0]}x{c[1][1]}")
def test_uneven_spatial_matches_oracle_per_image(csc, case):
    K, fs, beta, rho, iters = case
    sizes = SIZES if fs[0] <= 7 else [hw for hw in SIZES if min(hw) >= 11]
    xs, d = batch(300 + K, sizes, K, fs)
    v, z = code(csc, xs, d, sizes, beta, rho, iters, csc.CSC_FLAG_SPATIAL)
    vs, zs = split(v, sizes, K), split(z, sizes, K)
    for i, x in enumerate(xs):
        vo, zo = O.code_admm(x, d, beta, rho, iters)
        assert rel(vs[i], vo) <= REL_TOL, (sizes[i], rel(vs[i], vo))
        assert maxrel(vs[i], vo) <= REL_TOL, (sizes[i], maxrel(vs[i], vo))
        if np.any(zo != 0):
            assert rel(zs[i], zo) <= REL_TOL, (sizes[i], rel(zs[i], zo))


def test_uneven_spatial_equals_fourier_route(csc):
    """Both routes compute the iteration of Eq. Inference_solution in float32 on the same batch."""
    sizes = [(67, 131), (100, 100), (129, 70), (97, 33), (200, 150)]
    K, fs, beta, rho, iters = 16, (11, 11), 1.0, 0.1, 8
    xs, d = batch(17, sizes, K, fs)
    vs, zs = code(csc, xs, d, sizes, beta, rho, iters, csc.CSC_FLAG_SPATIAL)
    vf, zf = code(csc, xs, d, sizes, beta, rho, iters, 0)
    a, b = vs.cpu().numpy().astype(np.float64), vf.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - b) <= 2e-5 * np.linalg.norm(b)
    a, b = zs.cpu().numpy().astype(np.float64), zf.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - b) <= 2e-5 * np.linalg.norm(b)


def test_uneven_spatial_split_calls_repeats_and_objective(csc):
    """Every sum runs in a fixed order: a repeated call gives the same bits, and 3 + 4 warm-started
    iterations the bits of 7. The objective of such a context (the Fourier engine's) matches the
    oracle's objective of the codes."""
    sizes = [(67, 131), (64, 64), (37, 53)]
    K, fs, beta, rho = 6, (11, 11), 0.3, 1.0
    xs, d = batch(5, sizes, K, fs)
    flags = csc.CSC_FLAG_SPATIAL
    v7, z7 = code(csc, xs, d, sizes, beta, rho, 7, flags)
    v7b, z7b = code(csc, xs, d, sizes, beta, rho, 7, flags)
    assert bool((v7 == v7b).all()) and bool((z7 == z7b).all())
    v3, _ = code(csc, xs, d, sizes, beta, rho, 3, flags)
    v34, z34 = code(csc, xs, d, sizes, beta, rho, 4, flags, v0=v3)
    assert bool((v34 == v7).all()) and bool((z34 == z7).all())
    zs = split(z7, sizes, K)
    want = sum(O.objective(xs[i], d, zs[i], beta) for i in range(len(sizes)))
    with csc.Solver(J=1, K=K, fs=fs, dims_list=sizes, beta=beta, rho=rho, flags=flags) as sv:
        got = sv.objective(flat(xs), flat([d]), z7)
    assert abs(got - want) <= 1e-5 * abs(want), (got, want)


@pytest.mark.parametrize("kw", [
    dict(J=3, K=4, fs=(3, 3)),                       # colour
    dict(J=1, K=4, fs=(13, 13)),                     # support above 11 x 11
    dict(J=1, K=4, fs=(5, 5), precision=1),          # CSC_MIXED_BF16
    dict(J=1, K=1000, fs=(5, 5)),                    # filters beyond shared memory
])
def test_uneven_spatial_unsupported_shapes_are_refused(csc, kw):
    with pytest.raises(csc.CscError) as e:
        csc.Solver(dims_list=[(64, 64), (40, 48)], beta=1.0, rho=1.0, flags=csc.CSC_FLAG_SPATIAL, **kw)
    assert e.value.status == 8


def test_uneven_spatial_full_batch_sampled_images(csc):
    """The 256-image batch (H and W uniform in [64, 512], K = 64, 11 x 11, beta = 1, rho = 0.1) in the
    launch configuration the benchmark times; coding is separable per image, so sampled images are
    checked element by element against the oracle after 3 iterations."""
    import torch
    from paper_1709_09479_gb300 import inputs
    rng = np.random.default_rng(3)
    sizes = [(int(rng.integers(64, 513)), int(rng.integers(64, 513))) for _ in range(256)]
    K, S, beta, rho, iters = 64, 11, 1.0, 0.1, 3
    xs = [f32(inputs.powerlaw_field(1000 + i, 1, 1, hw)).astype(np.float64) for i, hw in enumerate(sizes)]
    d = f32(inputs.unit_filters(30, K, 1, (S, S))).astype(np.float64)
    v, z = code(csc, xs, d, sizes, beta, rho, iters, csc.CSC_FLAG_SPATIAL)
    offs = np.cumsum([0] + [K * H * W for H, W in sizes])
    for i in (0, 131, 255):
        H, W = sizes[i]
        vi = v[offs[i]:offs[i + 1]].cpu().numpy().astype(np.float64).reshape(1, K, H, W)
        zi = z[offs[i]:offs[i + 1]].cpu().numpy().astype(np.float64).reshape(1, K, H, W)
        vo, zo = O.code_admm(xs[i], d, beta, rho, iters)
        assert rel(vi, vo) <= REL_TOL, (sizes[i], rel(vi, vo))
        assert maxrel(vi, vo) <= REL_TOL
        if np.any(zo != 0):
            assert rel(zi, zo) <= REL_TOL
    del torch


def test_uneven_spatial_graph_replay_equals_eager(csc):
    """With CSC_FLAG_GRAPH the launches of a call are recorded once and replayed: the replayed calls
    give the eager call's bits."""
    sizes = [(67, 131), (100, 100), (37, 53)]
    K, fs, beta, rho, iters = 8, (11, 11), 0.5, 1.0, 4
    xs, d = batch(23, sizes, K, fs)
    ve, ze = code(csc, xs, d, sizes, beta, rho, iters, csc.CSC_FLAG_SPATIAL)
    import torch
    n_v = sum(K * H * W for H, W in sizes)
    with csc.Solver(J=1, K=K, fs=fs, dims_list=sizes, beta=beta, rho=rho,
                    flags=csc.CSC_FLAG_SPATIAL | csc.CSC_FLAG_GRAPH) as sv:
        for _ in range(3):
            v = torch.zeros(n_v, device="cuda")
            z = torch.empty_like(v)
            sv.code(flat(xs), flat([d]), v, z, iters)
            torch.cuda.synchronize()
            assert bool((v == ve).all()) and bool((z == ze).all())
