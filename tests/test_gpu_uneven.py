"""GPU parity of batched coding over images of different sizes (one persistent launch per ADMM
iteration, per-size FFT plans, cost-balanced CTA ranges, autotuned launch shape), of the CUDA-graph
replay of csc_code, and of the uneven objective, against the float64 oracle run image by image."""
import json

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


def batch(seed, sizes, K, J, s):
    from paper_1709_09479_gb300 import inputs
    xs = [f32(inputs.powerlaw_field(seed + i, 1, J, hw)).astype(np.float64) for i, hw in enumerate(sizes)]
    d = f32(inputs.unit_filters(seed + 99, K, J, (s, s))).astype(np.float64)
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


SIZES = [(64, 64), (48, 40), (100, 100), (24, 32), (64, 64), (128, 128), (40, 48), (96, 70)]


@pytest.mark.parametrize("J,K,s,iters", [(1, 5, 5, 5), (1, 40, 3, 3), (3, 4, 3, 4)])
def test_uneven_coding_matches_oracle_per_image(csc, J, K, s, iters):
    import torch
    # three channels need 3x the spectrum space per CTA: sizes up to 64 x 64 fit
    sizes = SIZES if J == 1 else [(64, 64), (48, 40), (24, 32), (40, 48)]
    beta, rho = 0.3, 1.0
    xs, d = batch(200 + K, sizes, K, J, s)
    n_v = sum(K * H * W for H, W in sizes)
    with csc.Solver(J=J, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho) as sv:
        v = torch.zeros(n_v, device="cuda")
        z = torch.empty_like(v)
        sv.code(flat(xs), flat([d]), v, z, iters)
        torch.cuda.synchronize()
        info = json.loads(sv.describe())
    assert info["uneven"] and info["autotuned"] and info["size_classes"] == len(set(sizes))
    for xo, vg, zg in zip(xs, split(v, sizes, K), split(z, sizes, K)):
        vo, zo = O.code_admm(xo, d, beta, rho, iters)
        assert rel(vg, vo) <= REL_TOL and maxrel(vg, vo) <= REL_TOL
        if np.any(zo != 0):
            assert rel(zg, zo) <= REL_TOL


def test_uneven_equals_uniform_and_graph_replay(csc):
    """A batch of equal sizes through the uneven path gives the uniform path's state; repeated
    calls under CSC_FLAG_GRAPH (graph replay) give the eager calls' state."""
    import torch
    N, K, s, beta, rho = 4, 6, 5, 0.3, 1.0
    dims = (64, 64)
    xs, d = batch(300, [dims] * N, K, 1, s)
    x, dv = flat(xs), flat([d])
    states = {}
    for mode in ("uniform", "uneven", "graph"):
        flags = csc.CSC_FLAG_GRAPH if mode == "graph" else 0
        kw = dict(dims=dims, n_images=N) if mode != "uneven" else dict(dims_list=[dims] * N)
        with csc.Solver(J=1, K=K, fs=(s, s), beta=beta, rho=rho, flags=flags, **kw) as sv:
            v = torch.zeros(N * K * 64 * 64, device="cuda")
            z = torch.empty_like(v)
            for _ in range(3):          # the graph is recorded on the first call, replayed after
                sv.code(x, dv, v, z, 4)
            torch.cuda.synchronize()
            if mode == "graph":
                assert json.loads(sv.describe())["graph_recorded"]
            states[mode] = v.cpu().numpy().astype(np.float64)
    assert maxrel(states["uneven"], states["uniform"]) <= 1e-5
    np.testing.assert_array_equal(states["graph"], states["uniform"])
    vo = np.concatenate([O.code_admm(xo, d, beta, rho, 12)[0].reshape(-1) for xo in xs])
    assert rel(states["uniform"], vo) <= REL_TOL


def test_uneven_objective_matches_oracle(csc):
    K, s = 5, 5
    xs, d = batch(400, SIZES, K, 1, s)
    rng = np.random.default_rng(1)
    zs = [f32(np.where(rng.random((1, K) + hw) < 0.05, rng.standard_normal((1, K) + hw), 0.0)).astype(np.float64)
          for hw in SIZES]
    with csc.Solver(J=1, K=K, fs=(s, s), dims_list=SIZES, beta=0.6, rho=1.0) as sv:
        f = sv.objective(flat(xs), flat([d]), flat(zs))
    fo = sum(O.objective(xo, d, zo, 0.6) for xo, zo in zip(xs, zs))
    assert abs(f - fo) <= 1e-5 * fo


def test_uneven_rejects_unsupported_sizes_and_calls(csc):
    for bad in [(2000, 64), (64, 6), (9, 4)]:
        with pytest.raises(csc.CscError) as e:
            csc.Solver(J=1, K=2, fs=(5, 5), dims_list=[(64, 64), bad], beta=1.0, rho=1.0)
        assert e.value.status == 2 and f"{bad[0]}x{bad[1]}" in str(e.value)


# sides the one-map-per-CTA sweep cannot hold: odd widths, prime sides (Bluestein), sides above 128
LARGE = [(67, 131), (64, 64), (200, 181), (256, 300), (9, 8), (130, 97), (509, 64), (100, 100), (67, 131)]


@pytest.mark.parametrize("J,K,s,iters,sizes", [
    (1, 4, 5, 4, LARGE),
    (3, 3, 3, 3, [(31, 45), (64, 64), (97, 128), (140, 77)]),
    (1, 6, 11, 3, [(173, 211), (96, 70), (512, 509)]),
])
def test_uneven_large_odd_and_prime_sizes_match_oracle(csc, J, K, s, iters, sizes):
    """Images outside the one-map-per-CTA sweep (multi-pass transforms through HBM, Bluestein's
    chirp z-transform for lengths with prime factors above 7) mixed with images it holds: the state
    and the codes of every image against the oracle run image by image, and the objective."""
    import torch
    beta, rho = 0.3, 1.0
    xs, d = batch(500 + K, sizes, K, J, s)
    n_v = sum(K * H * W for H, W in sizes)
    with csc.Solver(J=J, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho) as sv:
        v = torch.zeros(n_v, device="cuda")
        z = torch.empty_like(v)
        sv.code(flat(xs), flat([d]), v, z, iters)
        torch.cuda.synchronize()
        info = json.loads(sv.describe())
        f = sv.objective(flat(xs), flat([d]), z)
    assert info["large_images"] > 0
    fo = 0.0
    for xo, vg, zg in zip(xs, split(v, sizes, K), split(z, sizes, K)):
        vo, zo = O.code_admm(xo, d, beta, rho, iters)
        assert rel(vg, vo) <= REL_TOL and maxrel(vg, vo) <= REL_TOL
        if np.any(zo != 0):
            assert rel(zg, zo) <= REL_TOL
        fo += O.objective(xo, d, zg, beta)
    assert abs(f - fo) <= 1e-5 * fo


def test_uneven_all_large_with_graph_replay(csc):
    """A batch with no image for the one-map-per-CTA sweep; CSC_FLAG_GRAPH replay equals eager."""
    import torch
    sizes = [(131, 67), (150, 150), (77, 301)]
    K, s, beta, rho = 3, 5, 0.3, 1.0
    xs, d = batch(700, sizes, K, 1, s)
    n_v = sum(K * H * W for H, W in sizes)
    out = {}
    for flags in (0, csc.CSC_FLAG_GRAPH):
        with csc.Solver(J=1, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho, flags=flags) as sv:
            v = torch.zeros(n_v, device="cuda")
            z = torch.empty_like(v)
            for _ in range(2):
                sv.code(flat(xs), flat([d]), v, z, 3)
            torch.cuda.synchronize()
            out[flags] = v.cpu().numpy()
    np.testing.assert_array_equal(out[0], out[csc.CSC_FLAG_GRAPH])
    vo = np.concatenate([O.code_admm(xo, d, beta, rho, 6)[0].reshape(-1) for xo in xs])
    assert rel(out[0].astype(np.float64), vo) <= REL_TOL


@pytest.mark.parametrize("sizes", [SIZES, [(67, 131), (64, 64), (150, 97), (200, 128)]])
def test_uneven_bf16_contractions_against_oracle(csc, sizes):
    """The uneven batch in CSC_MIXED_BF16 (bfloat16 operands of the per-frequency contractions,
    float32 accumulation), with and without images for the multi-pass engine: a stated error bound
    against the float64 oracle, the float32 run on the same batch within the float32 bar, and the
    objective float32 in both modes."""
    import torch
    from tests.test_gpu_precision import CODE_BF16_TOL
    K, s, iters, beta, rho = 6, 5, 6, 0.3, 1.0
    xs, d = batch(400, sizes, K, 1, s)
    n_v = sum(K * H * W for H, W in sizes)
    out = {}
    for prec in (csc.CSC_FP32, csc.CSC_MIXED_BF16):
        with csc.Solver(J=1, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho, precision=prec) as sv:
            v = torch.zeros(n_v, device="cuda")
            z = torch.empty_like(v)
            sv.code(flat(xs), flat([d]), v, z, iters)
            torch.cuda.synchronize()
            f = sv.objective(flat(xs), flat([d]), z)
            out[prec] = (split(z, sizes, K), f)
    zo = [O.code_admm(xo, d, beta, rho, iters)[1] for xo in xs]
    ref = np.concatenate([a.reshape(-1) for a in zo])
    e32 = rel(np.concatenate([a.reshape(-1) for a in out[csc.CSC_FP32][0]]), ref)
    e16 = rel(np.concatenate([a.reshape(-1) for a in out[csc.CSC_MIXED_BF16][0]]), ref)
    print(f"uneven coding rel err vs oracle: fp32 {e32:.2e}  bf16 {e16:.2e}")
    assert e32 <= REL_TOL
    assert 0 < e16 <= CODE_BF16_TOL
    # the objective of the bf16 codes, evaluated in float32, against the oracle on the same codes
    z16 = out[csc.CSC_MIXED_BF16][0]
    fo = sum(O.objective(xo, d, zz, beta) for xo, zz in zip(xs, z16))
    assert abs(out[csc.CSC_MIXED_BF16][1] - fo) <= 1e-5 * fo


@pytest.mark.parametrize("sizes", [[(128, 128), (64, 64), (40, 48)], [(67, 131), (64, 64), (200, 181)]])
def test_uneven_zero_iterations_codes_from_state(csc, sizes):
    """csc_code with zero iterations turns the state of every image into codes, z = rho (clamp(v) - v),
    over the whole batch and nothing beyond it."""
    import torch
    K, s, beta, rho = 3, 5, 0.3, 2.0
    xs, d = batch(800, sizes, K, 1, s)
    n_v = sum(K * H * W for H, W in sizes)
    g = torch.Generator(device="cuda").manual_seed(5)
    v = torch.randn(n_v, device="cuda", generator=g)
    z = torch.full((n_v + 1024,), 7.0, device="cuda")
    with csc.Solver(J=1, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho) as sv:
        sv.code(flat(xs), flat([d]), v, z[:n_v], 0)
        torch.cuda.synchronize()
    vn = v.cpu().numpy()
    zn = z.cpu().numpy()
    np.testing.assert_allclose(zn[:n_v], rho * (np.clip(vn, -beta, beta) - vn), rtol=1e-6, atol=1e-6)
    assert np.all(zn[n_v:] == 7.0)


def test_uneven_size_limits_match_oracle(csc):
    """The largest accepted side (1024; 1021 is prime, so its rows take a 2048-point Bluestein
    convolution) next to the smallest odd and prime ones, K = 2."""
    import torch
    sizes = [(1024, 1021), (8, 11), (13, 8), (9, 9)]
    K, s, iters, beta, rho = 2, 3, 3, 0.3, 1.0
    xs, d = batch(900, sizes, K, 1, s)
    n_v = sum(K * H * W for H, W in sizes)
    with csc.Solver(J=1, K=K, fs=(s, s), dims_list=sizes, beta=beta, rho=rho) as sv:
        v = torch.zeros(n_v, device="cuda")
        z = torch.empty_like(v)
        sv.code(flat(xs), flat([d]), v, z, iters)
        torch.cuda.synchronize()
        info = json.loads(sv.describe())
    assert info["large_images"] == 4
    for xo, vg in zip(xs, split(v, sizes, K)):
        vo, _ = O.code_admm(xo, d, beta, rho, iters)
        assert rel(vg, vo) <= REL_TOL and maxrel(vg, vo) <= REL_TOL


def test_uneven_autotune_cache(csc):
    """A second context on the same batch shape (sizes, K, J, precision) takes the launch shape the
    first one timed, without timing, and computes the same state."""
    import torch
    K, s, beta, rho = 7, 5, 0.3, 1.0
    xs, d = batch(950, SIZES, K, 1, s)
    n_v = sum(K * H * W for H, W in SIZES)
    out = []
    for _ in range(2):
        with csc.Solver(J=1, K=K, fs=(s, s), dims_list=SIZES, beta=beta, rho=rho) as sv:
            v = torch.zeros(n_v, device="cuda")
            z = torch.empty_like(v)
            sv.code(flat(xs), flat([d]), v, z, 3)
            torch.cuda.synchronize()
            out.append((json.loads(sv.describe()), v.cpu().numpy()))
    (da, va), (db, vb) = out
    assert db["autotuned"] and db["autotune_cached"]
    assert (db["threads_per_cta"], db["ctas"]) == (da["threads_per_cta"], da["ctas"])
    np.testing.assert_array_equal(vb, va)
