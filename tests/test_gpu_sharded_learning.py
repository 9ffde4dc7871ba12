"""Data-parallel learning over image shards (the dictionary is shared by all images, Sec. 3.2; coding is
separable per image, Sec. 3.1): each shard's context codes its own images and returns its sums over
images (csc_learn_stats: the lag-window cross-correlations C and the right-hand side S Z^T x); the
shards' sums are added (the one reduction of a learning call) and csc_learn_solve runs the learning
steps from the reduced sums. The learned filters must equal those of one context holding every image
(within 1e-5, the float32 CG tolerance on slightly reordered sums) and the float64 oracle's.

The two-process case runs the shards as gloo ranks on this GPU. They never wait on each other inside
a kernel: the reduction is a host all-reduce, and the ranks take turns on the GPU between barriers.
"""
import os
import socket

import numpy as np
import pytest

from oracle import csc_oracle as O
from tests.gpu_common import REL_TOL, f32, make_problem, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu

CASE = dict(N=6, K=8, dims=(64, 64), s=5, beta=0.3, rho=1.0, n_code=10, steps=3, cg_tol=1e-7)


@pytest.fixture(scope="module")
def csc():
    import torch
    assert torch.cuda.is_available()
    from paper_1709_09479_gb300 import csc as lib
    return lib


def solver(csc, n_images, c=CASE):
    return csc.Solver(J=1, K=c["K"], fs=(c["s"], c["s"]), dims=c["dims"], n_images=n_images, beta=c["beta"],
                      rho=c["rho"], cg_max=400, cg_tol=c["cg_tol"])


def single_context(csc, x, d, c=CASE):
    import torch
    with solver(csc, x.shape[0], c) as sv:
        v = torch.zeros((x.shape[0], c["K"]) + c["dims"], device="cuda")
        z = torch.empty_like(v)
        sv.code(to_cuda(x), to_cuda(d), v, z, c["n_code"])
        dv = to_cuda(d)
        mu = torch.full((c["K"],), 0.5, dtype=torch.float64, device="cuda")
        sv.learn(to_cuda(x), z, dv, mu, c["steps"])
        return to_np(dv), mu.cpu().numpy(), to_np(z)


def shard_stats(csc, xs, d, c=CASE):
    """Code one shard and return (C, b, z) as host arrays."""
    import torch
    with solver(csc, xs.shape[0], c) as sv:
        v = torch.zeros((xs.shape[0], c["K"]) + c["dims"], device="cuda")
        z = torch.empty_like(v)
        sv.code(to_cuda(xs), to_cuda(d), v, z, c["n_code"])
        cs, bs = sv.stats_shapes()
        C = np.zeros(cs, dtype=np.float32)
        b = np.zeros(bs, dtype=np.float32)
        sv.learn_stats(to_cuda(xs), z, C, b)
        return C, b, to_np(z)


def test_stats_are_sums_over_images_and_sharded_learning_matches(csc):
    c = CASE
    x, d = make_problem(400, c["N"], c["K"], 1, c["dims"], c["s"])
    d_full, mu_full, z_full = single_context(csc, x, d)
    h = c["N"] // 2
    C0, b0, z0 = shard_stats(csc, x[:h], d)
    C1, b1, z1 = shard_stats(csc, x[h:], d)
    Cf, bf, _ = shard_stats(csc, x, d)
    # coding is per image: the shards' codes are the full batch's
    assert rel(np.concatenate([z0, z1]), z_full) <= 1e-6
    # C and b are sums over images
    assert rel(C0 + C1, Cf) <= 1e-5 and rel(b0 + b1, bf) <= 1e-5
    # C is the code cross-correlation on the lag window, b = S Z^T x (oracle operators, float64)
    zf = f32(z_full).astype(np.float64)
    fh = fw = c["s"]
    ops = O.LearningOperators(zf)
    b_ref = O.crop_support(ops.ZT(x[:, 0]), (fh, fw))
    assert rel(bf[:, 0], b_ref) <= 1e-5
    for k in range(c["K"]):
        for kp in (0, c["K"] - 1):
            # C[k][k'][ta][tb] = sum_n sum_p z_nk(p) z_nk'(p + t): correlation of z_k with z_k'
            corr = O.irdft(np.sum(np.conj(O.rdft(zf[:, k], 2)) * O.rdft(zf[:, kp], 2), axis=0), c["dims"])
            win = np.roll(corr, (fh - 1, fw - 1), axis=(0, 1))[: 2 * fh - 1, : 2 * fw - 1]
            assert rel(Cf[k, kp], win) <= 1e-5
    # learning from the reduced sums equals learning on one context
    import torch
    with solver(csc, h) as sv:
        dv = to_cuda(d)
        mu = torch.full((c["K"],), 0.5, dtype=torch.float64, device="cuda")
        its = sv.learn_solve(to_cuda(C0 + C1), to_cuda(b0 + b1), dv, mu, c["steps"])
        d_sh, mu_sh = to_np(dv), mu.cpu().numpy()
    assert len(its) == c["steps"]
    assert rel(d_sh, d_full) <= 1e-5, rel(d_sh, d_full)
    np.testing.assert_allclose(mu_sh, mu_full, rtol=1e-5)
    # and the oracle's learning on the full batch's codes
    d_o, mu_o, _, _ = O.learn_paper(x, zf, d, np.full(c["K"], 0.5), np.zeros_like(x), c["steps"])
    assert rel(d_sh, d_o) <= REL_TOL
    # host arrays for C, b, d and mu give the same bits as device arrays
    with solver(csc, h) as sv:
        dh = f32(d)
        muh = np.full(c["K"], 0.5)
        sv.learn_solve(C0 + C1, b0 + b1, dh, muh, c["steps"])
    np.testing.assert_array_equal(dh.astype(np.float64), d_sh)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1709_09479_gb300 import csc
    c = CASE
    x, d = make_problem(400, c["N"], c["K"], 1, c["dims"], c["s"])
    per = c["N"] // world
    xs = x[rank * per:(rank + 1) * per]
    C = b = None
    for turn in range(world):            # the ranks take turns on the GPU
        if turn == rank:
            C, b, _ = shard_stats(csc, xs, d)
            torch.cuda.synchronize()
        dist.barrier()
    Ct, bt = torch.from_numpy(C), torch.from_numpy(b)
    dist.all_reduce(Ct)                  # the one reduction of the learning call
    dist.all_reduce(bt)
    d_out = mu_out = None
    for turn in range(world):
        if turn == rank:
            with solver(csc, per) as sv:
                dv = to_cuda(d)
                mu = torch.full((c["K"],), 0.5, dtype=torch.float64, device="cuda")
                sv.learn_solve(Ct.numpy(), bt.numpy(), dv, mu, c["steps"])
                d_out, mu_out = to_np(dv), mu.cpu().numpy()
        dist.barrier()
    np.save(os.path.join(outdir, f"d{rank}.npy"), d_out)
    np.save(os.path.join(outdir, f"mu{rank}.npy"), mu_out)
    dist.destroy_process_group()


def test_two_gloo_ranks_learn_the_single_context_dictionary(csc, tmp_path):
    import torch.multiprocessing as mp
    c = CASE
    x, d = make_problem(400, c["N"], c["K"], 1, c["dims"], c["s"])
    d_full, mu_full, _ = single_context(csc, x, d)
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    d0, d1 = np.load(tmp_path / "d0.npy"), np.load(tmp_path / "d1.npy")
    np.testing.assert_array_equal(d0, d1)          # replicated solve: identical on every rank
    assert rel(d0, d_full) <= 1e-5, rel(d0, d_full)
    np.testing.assert_allclose(np.load(tmp_path / "mu0.npy"), mu_full, rtol=1e-5)
