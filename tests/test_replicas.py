"""Host logic of the multi-GPU benchmark mode on CPU (gloo, world size 2).

The job's time is the slowest rank's, the value counts every rank's iterations, and rank 0 alone
prints. Coding is separable per image (Sec. 3.1), so ranks code their own images with no exchange;
learning shares the dictionary (Sec. 3.2), so each learning call reduces two sums over images across
the ranks: the code cross-correlations on the (2fh-1) x (2fw-1) lag window, C_kk'(t) =
sum_n sum_p z_nk(p) z_nk'(p + t), and the right-hand side b = S Z^T x. Here two gloo ranks check the
max-over-ranks reduction, that the all-reduced shard sums equal the sums over all images, and that the
normal equations assembled from the reduced C and b give the filters of the oracle's learning route;
and that the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 7.0 * rank, dist)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put((rank, got))


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 17.0, 1: 17.0}


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 3, 2

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def _shard_sums(x, z, fs):
    """(C, b) of a set of images, written out with numpy FFTs: C [K][K][2fh-1][2fw-1], b [K][fh][fw]."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import csc_oracle as O
    fh, fw = fs
    K = z.shape[1]
    dims = z.shape[2:]
    zh = np.fft.rfft2(z)
    C = np.zeros((K, K, 2 * fh - 1, 2 * fw - 1))
    for k in range(K):
        for kp in range(K):
            corr = np.fft.irfft2(np.sum(np.conj(zh[:, k]) * zh[:, kp], axis=0), s=dims)
            C[k, kp] = np.roll(corr, (fh - 1, fw - 1), axis=(0, 1))[: 2 * fh - 1, : 2 * fw - 1]
    b = O.crop_support(O.LearningOperators(z).ZT(x[:, 0]), fs)
    return C, b


def _sums_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    x, z = _shard_problem()
    per = x.shape[0] // world
    C, b = _shard_sums(x[rank * per:(rank + 1) * per], z[rank * per:(rank + 1) * per], (3, 3))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Ct, bt = torch.from_numpy(C), torch.from_numpy(b)
        dist.all_reduce(Ct)
        dist.all_reduce(bt)
    finally:
        dist.destroy_process_group()
    out.put((rank, Ct.numpy(), bt.numpy()))


def _shard_problem():
    import numpy as np
    rng = np.random.default_rng(90)
    N, K, dims = 4, 3, (9, 10)
    x = rng.standard_normal((N, 1) + dims)
    z = np.where(rng.random((N, K) + dims) < 0.3, rng.standard_normal((N, K) + dims), 0.0)
    return x, z


def test_sharded_learning_sums_gloo_world2():
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import csc_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sums_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, C, b = q.get(timeout=120)
        res[r] = (C, b)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    x, z = _shard_problem()
    C_all, b_all = _shard_sums(x, z, (3, 3))
    for r in (0, 1):
        np.testing.assert_allclose(res[r][0], C_all, atol=1e-12)
        np.testing.assert_allclose(res[r][1], b_all, atol=1e-12)
    # the normal equations from the reduced sums: [S Z^T Z S^T p]_k(q) = sum_k' sum_q' C_kk'(q - q') p_k'(q')
    C, b = res[0]
    K, fh, fw = C.shape[0], 3, 3
    M = np.zeros((K * fh * fw, K * fh * fw))
    for k in range(K):
        for a in range(fh):
            for c in range(fw):
                for kp in range(K):
                    for ap in range(fh):
                        for cp in range(fw):
                            M[(k * fh + a) * fw + c, (kp * fh + ap) * fw + cp] = C[k, kp, a - ap + fh - 1, c - cp + fw - 1]
    mu = np.array([0.4, 0.9, 1.7])
    d = np.linalg.solve(M + 2.0 * np.diag(np.repeat(mu, fh * fw)), b.reshape(-1)).reshape(K, fh, fw)
    want = O.learn_normal_equations(x, z, (K, 1, fh, fw), mu)[:, 0]
    np.testing.assert_allclose(d, want, atol=1e-10)
