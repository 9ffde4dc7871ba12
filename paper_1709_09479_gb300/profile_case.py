"""A short run of one hot-path kernel family on a fixed workload, as a target for ncu.

    python -m paper_1709_09479_gb300.profile_case coding [--N 100 --K 100 --H 128 --W 128 --iters 3]
    python -m paper_1709_09479_gb300.profile_case learning [...]
    python -m paper_1709_09479_gb300.profile_case uneven [--iters 3]
    python -m paper_1709_09479_gb300.profile_case video [--iters 3 --steps 2]

coding: csc_code with `iters` ADMM iterations (launch order: 2 spectra, solve setup, spectra,
prologue sweep, then `iters` sweeps). learning: one csc_code of `iters` iterations, then csc_learn
with `steps` learning steps. uneven: the 256-image batch of bench.py's uneven256 workload (sides uniform
in [64, 512], K = 64; `--images` takes its first images only; `--sides smooth64-128` draws the sides
from the even 7-smooth sizes in [64, 128] instead), one csc_code of `iters` iterations (launch order: the setup transforms and the
per-class solve setup, the autotuner's sweeps when some images fit one map per CTA, then the call's
prologue and sweeps). video: bench.py's
video3d workload (3 x 32 x 128^2, K = 64 colour filters 5 x 11 x 11), one csc_code of `iters`
iterations, then csc_learn with `steps` learning steps (CG to 1e-6, at most 100 iterations). Inputs
are the seeded 1/f^2 fields and Gaussian dictionaries of bench.py.
"""
import argparse
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["coding", "learning", "uneven", "video"])
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--K", type=int, default=100)
    ap.add_argument("--H", type=int, default=128)
    ap.add_argument("--W", type=int, default=128)
    ap.add_argument("--s", type=int, default=11)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--images", type=int, default=256, help="uneven: number of images")
    ap.add_argument("--sides", choices=["64-512", "smooth64-128"], default="64-512",
                    help="uneven: sides uniform in [64, 512], or drawn from the even 7-smooth sizes in [64, 128]")
    a = ap.parse_args()
    import torch

    from paper_1709_09479_gb300 import csc, inputs
    if a.what == "video":
        J, T, K, ft = 3, 32, 64, 5
        x = torch.from_numpy(inputs.powerlaw_field(4, 1, J, (T, 128, 128)).astype(np.float32)).cuda()
        d = torch.from_numpy(inputs.unit_filters(40, K, J, (ft, a.s, a.s)).astype(np.float32)).cuda()
        v = torch.zeros((1, K, T, 128, 128), device="cuda")
        z = torch.empty_like(v)
        mu = torch.full((K,), 0.5, dtype=torch.float64, device="cuda")
        with csc.Solver(J=J, K=K, fs=(a.s, a.s), ft=ft, dims=(T, 128, 128), n_images=1, beta=0.5, rho=0.1,
                        cg_max=100, cg_tol=1e-6) as sv:
            sv.code(x, d, v, z, a.iters)
            its = sv.learn(x, z, d, mu, a.steps)
        torch.cuda.synchronize()
        print("ok", float(v.abs().sum()), list(its))
        return 0
    if a.what == "uneven":
        rng = np.random.default_rng(3)
        if a.sides == "64-512":
            sizes = [(int(rng.integers(64, 513)), int(rng.integers(64, 513))) for _ in range(a.images)]
        else:
            sides = [64, 70, 72, 80, 84, 90, 96, 98, 100, 108, 112, 120, 126, 128]
            sizes = [(int(rng.choice(sides)), int(rng.choice(sides))) for _ in range(a.images)]
        K = 64
        xs = np.concatenate([inputs.powerlaw_field(1000 + i, 1, 1, hw).reshape(-1) for i, hw in enumerate(sizes)])
        x = torch.from_numpy(xs.astype(np.float32)).cuda()
        d = torch.from_numpy(inputs.unit_filters(30, K, 1, (a.s, a.s)).astype(np.float32)).cuda()
        npx = sum(H * W for H, W in sizes)
        v = torch.zeros(K * npx, device="cuda")
        z = torch.empty_like(v)
        with csc.Solver(J=1, K=K, fs=(a.s, a.s), dims_list=sizes, beta=1.0, rho=0.1) as sv:
            sv.code(x, d, v, z, a.iters)
        torch.cuda.synchronize()
        print("ok", float(v.abs().sum()))
        return 0
    x = torch.from_numpy(inputs.powerlaw_field(2, a.N, 1, (a.H, a.W)).astype(np.float32)).cuda()
    d = torch.from_numpy(inputs.unit_filters(21, a.K, 1, (a.s, a.s)).astype(np.float32)).cuda()
    v = torch.zeros((a.N, a.K, a.H, a.W), device="cuda")
    z = torch.empty_like(v)
    with csc.Solver(J=1, K=a.K, fs=(a.s, a.s), dims=(a.H, a.W), n_images=a.N, beta=1.0, rho=0.1) as sv:
        if a.what == "coding":
            sv.code(x, d, v, z, a.iters)
        else:
            sv.code(x, d, v, z, a.iters)
            mu = torch.full((a.K,), 0.5, dtype=torch.float64, device="cuda")
            sv.learn(x, z, d, mu, a.steps)
    torch.cuda.synchronize()
    print("ok", float(v.abs().sum()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
