"""A short run of one hot-path kernel family on a fixed workload, as a target for ncu.

    python -m paper_1709_09479_gb300.profile_case coding [--N 100 --K 100 --H 128 --W 128 --iters 3]
    python -m paper_1709_09479_gb300.profile_case learning [...]

coding: csc_code with `iters` ADMM iterations (launch order: 2 spectra, solve setup, spectra,
prologue sweep, then `iters` sweeps). learning: one csc_code of `iters` iterations, then csc_learn
with `steps` learning steps. Inputs are the seeded 1/f^2 fields and Gaussian dictionary of bench.py.
"""
import argparse
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["coding", "learning"])
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--K", type=int, default=100)
    ap.add_argument("--H", type=int, default=128)
    ap.add_argument("--W", type=int, default=128)
    ap.add_argument("--s", type=int, default=11)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    a = ap.parse_args()
    import torch

    from paper_1709_09479_gb300 import csc, inputs
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
