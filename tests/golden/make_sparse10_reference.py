"""Writes tests/golden/sparse10_oracle.json: the float64 oracle's objective trajectory on the
10-image sparse-synthetic workload (N=10 grey 100x100 images, K=16 filters 11x11, beta=1, rho=10,
10 outer rounds of 20 coding iterations and 20 learning steps; Algorithm 1).

Inputs are the seeded generators of paper_1709_09479_gb300.inputs (image seed 0, dictionary seed
1), rounded to float32 exactly as the GPU receives them. Only oracle/ computes. Run:
    python tests/golden/make_sparse10_reference.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import csc_oracle as O  # noqa: E402
from paper_1709_09479_gb300 import inputs  # noqa: E402

CONFIG = {"N": 10, "H": 100, "W": 100, "K": 16, "s": 11, "beta": 1.0, "rho": 10.0,
          "n_outer": 10, "n_code": 20, "n_learn": 20, "image_seed": 0, "dict_seed": 1,
          "density": 0.01, "noise": 0.01}


def workload():
    c = CONFIG
    data = inputs.sparse_synthetic(seed=c["image_seed"], N=c["N"], dims=(c["H"], c["W"]), K=c["K"],
                                   s=c["s"], density=c["density"], noise=c["noise"])
    x = data["x"].astype(np.float32).astype(np.float64)
    d0 = inputs.unit_filters(c["dict_seed"], c["K"], 1, (c["s"], c["s"])).astype(np.float32).astype(np.float64)
    return x, d0


def main():
    c = CONFIG
    x, d0 = workload()
    t0 = time.time()
    out = O.csc_alternate(x, d0, c["beta"], c["rho"], c["n_outer"], c["n_code"], c["n_learn"],
                          log=lambda h: print(h["outer"], h["f_code"], h["f_learn"], sum(h["cg_iters"]), flush=True))
    hist = [{"outer": h["outer"], "f_code": h["f_code"], "f_learn": h["f_learn"],
             "cg_iters": h["cg_iters"]} for h in out["history"]]
    res = {"config": c, "history": hist, "f_final": hist[-1]["f_learn"],
           "oracle_seconds": time.time() - t0, "generator": "tests/golden/make_sparse10_reference.py"}
    with open(os.path.join(HERE, "sparse10_oracle.json"), "w") as f:
        json.dump(res, f, indent=1)
    print("f* =", res["f_final"], "in", res["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
