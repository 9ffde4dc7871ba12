"""Helpers shared by the GPU parity tests (imported lazily so CPU-only collection never loads CUDA)."""
import numpy as np

#: relative (norm-wise) error bar of the float32 GPU path against the float64 oracle, and the
#: element-wise bar relative to the largest magnitude. FP32 FFTs of 10^4 points carry ~1e-6
#: relative error per transform and the ADMM map is non-expansive, so 20 iterations stay near
#: 2e-5; 1e-4 leaves a factor of ~5.
REL_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def to_cuda(a):
    import torch
    return torch.from_numpy(f32(a)).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def make_problem(seed, N, K, J, dims, s, kind="powerlaw"):
    """Seeded images (float32-representable) and unit-norm filters, returned as float64 arrays."""
    from paper_1709_09479_gb300 import inputs
    if kind == "sparse":
        data = inputs.sparse_synthetic(seed=seed, N=N, dims=dims, K=K, s=s)
        x = data["x"] if J == 1 else np.repeat(data["x"], J, axis=1)
    else:
        x = inputs.powerlaw_field(seed, N, J, dims)
    d = inputs.unit_filters(seed + 100, K, J, (s, s))
    return f32(x).astype(np.float64), f32(d).astype(np.float64)
