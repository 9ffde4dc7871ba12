"""torch.autograd wrappers of the library's unrolled coding and reconstruction (argument marshalling
only; forward and backward both run in libcsc.so's kernels).

    z_T = UnrolledCode.apply(solver, x, d, iters, every)    # T dual-ADMM iterations from v = 0
    xr  = Synthesize.apply(solver, d, z)                    # sum_k d_k * z_k

UnrolledCode's backward runs the hand-written adjoint (csc_code_backward) through the T iterations,
recomputing states from checkpoints taken every `every` iterations.
"""
import torch

from . import csc as _csc


def _c(t):
    return t.detach().contiguous()


class UnrolledCode(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, x, d, iters, every):
        x, d = _c(x), _c(d)
        v = torch.zeros((solver.N, solver.K) + tuple(solver.dims), device=x.device, dtype=torch.float32)
        z = torch.empty_like(v)
        tape = torch.empty(_csc.csc_tape_bytes(solver.ctx, iters, every), dtype=torch.uint8, device=x.device)
        _csc.csc_code_unrolled(solver.ctx, x, d, v, z, iters, every, tape)
        ctx.solver, ctx.iters, ctx.every = solver, iters, every
        ctx.save_for_backward(x, d, tape)
        return z

    @staticmethod
    def backward(ctx, gz):
        x, d, tape = ctx.saved_tensors
        gx = torch.empty_like(x)
        gd = torch.empty_like(d)
        _csc.csc_code_backward(ctx.solver.ctx, x, d, tape, ctx.iters, ctx.every, _c(gz), gx, gd)
        return None, gx, gd, None, None


class Synthesize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, d, z):
        d, z = _c(d), _c(z)
        out = torch.empty((solver.N, solver.J) + tuple(solver.dims), device=z.device, dtype=torch.float32)
        _csc.csc_synthesize(solver.ctx, d, z, out)
        ctx.solver = solver
        ctx.save_for_backward(d, z)
        return out

    @staticmethod
    def backward(ctx, gout):
        d, z = ctx.saved_tensors
        gz = torch.empty_like(z)
        gd = torch.empty_like(d)
        _csc.csc_synthesize_backward(ctx.solver.ctx, d, z, _c(gout), gz, gd)
        return None, gd, gz
