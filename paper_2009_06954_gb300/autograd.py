"""torch.autograd wrapper: x = A^-1 b with the adjoint in the backward pass.

Backward of L(x): lambda solves A^T lambda = dL/dx (the transposed system,
preconditioned with P^T = M~_r + I - J~, inner mrs on the transposed deflated
system); dL/db = lambda and dL/dA_ij = -lambda_i x_j on A's nonzeros only.
"""
import torch


class AsssSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, b, a_values):
        # a_values carries A's nonzeros (CSR order) for autograd; the solver was set
        # up from the same values.
        x, st = solver.solve(b.detach().contiguous())
        ctx.solver = solver
        ctx.stats = st
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, dA, _ = ctx.solver.solve_adjoint(gx.detach().contiguous(), x=x)
        return None, lam, dA
