"""GB300 (sm_103a) implementation of the solve path of the two-level ASSS + mrs
scheme for general sparse A x = b (Manguoglu & Mehrmann, arXiv 2009.06954).

The compute runs in ``libasss.so`` (hand-written CUDA, C ABI in ``include/asss.h``);
this package only marshals arguments.  ``Solver`` wraps set-up/solve/adjoint,
``skew_symmetrizer``, ``skew_lanczos`` and ``mrs`` expose single steps, and
``asss_solve`` is the differentiable PyTorch entry (adjoint in the backward pass).
"""
from .binding import (EXPORTED, LIB_PATH, AsssError, BatchSolver, Solver, lib, matching_scaling, mrs,  # noqa: F401
                      mrs_multi, skew_lanczos, skew_symmetrizer)


def asss_solve(solver, b, a_values):
    """Differentiable x = A^-1 b (torch); see ``autograd.AsssSolveFn``."""
    from .autograd import AsssSolveFn
    return AsssSolveFn.apply(solver, b, a_values)
