"""FP64 CPU oracle for the two-level ASSS + mrs scheme (arXiv 2009.06954).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method in numpy/scipy float64.  It shares no code with the
CUDA path and is imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``.  The product path never calls it.

Every function cites the part of the paper it restates (section, equation,
figure or appendix).  Pins that tie it to the paper and to mathematics other
than itself live in ``tests/test_oracle_*.py``.

Functions without an independent pin: none at present (see the test files for
which check pins which function).
"""
from .asss import (  # noqa: F401
    splitmix64_uniform,
    equilibrate,
    lls_system,
    skew_symmetrizer,
    shift_and_lowrank,
    lowrank_decomposition,
    inner_skew_operator,
    skew_lanczos,
    lanczos_tridiagonal,
    mrs,
    AsssOracle,
    tfqmr_cycle,
    fgmres_cycle,
)
from .ildl import (  # noqa: F401
    FactoredSkew,
    colour_order,
    colouring_priorities,
    ildl0,
    jp_colouring,
    splitmix64_u64,
    structural_pattern,
    values_on_pattern,
)
from .matching import matching_costs, matching_scaling, max_product_matching  # noqa: F401
