"""FP64 CPU oracle for isoparametric FE assembly -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and the product path never calls it.
"""
from .oracle import (  # noqa: F401
    build,
    n_ref,
    tabulate,
    pattern,
    eval_points,
    geometry,
    local_matrices,
    assemble,
    assemble_threads,
    max_threads,
    adjoint,
    load,
    kll,
    mcf_step,
    p1_exact,
)
from .lift import lift_order  # noqa: F401
