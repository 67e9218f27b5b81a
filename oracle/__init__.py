"""Plain FP64 CPU oracle of the two-phase lattice Boltzmann step (accLB, arXiv
2505.01126, Sec. 2).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2505_01126_gb300``; the two meet only through
the seeded input generators, which hold none of the method's arithmetic.
"""
from .oracle import (  # noqa: F401
    FORCE_ABC,
    FORCE_CONST,
    FORCE_LINEAR,
    FORCE_NONE,
    Oracle,
    build,
    equilibrium,
    gradient,
    guo_source,
    interface,
    lattice7,
    lattice27,
    phase_equilibrium,
    regularized_neq,
    set_threads,
    threads,
    weno5_face,
)
