"""FP64 CPU oracle for the three-distribution MRT-LB step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1608_04118_gb300``.
"""
from .ltne_oracle import (  # noqa: F401
    OracleParams,
    Oracle,
    ComplexOracle,
    build,
    ergun_diameter,
    lattice_tables,
    num_threads,
    set_num_threads,
)
