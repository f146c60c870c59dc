"""CPU oracle of the pf-FRG flow (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product library never loads it.
"""
from .oracle import OracleFlow, OracleFlowTRI, tri_spin_tables, build, load, mesh_exponential, cutoff_exponential, spin_tables  # noqa: F401
