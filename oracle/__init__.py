"""Plain FP64 CPU oracle of the sub-grid DG shallow-water hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.
"""
