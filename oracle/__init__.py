"""FP64 CPU oracle of AA-PDHG / FAA-PDHG (test infrastructure, not product code).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.
"""
