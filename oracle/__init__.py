"""CPU oracle of the FMM data-structure build (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg may import this package.  The library itself never does.
"""
