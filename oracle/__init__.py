"""CPU oracle for the free-mesh transform: test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` /
``--impl reference`` legs may import this package.  The CUDA library never
links or calls it.
"""
