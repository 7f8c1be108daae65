"""ORACLE: test infrastructure for the q-NSCH primitive-method solver.

A plain, serial FP64 CPU implementation (``qnsch_ref.c``) of the fully discrete
primitive scheme of Sec. 6.1 and the FAS multigrid of Sec. 7.1 of Guo, Lin,
Lowengrub & Wise (arXiv:1703.06606), with a ctypes wrapper (``ref.py``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA product library.
"""
