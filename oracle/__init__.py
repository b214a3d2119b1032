"""Oracle: plain, slow, obviously-correct CPU reference of the method (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` / reference leg
may import anything from here.  It shares no code with the GPU path (``paper_1710_05134_gb300``)
and never imports it; both draw inputs from ``gen`` only.

Contents
  core.py          inertia by dense Bunch-Kaufman (c1) and by plain sparse multifrontal LDL^T (c3),
                   dense Cholesky-reduced generalized eigensolver (c2), closed-form spectra.
  three_stage.py   Algorithms 1, 1', 2, 3 and 4 of the paper, step by step, on top of core.py.
  orc.c            the C parts of core.py (compiled by build.py with gcc).

Parity pins: every function is pinned in tests/test_oracle_*.py against something other than
itself (closed forms, brute force, library routines it does not call, invariants); see the header
of each function.  Functions with no such pin say "parity unpinned".
"""
