"""CPU oracle for ALTO encode, MTTKRP and CP-ALS (test infrastructure only).

This package is the plain, slow, obviously-correct restatement of what the
GPU path computes, written from the paper (ALTO, arXiv 2403.06348):

* ``alto_ref``  -- numpy/Python: the bit plan and linearization of Section III-A
  (Fig. 5/6 text), the ordering step, the nnz-balanced line segments and mode
  intervals of Section IV-A, MTTKRP by its definition (Alg. 1 MTTKRP line,
  Alg. 3), the dense unfolding x Khatri-Rao check of Section II-A, CP-ALS in
  the order of Alg. 1, and the storage formulas Eq. 1-3.
* ``coo_ref.c`` (via ``cref``) -- plain C fp64 COO MTTKRP / linearization for
  sizes where numpy would need too much memory; it is also what the CPU
  baseline times.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import, call, link or run anything in this package.
The product path (``paper_2403_06348_gb300``) never imports it and shares no
code with it; the two meet only through the seeded inputs from ``synth``.

Parity pins (tests/test_oracle_*.py) tie every function to something other
than itself: the worked example printed in the paper, closed forms, dense
brute force, invariants and the mathematics of least squares. No function
here is "parity unpinned".
"""
