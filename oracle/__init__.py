"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct CPU statement of what the FastWalk hot path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline legs may import it.  It shares no code with the CUDA path
(``paper_2510_20604_gb300``), and neither side imports the other; the seeded
input generators live in ``synth`` and hold none of the method's arithmetic.

Modules
-------
``wilson``  (C, via ctypes): Philox-4x32-10, Vose alias tables, the successor
            stacks and the sequential Wilson loop of Algorithm 3 (FastWalk).
``exact``   dense FP64 random walk centrality by three independent routes
            (Section 2.2-2.3, Eq. 2) and diag of the pivot-deleted inverse.
``apprwc``  Algorithm 1 (AppRWC) / Theorem 3.1 (Eq. 3) recovery.
``grad``    dense gradient of J(w) = sum_v c_v H_v(w) and its central finite
            difference.

Parity status of every function is listed in each module's docstring.
"""
from . import wilson, exact, apprwc, grad  # noqa: F401
