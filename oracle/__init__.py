"""FP64 CPU oracle for the fractional-Laplacian solver of Minden & Ying,
"A simple solver for the fractional Laplacian in multiple dimensions"
(arXiv:1802.03770).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.
It shares no code, table or constant generator with the CUDA library in
``paper_1802_03770_gb300/csrc``; the two meet only in the seeded input
generator ``paper_1802_03770_gb300/inputs.py``, which holds none of the
method's arithmetic.

Layout (each function cites the passage it follows):

* ``constants`` -- C_{alpha,d} (eq. fl), the window W_delta (eq. window),
  the constants A_{1,d}, A_{2,d} (eq. int1constants) and A_{3,d} (eq. a3).
* ``operator``  -- the discrete operator M of eq. linearelliptic: dense
  matrix (direct summation) and the zero-padded FFT apply (Sec. 3.1).
* ``precond``   -- the finite-difference Laplacian part L of the split
  M = C h^d (K + L) and its fast (DST-I) solve (Sec. 3.1, Sec. 3.2).
* ``solvers``   -- CG / PCG (Sec. 3.1), the theta time step (eq.
  timestepping, Sec. 3.2) and mixed-precision iterative refinement.

Precision is FP64 throughout except where a function says otherwise.
Parity status: every function is pinned by a test under ``tests/``
(``test_oracle_*.py``) against printed values of the paper, closed forms
or invariants; see the module docstrings.
"""

from . import constants, operator, precond, solvers  # noqa: F401
