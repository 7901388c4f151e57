"""FP64 CPU oracle for CutQC's reconstruction (arXiv 2012.02333).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package; only the test suite, the smoke check in
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA path: its gate matrices,
its statevector simulator, its attribution and its reconstruction are all its
own, written from the paper in plain numpy (float64 / complex128), slow and
obviously correct.  The only thing it takes from the package is the seeded
circuit and cut structure in ``paper_2012_02333_gb300.circuits``, which holds
none of the method's arithmetic.

Modules
  statevector   textbook statevector simulation (Sec. 2, Fig. 2a ground truth)
  attribution   subcircuit variants (Fig. 3 / Sec. 3.1) and shot attribution
                (Eq. 3, Sec. 3.2.2) into Pauli-indexed subcircuit tensors, and
                the merged tensors of a dynamic-definition recursion taken
                straight from the variant distributions
  reconstruct   full-definition sum (Sec. 3.2.3, Sec. 3.3, Sec. 4.2), dynamic
                definition (Algorithm 1, Sec. 4.3), and the gradient of an
                expectation value over the reconstructed distribution
  metrics       the chi^2 loss of Eq. 16, total variation, and inverse-transform
                sampling of outcomes from a reconstructed distribution
  cutsearch     exhaustive search of the cut model of Sec. 4.1 (Eqs. 4-15) on
                tiny circuits: every assignment enumerated, cost by Eq. 14

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself: textbook states, the paper's worked single-cut formulas,
brute-force simulation of the uncut circuit (exactness, Sec. 3.2.3), the
Fig. 7 dynamic-definition example, closed forms and invariants.
"""
