"""Plain FP64 CPU oracle for sketched-preconditioned SVRG ridge regression.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct reference
that the CUDA path is checked against.  Only the test-suite, the smoke check of
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The product library never calls it and shares no
code with it: the two sides meet only at the seeded input generator
(``paper_1602_02350_gb300.synth``), which holds none of the method's arithmetic.

Everything is numpy in float64 and follows the paper (Gonen, Orabona,
Shalev-Shwartz, "Solving Ridge Regression using Sketched Preconditioned SVRG")
step by step:

* ``ridge``     - Eq. (1) objective, Eq. (2) correlation matrix, Eq. (3) average
                  condition number, the normal-equation closed form (Sec. 3).
* ``streams``   - the counter-based Philox4x32-10 generator (Salmon et al.,
                  SC'11) and the random draws the method makes from it:
                  Gaussian test matrix (Alg. 2), CountSketch hash, the
                  importance-sampling index stream of Alg. 1.
* ``sketch``    - Alg. 2 (randomized Block Lanczos; q = 1 is the range sketch).
* ``precond``   - Eq. (11) sketched preconditioner, the data transform and the
                  n+d decomposition of Sec. 5.1, smoothness constants of Alg. 3.
* ``svrg``      - Alg. 1 (SVRG with importance sampling) on the n+d components.
* ``pipeline``  - Alg. 3 end to end.
* ``catalyst``  - accelerated SVRG (Catalyst) around Alg. 1 on the same components (Sec. 1, Thm 1).
* ``proposal``  - the theory-set parameters of Sec. 3 / Thm 1 and the parameter-proposal
                  network (forward, backpropagation, Adam) that the library trains.

Every pinned function is tested in ``tests/test_oracle_*.py`` against facts the
paper and linear algebra fix (closed forms, identities, brute force on tiny
inputs, library routines).  Functions without such a pin say
"parity unpinned" in their docstring.
"""

from . import ridge, streams, sketch, precond, svrg, pipeline, proposal, catalyst  # noqa: F401
