"""CPU FP64 oracle for the cell-centred finite-volume method of Manapy
(arXiv 2203.00925): plain, slow, written to be checked against the paper by eye.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The GPU library never calls it
and shares no code with it; the two meet only in the seeded inputs of ``synth/``.

Modules (each function cites the passage it follows):

* ``geometry``  - faces, volumes, centroids, area vectors (Section 2.1, eq. 2-4).
* ``ls``        - least-squares cell gradient (Algorithm "grad") and least-squares
                  vertex interpolation (Algorithm "ls").
* ``fv``        - diamond face gradient (eq. "diamond"), upwind convective flux
                  (eq. 15 with psi = 0), the residual of eq. 4, explicit Euler and the
                  three-stage Runge-Kutta of eq. 6.
* ``poisson``   - the diamond Poisson operator (eq. 7 / eq. "laplace"), its assembled
                  sparse matrix, the Dirichlet lift and a direct solve.
* ``streamer``  - the electron drift-diffusion + Poisson step (eq. 10) with the
                  coefficient readings of the synthetic streamer workloads.

Pins (tests/test_oracle_*.py) tie every function to something other than itself:
closed forms, invariants, brute force. Functions without such a pin are listed
here as "parity unpinned": none at present.
"""
