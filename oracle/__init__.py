"""FP64 CPU oracle for the particle-mesh (PM) + BullFrog hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never calls it, shares no code, headers,
tables or constants with it, and this package imports nothing from the
product package.

It restates, step by step and in double precision, what the paper
"DISCO-DJ II: a differentiable particle-mesh code for cosmology"
(arXiv:2510.05206) defines:

* ``cosmology``  - growth ODEs for D and E (App. B), the BullFrog and FastPM
  kick coefficients (Sec. 2.4), the BBKS linear spectrum normalised to sigma8.
* ``mesh``       - mass-assignment kernels (Table 1), scatter / gather and
  their position derivatives (App. C), finite-difference gradient and
  Laplacian kernels (Table 2), the Poisson force field (Sec. 2.5, Eq. poisson)
  with optional deconvolution by the squared kernel (Sec. 2.5, Table 1),
  the NUFFT force (ES kernel on an upsampled grid), interlacing, and the
  binned power spectrum.
* ``nbody``      - Zel'dovich and 2LPT initial conditions (Sec. 2.2, Eqs. LPT,
  helmholtz, LPT_L_and_T), the DKD stepper (Eq. dkd), full runs, the
  adjoint method (Sec. 2.7, Table 5, App. C) and its forward-mode counterpart
  (tangents of the run and of P(k)).

Readings of places where the paper is silent, ambiguous or garbled are stated
in the docstring of the function that takes them.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (no function is unpinned).
"""
