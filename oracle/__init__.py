"""FP64 CPU oracle: TEST INFRASTRUCTURE ONLY.

A plain, slow, step-by-step restatement of the method of "Model reduction for
the material point method via an implicit neural representation of the
deformation map" (Chen, Chiaramonte, Grinspun, Carlberg): the explicit MPM
step (Algorithm 1), the implicit neural decoder and its Jacobians (Eqs. for
the deformation gradient and the velocity of the manifold, Section 3.1), the
training loss (Section 4.2), the reduced-order step (Algorithms 2, 3, 5, 6, 7)
and the accumulated position error (Section 5).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2109_12390_gb300``) never imports it and shares no code
with it: the two meet only in the seeded input generators of ``synth``.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or textbook library routines;
see each module's header for the list.
"""
