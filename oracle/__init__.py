"""CPU oracle for the HIF-IE hot path (Ho & Ying, "Hierarchical Interpolative
Factorization for Elliptic Operators: Integral Equations").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The GPU library never calls it, and it shares no code with the GPU path:
the two meet only at the seeded input generators in ``hif_inputs``.

Everything is plain, slow FP64 numpy written from the paper:

* ``kernels``  -- the discretized operator A = diag(a) + diag(b) K diag(c)
  (Sec. 1 Eq. (1.1), Sec. 3.1 Eq. (3.1) with one-point off-diagonal quadrature
  and the exact self-cell integral on the diagonal), dense assembly and the
  direct-sum matvec.
* ``idqr``     -- interpolative decomposition by column-pivoted Householder QR
  (Sec. 2.2, Lemma 2.2, adaptive rank), and the 2-norm estimate used for the
  second-kind tolerance rho (Sec. 4.4).
* ``hifie``    -- sequential HIF-IE in 2D/3D (Algorithms 4.1 and 4.2,
  skeletonization Lemma 2.4, proxy compression Sec. 3.3 / 4.3, second-kind
  modifications Sec. 4.4) with apply / solve / transposes in factored form
  (Eqs. (4.1), (4.2)).
* ``krylov``   -- right-preconditioned restarted GMRES (Sec. 5) and the power
  iteration error estimates e_a, e_s (Sec. 5).
* ``dense``    -- dense FP64 LU solve, the ground truth for small N.
* ``helmholtz`` -- the Helmholtz / Lippmann-Schwinger operator of Sec. 5
  Example 3 and its real 2 x 2 embedding, on which ``hifie`` runs unchanged.

Every function is pinned by tests/test_oracle_pins*.py (closed forms,
invariants, brute force, library routines), and tests/test_oracle_mutations.py
plants mistakes that those pins must catch.  Parity unpinned: the factor
values of single boxes (T, X, Y, L, U), which a rank decision within rounding
of its threshold changes; they are compared only through the accuracy of F
and F^{-1}.
"""
from . import kernels, idqr, hifie, krylov, dense  # noqa: F401
