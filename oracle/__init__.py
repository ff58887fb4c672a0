"""FP64 CPU oracle for the sparse-inverse local-global solve with frictional contact.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The CUDA
library never calls it and shares no code with it.

What it computes (Zeng et al., "Fast But Accurate: A Real-Time Hyperelastic Simulator with
Robust Frictional Contact"): one implicit-Euler frame (Eq. 1) solved by local-global
iterations (Eqs. 5-6, Alg. 1) constrained by Fischer-Burmeister complementarity functions
(Sec. 5.2, Eqs. 14-23; App. B.2, Eqs. 52-57) with split non-smooth indicators (Sec. 5.3,
Eqs. 24-26), the Delassus operator W = H A^-1 H^T (Eq. 27) and its diagonal as the
complementarity preconditioner (Sec. 5.4, Eq. 28), in the order of Alg. 4.

Where the method reaches a quantity with a plain definition, the oracle uses that
definition: the global step q = A^-1 b is a direct sparse solve of the full 3n x 3n system
(never the per-vertex Kronecker shortcut), W is H A^-1 H^T from direct solves. The sparse
inverse S = L^-1 itself (Theorem 1, Alg. 2) is built in ``sparse_inverse`` for small
matrices and pinned against the ancestor-closure theorem and dense inversion.

Modules:
  fem             rest-shape data, the deformation-gradient operator G, lumped masses,
                  weights and the system matrix A (Eq. 6), for tetrahedra and triangle
                  (membrane) elements, and the Laplace-Beltrami bending term
  local           per-element projections (Eq. 5) for ARAP, co-rotational and stable
                  Neo-Hookean energies; ARAP and co-rotational membranes
  contact         collision detection and linearisation (App. A.1), Fischer-Burmeister
                  functions and their derivatives (App. B.2), the minimum map (App. B.1),
                  anchors (bilateral constraints), contact between deformable bodies
                  (a vertex against another body's nearest surface triangle), conjugate
                  residual
  sparse_inverse  elimination tree, Cholesky factor and its inverse (Theorem 1, Alg. 2)
  integrator      the frame loop of Alg. 4, residual and energy diagnostics
  precision       BF16 storage of S and one residual correction (not from the paper)
  mlp             the learned warm start's network: forward, backward, loss (not from the
                  paper: a predictor of the initial contact impulses)
"""
from .integrator import Oracle, OracleOptions  # noqa: F401
