"""FP64 CPU oracle for the AB-/BA-GKB reconstruction path -- TEST INFRASTRUCTURE.

Plain, slow, obviously correct implementations of what the CUDA path
computes, written from the paper (Algorithms 3-5, Eqs. 16-18, Sec. 4 and 5):

* ``projectors`` -- Joseph forward projector A, pixel-driven back projector
  B, and the exact transposes A^T and B^T (plain C loops, FP64).
* ``dense``      -- the same operators as explicit matrices built from their
  closed forms, for tiny grids (an independent second route used as a pin).
* ``gkb``        -- the GKB recurrences of Algorithms 3 (matched), 4 (AB)
  and 5 (BA), step by step, with the one-sided reorthogonalisation of step
  9, the projected problem of Eq. (proj GKB) solved by the SVD of C_k, and
  the discrepancy principle / residual-norm stagnation stopping rules.
* ``mlp``        -- the learned stopping predictor's forward, backward and
  Adam step in FP64.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.
"""
