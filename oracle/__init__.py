"""CPU FP64 oracle of the blockBP surface-code decoder (arXiv 2402.04834).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the C-ABI library and its Python binding)
never calls it and shares no code with it.

The oracle is a plain, slow, step-by-step restatement of the paper:

* ``lattice``  -- planar surface code, checks, logicals, syndrome map,
                  pure error f_s and the Monte-Carlo ground truth (Sec. II).
* ``tn``       -- the coset tensor network T_s(L) (Sec. III.A, Fig. 1).
* ``exact``    -- exact references: brute-force sum over the stabilizer
                  group (Eq. noise-cosets) and exact TN contraction.
* ``mps``      -- MPS compression by QR and truncated SVD (Sec. III.A),
                  overlaps and direct sums.
* ``blockbp``  -- Algorithm 1 with Remarks 1-8: partition, boundary-MPS block
                  update (Eq. BP-update on blocks), normalisation, damping,
                  chessboard schedule, convergence Delta, Bethe read-out
                  (Lemma 1) and the decision rule.
* ``naive``    -- the fused-block dense BP of Remark 9, an independent
                  second implementation used only to pin ``blockbp``.

Every function works in float64.  Parity status of each part is recorded in
the docstring of the module that holds it.
"""
