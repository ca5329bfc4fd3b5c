"""FP64 CPU oracle for the KRP sketch, randomized Tucker and block-Hankel path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import or call anything here.
The CUDA library never imports, links or executes it, and this package imports
nothing from the library: the two share no code.  Inputs reach both sides from
the seeded generators in ``synth/``.

Every routine is the plain definition (or the paper's algorithm in the paper's
order), in float64, written for a reader to check against the paper by eye:
Khatri-Rao products are formed explicitly, unfoldings are explicit matrices,
sketches are unfolding-times-KRP matrix products.  numpy's matmul/QR/SVD appear
only as library steps.

Modules
  philox   Philox4x32-10 counter-based generator + Box-Muller (Def. of KRP, Sec. 2.5)
  tensor   Kronecker / Khatri-Rao products, unfoldings, TTM, MTTKRP (Sec. 2.1)
  linalg   Householder thin QR, one-sided Jacobi SVD, least squares (Sec. 2.2)
  tucker   HOSVD/ST-HOSVD (Alg. 4, 5), RHOSVD-KRP (Alg. 7) and its memoized
           variant, RSTHOSVD-KRP (Alg. 8), core truncation, residual (Sec. 5)
  hankel   block-Hankel matrices and the single-pass block-structured
           randomized SVD (Alg. 6, Sec. 4)
  quant    FP8 E4M3 storage of X with one scale per slab of the slowest mode
           (a storage option for the sketch; the paper uses one precision)

Parity pins live in tests/test_oracle_*.py.  Functions without an independent
pin are marked "parity unpinned" in their docstring; currently: none.
"""
