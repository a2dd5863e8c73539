"""Plain FP64 CPU oracle of the HODLR maximum-likelihood hot path.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference against which
the CUDA library is checked.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import it; the product path
(``paper_2303_10102_gb300``) never does, and it shares no code with it.

Contents (each function cites the passage of arXiv 2303.10102 it follows):
  tree.py        ordering (KD / Morton) and the cluster tree of index sets    (Sec. 5.2; Sec. 3.2.2)
  philox.py      Philox4x32-10 counter-based Gaussian probes                  (Alg. 1 step 1)
  physics.py     K(theta) = L K_u L^T + tau2 I and its parameter derivatives   (eq. cov model; eq. whittle covariance)
  hodlr.py       matrix-free randomized HODLR construction with peeling and
                 the differentiated construction                               (Alg. 1; Sec. 3.2.2; Alg. 2; Sec. 3.3)
  likelihood.py  NLL, score and Fisher information by their plain dense
                 definitions applied to the densified HODLR matrices          (eq. log-like; eq. score; eq. fisher info)
  scoring.py     Fisher-scoring outer loop                                     (Sec. 2.2, eq. CLT)

The hierarchical factorization and the trace operations of App. B/C compute their
results exactly (up to rounding), so the oracle states them by their plain
definitions (dense Cholesky, dense solves, dense traces) on the densified matrices.
The construction is an approximation, so it is followed step by step.

Parity unpinned (readings with no number in the paper to pin them): the adaptive
rank rule, the rank guard, leaf symmetrization, the oversampling use, the Matern
length-scale convention.
"""
