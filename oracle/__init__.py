"""CPU oracle for the forest-closeness hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatements of what the method computes,
written from the paper (van der Grinten, Angriman, Predari, Meyerhenke, "New
Approximation Algorithms for Forest Closeness Centrality", arXiv 2101.06192):

  dense.py        Omega = (alpha L + I)^{-1}, forest distance (Def. 1), farness
                  (Def. 2 and Eq. 3), closeness, ranking, Algorithm 1's tau/eta,
                  pivot solve and fill step.
  wilson_oracle.c sequential Wilson sampler on G* (Algorithm 2) with Philox
                  random stacks; R counts (Prop. 1), control-variate counts.
  native.py       ctypes loader for the C file.
  enumerate.py    brute-force spanning trees of G* (matrix-forest theorem).
  cg.py           FP64 CG ground truth (Sec. 6.1).
  cv.py           control-variate combination (not in the paper).
  mlp.py          FP64 forward/backward/Adam of the control-variate network.
  electrical.py   electrical closeness on G (Sec. 3, Eq. 2): L^+, effective
                  resistance, the UST path-sum estimator along a BFS tree.
  wilson_oracle.c also: Wilson on G rooted at a vertex (Sec. 3 insight (iii)).
  forest.py       forest roots and depths of sampled trees (Sec. 2, the
                  matrix-forest theorem's rooted forests).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
Every function is pinned by ``tests/test_oracle_*.py`` against facts the paper
and the mathematics fix (closed forms, brute force, invariants, library
routines); see the pins listed there.
"""
from . import cg, cv, dense, electrical, enumerate, forest, mlp, native  # noqa: F401
