"""Plain, slow FP64 CPU oracle for the Tucker-compressed coupling-matrix products.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs
may call it.  It shares no code with the CUDA library; both sides take their
inputs from paper_2103_06393_gb300.inputs.

Every function follows the paper (Giannakopoulos et al., "Compression of
volume-surface integral equation matrices via Tucker decomposition for magnetic
resonance applications", arXiv 2103.06393) and cites the equation, algorithm or
table it restates.  Computation is complex128 throughout.

Modules
  greens      dyadic Green's function and column assembly      (Eq. n6, Eq. nNt, Sec. III.A)
  tucker      truncated HOSVD, n-mode products, element eval   (Eq. Tucker, Sec. II.B.1)
  products    Algorithms 1 and 2, plus their ACA wrappers      (Sec. III.B, Table III)
  aca         partially pivoted ACA and Algorithm 3            (Sec. II.B.2, Sec. III.C)
  memory      storage model of Table II
  randomized  randomized range-finder Tucker (parity unpinned against the paper:
              the paper has no randomized variant; pinned by planted-rank tests)
  mlp         rank-predictor MLP forward/backward (no counterpart in the paper;
              pinned by finite differences)
"""
