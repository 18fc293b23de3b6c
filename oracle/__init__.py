"""CPU oracle for ESG range-filtered k-NN search (arxiv 2504.04018).

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct float64
implementation of what the GPU library computes, used to check it. Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the GPU library
(``paper_2504_04018_gb300``) and never imports it; both consume the seeded
inputs of ``synthetic.py``.

Parts and what pins them (see tests/test_oracle.py):
  - re-ranking (Section 1 footnote): a permutation check against numpy's
    stable sort;
  - elastic decomposition (Algorithm 4, Lemma 3): exhaustive enumeration of
    all ranges for small N against the partition / containment / elastic-ratio
    invariants and an independent closed form (the LCA construction);
  - exact range-filtered k-NN (Definitions 1-2): brute force against
    hand-computed tiny cases and numpy argsort;
  - graph search (Algorithm 1, POST principle): hand-traced golden fixtures,
    exactness when ef covers the graph, in-range results;
  - index build (Algorithm 3): a hand-traced build of 8 points (every row of
    every depth, every node's entries), which mutants of this C source with a
    planted mistake fail, and structural invariants (degree, no self loops, ids
    inside the node, reachability). Graph quality versus the paper's is parity
    unpinned (no datasets are available);
  - learned-budget network (mlp.py): hand-computed forward outputs and three
    Adam steps, finite-difference gradients, the pinball loss's quantile;
  - recall: a hand case with duplicates and an empty truth set.
"""
from .esg_oracle import *  # noqa: F401,F403
