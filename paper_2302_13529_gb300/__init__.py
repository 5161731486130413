"""GB300 (sm_103a) implementation of the sampled-dominator-tree estimator and the
AdvancedGreedy / GreedyReplace blocker-selection drivers of arXiv 2302.13529.

Submodules:
  build      compiles the CUDA C-ABI library (libimin.so) in-tree
  imin       Python binding of include/imin.h (loads libimin.so; no CPU fallback)
  workloads  seeded synthetic graphs, thresholds and seed sets
"""
