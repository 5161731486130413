"""CPU oracle for the sampled-dominator-tree estimator (test infrastructure only).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this package.
"""
