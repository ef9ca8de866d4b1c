"""FP64 CPU oracle for the BOA Constrictor hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU baseline leg are the only callers.  Nothing in the product
path imports this package.
"""
