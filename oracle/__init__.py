"""FP64 CPU oracle for the stochastic-delta-N first-passage sampler.

TEST INFRASTRUCTURE ONLY. This package is the independent reference that the
CUDA library is checked against. Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the product package never does,
and it shares no code with the product package.
"""
