"""FP64 CPU oracle of the SediFoam particle-side hot path (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg load this
package; the CUDA library never does.
"""
