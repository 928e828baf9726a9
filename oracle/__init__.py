"""Plain FP64 CPU oracle of the SD MHD+GLM hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product package.
"""
