"""FP64 CPU oracle of the DI-LBM hot path.

Test infrastructure only: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark; never by the product path.
"""
