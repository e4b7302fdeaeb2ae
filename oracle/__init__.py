"""FP64 CPU oracle of the permittivity chain and its adjoint.

Test infrastructure only: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the library.
"""
