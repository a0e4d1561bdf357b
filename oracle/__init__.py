"""FP64 CPU oracle for coded block Gram-Schmidt QR (test infrastructure only).

Loaded only by the tests, the smoke check and the benchmark's CPU-baseline leg.  It
shares no code with the CUDA library and never imports it.
"""
