"""Coded block Gram-Schmidt QR on one GB300 (arXiv 2311.11943), sm_103a CUDA kernels
behind a C-ABI library.  Import is light: the shared library is loaded on first use by
`paper_2311_11943_gb300.binding`."""
__all__ = ["binding", "synth"]
