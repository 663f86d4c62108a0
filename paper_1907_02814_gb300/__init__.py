"""GB300-native pairwise Coulomb-process collision step (arXiv:1907.02814).

The compute path is the CUDA library ``libpcc.so`` behind the C ABI in
``include/pcc.h``; ``paper_1907_02814_gb300.pcc`` is its thin ctypes binding.
"""
__all__ = ["pcc", "workloads"]
