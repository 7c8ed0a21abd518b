"""GB300-native FE-LBM contact-line step (arXiv:1708.04678, 2D D2Q9 form).

The compute path is the C-ABI CUDA library ``libfelbm.so`` (built by
``paper_1708_04678_gb300.build``); ``paper_1708_04678_gb300.felbm`` is its thin
ctypes binding.  ``inputs`` holds the seeded synthetic workloads.
"""
__all__ = ["inputs", "felbm", "build"]
