"""Balanced 3DGS render path for GB300 (sm_103a): C-ABI library + thin Python binding.

Importing the package does not load the CUDA library; ``paper_2412_17378_gb300.raster``
does, and raises if it is missing.
"""
