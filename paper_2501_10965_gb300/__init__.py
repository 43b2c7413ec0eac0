"""GB300 (sm_103a) implementation of the data-parallel hot path of the DIG
method for rarefied polyatomic gas flow (arXiv 2501.10965).

``paper_2501_10965_gb300.dsmc`` is the Python binding of the C ABI in
``include/dig_dsmc.h``; ``workloads`` describes the synthetic cases.  Importing
the package does not load the CUDA library; ``dsmc.load()`` does, and fails
loudly when it is missing.
"""
__all__ = ["dsmc", "workloads", "build"]
