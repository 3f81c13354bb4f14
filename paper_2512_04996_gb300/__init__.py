"""GB300 (sm_103a) implementation of the data-parallel hot path of
dilation-based ICP with per-voxel dynamic memory assignment (arXiv 2512.04996).

* ``paper_2512_04996_gb300.vicp``  -- Python binding of the C ABI (include/vicp.h)
* ``paper_2512_04996_gb300.build`` -- builds ``_build/libvicp.so`` with nvcc
* ``paper_2512_04996_gb300.synth`` -- seeded synthetic workloads (inputs only)

Importing the package does not import torch or load the CUDA library; the
binding loads ``libvicp.so`` on first use and raises if it is missing.
"""
__all__ = ["vicp", "build", "synth"]
