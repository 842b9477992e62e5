"""GB300 (sm_103a) particle hot path of the particle-in-cell method of
Gassmoeller, Heien, Puckett & Bangerth (arXiv 1612.03369).

  paper_1612_03369_gb300.pic        ctypes binding of libpic.so (include/pic.h)
  paper_1612_03369_gb300.workloads  seeded synthetic inputs (meshes, fields)
  paper_1612_03369_gb300.build      in-tree nvcc build of libpic.so

Importing the package itself loads nothing; `from paper_1612_03369_gb300
import pic` loads the CUDA library and raises if it is missing.
"""

__all__ = ["pic", "workloads", "build"]
