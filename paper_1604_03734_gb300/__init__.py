"""GB300-native hot path of DENSER Cities: hashing voxel grid allocation, projective
TSDF fusion and Omega-aware primal-dual TV regularisation, as hand-written sm_103a
CUDA behind the C ABI of include/denser.h.

``paper_1604_03734_gb300.native`` binds that ABI; ``paper_1604_03734_gb300.build``
compiles it.  Importing the package loads nothing.
"""

__all__ = ["native", "build"]
