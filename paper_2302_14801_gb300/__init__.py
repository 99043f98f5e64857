"""GB300-native LOD construction for point clouds.

Builds the hybrid voxel-point octree of "GPU-Accelerated LOD Generation for
Point Clouds" (Schuetz et al. 2023) with hand-written sm_103a CUDA kernels
behind the C ABI declared in include/lod.h.  ``paper_2302_14801_gb300.lod``
is the thin binding; ``paper_2302_14801_gb300.synth`` draws seeded inputs.
"""

__all__ = ["synth", "lod"]
