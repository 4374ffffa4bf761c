"""GB300-native skeletal animation: the fused Simulation -> Hierarchy-Scan ->
Bind MeshPose frame of arXiv 2505.06703 as sm_103a CUDA kernels behind a C
ABI (include/anim.h), with an adjoint kernel and batched IK.

The Python layer only marshals arguments (see anim.py); the CUDA library is
built in-tree by _build.build()."""
from .anim import (AnimError, Context, IK, Plan, analyze_skeleton, hierarchy_fn, lib_path, load)

__all__ = ["AnimError", "Context", "IK", "Plan", "analyze_skeleton", "hierarchy_fn", "lib_path", "load"]
