"""GB300-native solid voxelization of tetrahedral meshes (arXiv 2106.01326).

The compute path is a C-ABI CUDA library (``libvoxtet.so``, sm_103a) reached
through the thin ctypes binding in ``voxtet``; PyTorch supplies device memory
and streams only.  Importing this package does not load the library; the first
call that needs it does, and fails loudly if it is missing.
"""

__all__ = ["meshgen"]
