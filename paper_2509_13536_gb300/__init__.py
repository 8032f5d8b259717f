"""GB300-native splatting + voxel-merge hot path of MemGS (arXiv 2509.13536).

The compute lives in libmemgs.so (hand-written sm_103a CUDA behind include/memgs.h).
``api`` marshals torch tensors into that C ABI; ``scenegen`` holds the seeded
synthetic inputs; ``build`` compiles the library in-tree.
"""
__all__ = ["api", "build", "scenegen"]
