"""GB300-native m-Cubes: the VEGAS sampling hot path (arXiv 2202.01753) in
hand-written CUDA for sm_103a behind a C ABI (include/mcubes.h).

``mcubes`` is the ctypes binding of that ABI; ``workloads`` draws the seeded
synthetic integrals; ``build`` compiles the library in-tree.  Importing the
package does not load the CUDA library; ``mcubes.lib()`` does, and fails
loudly if it is missing.
"""

__all__ = ["build", "mcubes", "workloads"]
