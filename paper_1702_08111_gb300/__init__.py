"""GB300-native two-level Method of Local Corrections (free-space Poisson).

The solver is the CUDA library behind include/mlc.h; ``paper_1702_08111_gb300.mlc``
is its Python binding and ``paper_1702_08111_gb300.inputs`` the seeded charge
generator.  Importing the package loads nothing on the GPU.
"""
__all__ = ["mlc", "inputs", "build"]
