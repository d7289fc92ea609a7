"""B300-native (sm_103a) nodal-DG large-eddy-simulation hot path.

The compute path lives in the CUDA library libcmles.so (C ABI in
include/cmles.h); `cmles` is its thin Python binding (argument marshalling
only, torch tensors for device memory and streams) and `inputs` holds the
seeded synthetic workload descriptions.  Importing the package does not load
the library; creating a solver does, and fails loudly when it is missing.
"""
__all__ = ["cmles", "inputs"]
