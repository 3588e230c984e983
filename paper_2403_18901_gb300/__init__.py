"""GB300-native sliding-window GDG decoder for bivariate-bicycle codes.

The compute path is the C-ABI library libqdec.so (CUDA, sm_103a); the Python
module `qdec` only marshals arguments into it.
"""
