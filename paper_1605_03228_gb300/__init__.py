"""GB300-native element-parallel iHDG sweep (libihdg) and its Python binding.

The compute path is the CUDA library under csrc/ (built for sm_103a by build.py); the
binding in ihdg.py only marshals arguments.  See include/ihdg.h for the C ABI.
"""
