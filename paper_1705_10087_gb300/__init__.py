"""GB300-native segmented locally greedy convolutional sparse coding (DICOD hot path).

Submodules (imported on demand, so that importing the package loads nothing):
  capi    ctypes binding of the C ABI in include/csc.h (libcsc.so)
  build   nvcc build of libcsc.so for sm_103a
  synth   seeded synthetic problems (inputs only)
"""
