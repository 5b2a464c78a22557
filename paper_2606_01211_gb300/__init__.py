"""GB300-native (sm_103a) plain-LWE KEM hot path.

The compute lives in liblwe.so (C ABI in include/lwe.h, CUDA sources in
csrc/); `lwe` is its Python binding.  Importing the binding requires the
built library and raises otherwise.
"""
