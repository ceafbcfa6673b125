"""GB300-native (sm_103a) StopThePop hierarchical sorted Gaussian splatting.

The renderer lives in a C-ABI CUDA library (libstp.so, declared in include/stp.h); this
package holds its thin Python binding and the seeded synthetic input generators.
"""
