"""GB300-native (sm_103a) RNS-CKKS hybrid key switching.

The compute lives in the CUDA library libfhe_gb300.so (C ABI: include/fhe.h);
`binding` is its ctypes binding, `build` compiles it in-tree, `inputs` holds
the seeded synthetic input generators and `roofline` the key-switching byte
model used to report L2-roofline fractions.
"""
__all__ = ["binding", "build", "inputs", "roofline"]
