"""B300 (sm_103a) LO-AFQMC local-energy library: Python side.

``synth`` draws seeded synthetic inputs; ``lo_afqmc`` binds the C ABI of the
CUDA library (``liblo_afqmc.so``) with ctypes.  Importing the package does not
load the CUDA library; the first call into ``lo_afqmc`` does, and raises if it
is missing.
"""
