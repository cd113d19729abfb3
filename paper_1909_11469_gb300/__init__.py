"""GB300-native frontier-scheduled loopy belief propagation (LBP, RBP, RS, RnBP).

The compute path is a CUDA shared library (sm_103a) behind a C ABI declared in
include/bp_gb300.h; `paper_1909_11469_gb300.bp` is its thin ctypes binding.
"""
