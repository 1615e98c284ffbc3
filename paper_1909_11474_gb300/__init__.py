"""GB300-native (sm_103a) evaluation of the minimal Tersoff potential of arXiv:1909.11474.

The compute path lives in the CUDA shared library built from csrc/ (C-ABI declared in
include/tersoff.h); `paper_1909_11474_gb300.binding` is the thin Python marshalling layer over it.
Importing this package loads nothing: the library is opened on first use of the binding.
"""
