"""GB300-native (sm_103a) MPDO noisy-circuit update with tomography (chi-matrix) channels.

The compute path is the C-ABI library built from csrc/ (declared in include/mpdo.h);
`paper_2508_07610_gb300.mpdo` is a thin ctypes binding over it.
"""
