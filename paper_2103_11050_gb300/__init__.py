"""GB300-native MRCM / MPM-2P pressure-update hot path (arXiv 2103.11050).

The compute path is a C-ABI CUDA library (``csrc/``, header ``include/mpm2p.h``);
``binding`` marshals arguments to it through ctypes.
"""
