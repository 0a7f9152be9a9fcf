"""GB300-native LBM-IB library (Coclite et al., arXiv:1903.03356).

The CUDA library and its ctypes binding live in ``paper_1903_03356_gb300.lbmib``;
importing the package itself loads nothing, so that ``workloads`` can be used alone.
"""
