"""GB300-native encrypted FFConv layer (arXiv 2102.03494): RNS-BFV on one GPU.

The compute path is the CUDA library libhe.so (C ABI in include/he.h) built from csrc/ by
build_ext.build(); `he` is its thin Python binding.  Import submodules explicitly:
    from paper_2102_03494_gb300 import he, workloads
"""
__all__ = ["he", "workloads", "build_ext"]
