"""GB300 (sm_103a) implementation of the five-equation WENO5 / HLLC / TVD-RK3
finite-volume hot path of arXiv 2503.07953 (MFC 5.0).

``mfc`` is the binding of the C ABI (include/mfc.h); ``workloads`` defines
the seeded synthetic inputs; ``build`` compiles the CUDA library in-tree.
"""
__all__ = ["mfc", "workloads", "build"]
