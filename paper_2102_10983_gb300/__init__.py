"""GB300-native adaptive electron sub-cycling particle integrator (arXiv 2102.10983).

The hot path (criterion, temporal Lagrange interpolation, tent gather, Boris
push, position update) runs in hand-written CUDA kernels for sm_103a behind the
C ABI declared in include/pic_gb300.h.  ``paper_2102_10983_gb300.native`` is the
thin Python binding of that ABI; ``workloads`` holds the seeded input generators.
"""
__all__ = ["native", "workloads"]
