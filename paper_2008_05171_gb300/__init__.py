"""GB300-native k-medoids hot path: FastPAM1 / FastPAM2 / FasterPAM SWAP and
PAM BUILD (Schubert & Rousseeuw, arXiv 2008.05171) as sm_103a CUDA kernels
behind a C ABI (``include/kmedoids.h``).

The binding module ``kmedoids`` loads the in-tree ``libkmedoids.so`` on first
use and raises if it is missing; there is no CPU fallback.  ``workloads``
holds the seeded input generators.
"""
__all__ = ["kmedoids", "workloads"]
