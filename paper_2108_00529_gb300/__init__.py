"""GB300-native BigGraphVis hot path (arXiv 2108.00529).

``libbgv.so`` (CUDA kernels for sm_103a behind the C ABI in
``include/bgv.h``) computes the degree count-min sketch, the streaming
community rounds, the supergraph and the ForceAtlas2 layout.  ``bgv`` is its
ctypes binding; ``build`` compiles it in-tree with nvcc.
"""
from . import build  # noqa: F401

__all__ = ["build", "load"]


def load():
    """Import the binding (raises ImportError if libbgv.so is missing)."""
    from . import bgv
    return bgv
