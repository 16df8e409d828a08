"""B300-native Image-GS rasteriser: tile-binned differentiable rendering of
colored anisotropic 2D Gaussians (forward, adjoint, fit step) in hand-written
CUDA for sm_103a, behind the C-ABI library `libimgs.so`.

The CUDA library is loaded on first use by `paper_2407_01866_b300.lib`; there is
no CPU fallback, and a missing or unloadable library raises.
"""
__all__ = ["lib", "synth"]
