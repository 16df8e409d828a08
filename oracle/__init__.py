"""CPU oracle for the Image-GS rasteriser -- TEST INFRASTRUCTURE ONLY.

Only tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package. It shares no code with the CUDA path.
"""
from . import fp32, image_gs, placement, ssim  # noqa: F401
