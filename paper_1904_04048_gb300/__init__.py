"""GB300-native explicit time marching of the 2D wave equation with the
5-, 9- and 13-point schemes generated by Poisson's formula (arXiv:1904.04048).

The compute path is the CUDA library ``libwave2d.so`` (sources in ``csrc/``,
C ABI in ``include/wave2d.h``); ``wave2d`` is its ctypes binding.
"""
from .wave2d import (  # noqa: F401
    Wave2D, Wave2DError, exact, lambda_max, launch_count, lib, use_default_allocator,
    use_torch_allocator,
)
