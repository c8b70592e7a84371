"""GB300-native FDK hot path of iFDK (Chen et al., SC'19, arXiv 1909.02724).

The computation lives in a C-ABI CUDA library (``csrc/``, declared in
``include/ifdk.h``); ``binding`` is a thin ctypes layer with the same names and
``autograd`` wraps the operators as ``torch.autograd.Function``s.
"""
from .geometry import Geometry, circular, gups  # noqa: F401
