"""GB300-native volumetric Fourier-transform reconstruction (Sec. III of arXiv 1712.03084).

The reconstruction runs in the CUDA kernels of ``lib/libftr.so`` (sources in
``csrc/``, C ABI in ``include/ftr.h``); ``ftr`` is its Python binding and
``build`` compiles it for sm_103a.
"""

from . import ftr  # noqa: F401
from .ftr import Context, FtrError  # noqa: F401
