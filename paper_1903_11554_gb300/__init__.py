"""GB300 TT-cross quadrature (arXiv:1903.11554): CUDA kernels behind a C ABI
(include/ttq.h, libttq.so) and a thin ctypes binding."""
from . import inputs  # noqa: F401
