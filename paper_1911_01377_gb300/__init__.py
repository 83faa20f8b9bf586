"""GB300-native u-series electrostatics (arXiv:1911.01377).

The evaluation runs in libusr.so (hand-written sm_103a CUDA behind the C ABI
of include/usr.h); `usr` is its Python binding and `workloads` the seeded
synthetic inputs.  Build with `paper_1911_01377_gb300.build.build()`.
"""
from . import usr  # noqa: F401
from .usr import USeries, UsrError  # noqa: F401
