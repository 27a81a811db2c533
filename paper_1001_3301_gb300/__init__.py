"""GB300-native frequency-dependent first-order stellar irradiation ray tracer
(Kuiper et al. 2010, Sects. 2.2-2.3 and 3.3.4).

``Tracer`` wraps the C ABI of ``_build/librt_gb300.so`` (include/rt_irradiation.h).
Importing ``Tracer`` loads the CUDA library and raises if it is not built; there is
no CPU path. ``build()`` compiles it with nvcc for sm_103a.
"""
from __future__ import annotations

from .build import build  # noqa: F401

_LAZY = ("Tracer", "Batch", "Energy", "probe_ex2", "probe_alu_rates", "probe_tanh", "probe_umma",
         "probe_tensor_rates")
__all__ = ["build", "RtError", *_LAZY]


def __getattr__(name):
    if name == "RtError":
        from ._lib import RtError
        return RtError
    if name in _LAZY:
        from . import tracer
        return getattr(tracer, name)
    raise AttributeError(name)
