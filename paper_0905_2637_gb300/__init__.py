"""GB300 (sm_103a) fast multipole evaluation of the velocity of 2D Gaussian
vortex blobs (the PetFMM paper's vortex-method client, Sec. 3, evaluated by
the FMM of Sec. 2).

The compute lives in ``libpetfmm.so`` (CUDA, built in-tree by ``build.py``);
``_lib`` is its ctypes binding.  Importing this package does not load the
library: ``workloads`` (seeded input recipes) works without a GPU.
"""
from __future__ import annotations

__all__ = ["Context", "Server", "PetfmmError", "load", "build"]


def __getattr__(name):
    if name in ("Context", "Server", "PetfmmError", "load", "header_symbols") or name.startswith("petfmm_") \
            or name.startswith("PETFMM_"):
        from . import _lib
        return getattr(_lib, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
