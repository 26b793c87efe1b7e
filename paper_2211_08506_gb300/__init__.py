"""GB300-native batched Gaussian-density voxelization (ParticleGrid, arXiv 2211.08506).

The computation lives in libpg.so (hand-written CUDA for sm_103a behind the C ABI of
include/pg.h); ``binding`` is its ctypes mirror and ``api`` the PyTorch-facing layer.
"""
from ._build import build, LIB_PATH  # noqa: F401


def __getattr__(name):
    # The torch-facing API is imported lazily so that building needs no GPU and no torch.
    if name in ("api", "binding"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    from . import api
    return getattr(api, name)
