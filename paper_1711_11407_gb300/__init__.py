"""FPS-SFT (arXiv 1711.11407) recovery loop for GB300: CUDA kernels behind a C ABI, with a thin
PyTorch-facing binding.  The compute path lives in csrc/ (libfpssft.so); this package only
marshals arguments."""
from . import _lib
from ._lib import FpssftError, build, load

__all__ = ["FpssftError", "build", "load", "Params", "Plan", "RecoverOutput"]


def __getattr__(name):  # torch is imported lazily: the generators need only numpy
    if name in ("Params", "Plan", "RecoverOutput"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
