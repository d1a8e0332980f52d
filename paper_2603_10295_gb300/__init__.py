"""GB300-native Wannier interpolation of electron-phonon matrix elements.

The compute path is the CUDA library libeph (sm_103a) behind the C-ABI in
include/eph.h; `binding` marshals numpy arrays / torch tensors to it, and
`synth` builds seeded synthetic inputs shaped like the paper's workloads.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "binding", "build_lib"]


def __getattr__(name):
    if name in ("binding", "build_lib"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
