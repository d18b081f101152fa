"""GB300 fast random-walk Kalman filter (hierarchical-matrix covariance,
low-rank perturbative update).  The compute path is the CUDA library
libfkf.so behind the C-ABI in include/fkf.h; `fkf` is its ctypes binding."""

from .builder import build  # noqa: F401


def load():
    """Import the binding (raises ImportError if libfkf.so is not built)."""
    from . import fkf

    return fkf
