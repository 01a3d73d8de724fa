"""GB300-native quantized feature-correspondence scoring (QFCA hot path).

The compute path lives in the C-ABI library ``libqfca.so`` (hand-written
sm_103a CUDA kernels); :mod:`paper_2510_15602_gb300.qfca` is the thin Python
binding over it.  Importing this package does not load the library: import
``paper_2510_15602_gb300.qfca`` (or call :func:`load`) for that, which raises
when the library has not been built.
"""

__all__ = ["load"]


def load():
    """Import and return the binding module (loads ``libqfca.so``)."""
    from . import qfca

    return qfca
