"""B300-native recursive-Green's-function transmission library.

The compute path is the CUDA shared library ``librgf.so`` (C ABI in
``include/rgf.h``); ``rgf`` is its thin ctypes binding.
"""
from .rgf import *  # noqa: F401,F403
from .rgf import Plan, RGFError, lib  # noqa: F401
