"""GB300-native overset grid assembly (donor search) and boundary interpolation.

The compute path is libovs (hand-written sm_103a CUDA behind the C ABI of ``include/ovs.h``); this package
holds its sources (``csrc/``), its build script and the thin ctypes binding (``ovs``).
"""
from . import ovs  # noqa: F401
from .ovs import Context, load  # noqa: F401
