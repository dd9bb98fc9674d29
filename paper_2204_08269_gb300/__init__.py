"""GB300-native joint time-frequency scattering (JTFS) forward and backward.

The transform of "Differentiable time-frequency scattering on GPU" (DAFx 2022) behind the C
ABI of ``include/jtfs.h`` (``libjtfs.so``, CUDA for sm_103a); this package is its thin
Python binding."""
from .jtfs import JTFS, JTFSError, JTFSFunction, JTFSPlan, exported_symbols, lib  # noqa: F401
