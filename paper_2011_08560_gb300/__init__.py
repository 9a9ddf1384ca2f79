"""GB300-native generalized-ensemble Monte Carlo for the 3D +-J Edwards-Anderson spin glass.

Multicanonical (flat, power-law, 1/k, canonical) and parallel-tempering sweeps run as
hand-written sm_103a kernels behind the C ABI of include/eamc.h; ``eamc`` is its ctypes
binding.  Reference: Mueller, Schnabel, Janke, arXiv:2011.08560.
"""
from . import eamc  # noqa: F401  (raises if the CUDA library is missing)
