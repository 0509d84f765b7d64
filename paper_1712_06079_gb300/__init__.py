"""GB300-native D2Q9 pseudopotential lattice Boltzmann step with the
high-order-difference (HDM) interaction force (Qin et al., arXiv:1712.06079).

The step runs in hand-written CUDA kernels for sm_103a inside ``liblbm.so``
(a C-ABI library, ``include/lbm.h``).  This package is the thin Python binding
over it: ``lbm`` (ctypes marshalling of the C entry points), ``inputs``
(seeded synthetic density fields).  Importing the package does not load the
CUDA library; the first use of ``lbm`` does, and raises if it is missing.
"""

__all__ = ["lbm", "inputs"]
