"""B300-native (sm_103a) ADASAP hot path.

The compute path lives in the C-ABI shared library ``_lib/libadasap.so``
(sources in ``csrc/``, declarations in ``include/adasap.h``).  ``binding``
is the thin ctypes layer over it; ``synth`` draws the seeded workloads.
Importing this package loads nothing: ``from paper_2505_13723_b300 import
binding`` loads the library and fails loudly if it is missing.
"""

__all__ = ["binding", "synth", "build"]
