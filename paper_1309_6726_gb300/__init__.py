"""GB300-native reactive two-component lattice Boltzmann (arXiv:1309.6726).

The compute path lives in the CUDA library under ``csrc/`` and is reached
through the C-ABI declared in ``include/lbm.h``; :mod:`.lbm` is its thin
Python binding and :mod:`.inputs` builds seeded synthetic geometries.
Nothing is imported eagerly so that :mod:`.inputs` stays usable on hosts
without the compiled library.
"""

__all__ = ["inputs", "lbm"]
