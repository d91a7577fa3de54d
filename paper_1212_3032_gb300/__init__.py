"""GB300-native exponential-window frequency-domain elastodynamic BEM.

The compute path is the CUDA library ``libbem.so`` (sources in ``csrc/``,
C-ABI in ``include/bem.h``); ``binding`` is its thin Python binding and
``inputs`` the seeded synthetic input generators. Importing the package does
not load the library; ``binding.load_library()`` does, and raises if the
library has not been built.
"""
__all__ = ["binding", "build", "inputs"]
