"""GB300-native EOFA Dirac-equation solver (arXiv:1706.05843).

The product is ``libeofa.so`` (CUDA, sm_103a) behind the C ABI of
``include/eofa.h``; ``binding`` is its thin ctypes wrapper and ``inputs``
draws the seeded synthetic gauge fields and right-hand sides.  Importing
this package loads nothing: ``binding.lib()`` loads the library on first use
and raises if it has not been built (``build.build()``).
"""
