"""B300-native (sm_103a) Multi-Scale Non-Linear Fusion and ptychographic reconstruction.

The compute path is a C-ABI CUDA library (``libptycho_mnf.so``); ``paper_2608_01746_b300.api``
is its thin ctypes binding.  Importing this package loads nothing; import ``.api`` to load the
library (it raises if the library has not been built).
"""
