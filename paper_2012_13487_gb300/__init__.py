"""GB300-native finite element discrete Boltzmann solver (isothermal BGK).

The compute path is the CUDA shared library ``libfedbm.so`` (sources under
``csrc/``, C ABI declared in ``include/fedbm.h``); ``fedbm`` is its ctypes
binding.  Importing this package loads nothing; the library is loaded on
first use of ``paper_2012_13487_gb300.fedbm``.
"""
