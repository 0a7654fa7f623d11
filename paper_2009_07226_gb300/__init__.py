"""GB300-native memoized parallel-beam XCT projector and CGLS solver.

The compute path lives in the CUDA library ``libxct.so`` (sources under
``csrc/``, C-ABI declared in ``include/xct.h``); ``xct`` is its thin ctypes
binding.  ``inputs`` generates seeded synthetic data.  Importing this package
loads nothing; ``from paper_2009_07226_gb300 import xct`` loads the library.
"""
