"""B300-native (sm_103a) OpenSBLI residual / RK-stage path.

The compute path lives in ``libosbli.so`` (CUDA kernels behind the C ABI declared in
``include/osbli.h``); ``solver`` is its thin ctypes binding and ``inputs`` holds the seeded /
analytic problem set-ups.  Importing the package loads nothing; ``solver.load()`` loads the
library and raises if it is missing.
"""
