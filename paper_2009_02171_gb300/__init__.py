"""GB300-native preconditioned Krylov solve of the cubed-sphere shell dynamo.

The compute path is the CUDA library ``libfv.so`` (C ABI declared in
``include/fv.h``); ``paper_2009_02171_gb300.fv`` is its thin ctypes binding.
``inputs`` holds the seeded synthetic input generators.
"""
