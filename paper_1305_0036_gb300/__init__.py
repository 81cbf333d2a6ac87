"""GB300-native fourth-order Trotter-Suzuki (TS4) solver for spin-1/2 XYZ dynamics.

The compute path is the CUDA library ``libts4.so`` built from ``csrc/`` for
sm_103a, reached through its C ABI (``include/ts4.h``).  ``ts4`` is the thin
ctypes binding (argument marshalling only); importing it loads the library and
raises if it is missing -- there is no CPU fallback.  ``workloads`` holds the
seeded synthetic inputs.
"""
__all__ = ["ts4", "workloads", "build"]
