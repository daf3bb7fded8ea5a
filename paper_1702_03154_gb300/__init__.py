"""GB300-native (sm_103a) cascading-bit-array minimal perfect hash function.

The compute path is the CUDA library ``libmphf.so`` (``csrc/``) behind the C
ABI declared in ``include/mphf.h``; ``paper_1702_03154_gb300.mphf`` is a thin
ctypes binding with the same names.  Importing this package loads nothing; the
first call into the binding loads the library and fails loudly if it is
missing.
"""

__all__ = ["mphf", "inputs"]
