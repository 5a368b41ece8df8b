"""GB300-native count-and-emit frequency sort (CAFS) for int32/int64 columns.

The compute path is the CUDA library ``libcafs.so`` built from ``csrc/`` for
sm_103a; ``cafs`` is its thin ctypes binding.  Importing this package does not
load the library: the first call into ``cafs`` does, and fails loudly when the
library has not been built.
"""

__all__ = ["cafs", "datagen", "build"]
