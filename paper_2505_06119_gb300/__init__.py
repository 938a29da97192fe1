"""GB300-native matrix-product-state two-site gate engine.

The compute path is the CUDA library built from csrc/ (C ABI in include/mps.h);
this package holds only its build script and a ctypes binding.  Importing the
package does not load the library; ``MPS(...)`` does, and raises ImportError
if it has not been built.
"""

from ._lib import load as load_library  # noqa: F401
from .mps import MPS, MPSError, config  # noqa: F401
