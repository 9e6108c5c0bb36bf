"""B300-native GMCP contact pass (Geometric Mortar Contact Potential, IsaacIPC).

The compute path lives in the CUDA library ``libgmcp.so`` (C ABI declared in
``include/gmcp.h``); :mod:`.binding` marshals arguments to it.  Importing the
package does not load the library: ``binding.lib()`` does, and raises if the
library has not been built.
"""
__all__ = ["scenes", "binding"]
