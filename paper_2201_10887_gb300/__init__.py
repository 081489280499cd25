"""GB300-native adaptive-heightfield rendering with RBF discretization and
max-mipmap ray casting (Cornel, Horvath, Waser, 2022).

``hf`` is the ctypes binding of the C ABI (include/hf.h); ``Renderer``
owns the device buffers of one heightfield.  Importing the package loads
``libhf.so`` and fails if it has not been built.
"""

from . import hf
from .renderer import Renderer, camera_struct
from .batch import Batch, autotune
from .serving import Arena, Server

__all__ = ["hf", "Renderer", "camera_struct", "Batch", "autotune", "Arena", "Server"]
