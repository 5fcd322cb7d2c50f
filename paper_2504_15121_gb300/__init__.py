"""GB300-native stereo surface-normal estimation (arXiv 2504.15121).

The compute path is libsn.so: hand-written sm_103a CUDA kernels behind the C
ABI declared in include/sn.h.  `sn` is its ctypes binding (argument
marshalling only); `pipeline` adds frame-level conveniences on top of it.
"""
from . import sn  # noqa: F401  (raises ImportError if the library is not built)
from .sn import *  # noqa: F401,F403
from .pipeline import Pipeline, FrameBuffers  # noqa: F401
