"""GB300-native exact subgraph matching (gMatch-style fine-grained search).

The engine is libsgm.so, a CUDA library for sm_103a with the C ABI declared
in include/sgm.h; `sgm` is its Python binding. PyTorch is used only for
device memory and streams.
"""
from . import sgm  # noqa: F401
from .sgm import Engine, SgmError  # noqa: F401
