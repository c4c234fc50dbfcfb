"""GB300 batched polar SCL decoder: libpolarscl (CUDA, sm_103a) and its binding."""
from . import polarscl  # noqa: F401
from .polarscl import Code, pruning  # noqa: F401
