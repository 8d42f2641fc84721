"""GB300-native fixed-precision randomized low-rank approximation (farPCA with
cheap test matrices, arxiv 2506.03859).

The compute path is the C-ABI library ``liblra.so`` (hand-written CUDA for
sm_103a, declared in ``include/lra.h``); ``paper_2506_03859_gb300.lra`` is its
thin ctypes binding, with PyTorch used only for device memory and streams.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from .build import build  # noqa: F401
