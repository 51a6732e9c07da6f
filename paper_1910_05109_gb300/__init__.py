"""GB300-native base64 codec (Mula & Lemire, arXiv:1910.05109).

The codec itself is CUDA in ``csrc/`` behind a C ABI (``include/b64gpu.h``),
compiled into ``libb64gpu.so`` in this directory. ``binding`` marshals
arguments to that library; it loads the library on first use and raises if it
is missing, so there is no CPU path.
"""
__all__ = ["binding", "workloads"]
