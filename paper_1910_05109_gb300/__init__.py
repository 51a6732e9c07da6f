"""GB300-native base64 codec (Mula & Lemire, arXiv:1910.05109).

The codec itself is CUDA in ``csrc/`` behind a C ABI (``include/b64gpu.h``),
compiled into ``libb64gpu.so`` in this directory. ``binding`` marshals
arguments to that library; it loads the library on first use and raises if it
is missing, so there is no CPU path. ``batch`` keeps a batch resident and
replays it as a CUDA graph, ``autotune`` picks its tile size, ``serve`` wraps
the serving engine, ``build`` compiles the library, and ``workloads`` draws
the seeded synthetic inputs.
"""
__all__ = ["autotune", "batch", "binding", "build", "serve", "workloads"]
