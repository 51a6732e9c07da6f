"""Resident batched codec: buffers kept on the device, the launch sequence
recorded once as a CUDA graph and replayed. The tile size is the caller's
(`tile_units`, 4 by default; `autotune.best_units` picks one for a batch).

A BatchCodec is built for one batch shape (string count, total bytes, output
capacity). With align16 its output offsets give every string a 16-byte aligned
start (b64_batch_offsets' B64_OFFSETS_ALIGN16), which the kernels store
straight from registers. `run(src, src_off, alph_id)` copies nothing itself: the caller's
device tensors are copied into the codec's resident input buffers (one
device-to-device copy each, captured in the graph too), so every replay reads
the same addresses.
"""
from __future__ import annotations

import torch

from . import binding as b64


class BatchCodec:
    def __init__(self, op: str, n: int, src_bytes: int, alphabets, device=None,
                 tile_units: int | None = None, use_graph: bool = True, stream=None,
                 align16: bool = False):
        if op not in ("encode", "decode"):
            raise ValueError("op must be 'encode' or 'decode'")
        self.op, self.n = op, n
        self.device = torch.device(device or "cuda")
        self.alphabets = list(alphabets)
        self.stream = stream or torch.cuda.Stream(device=self.device)
        z = dict(device=self.device)
        self.src = torch.empty(max(src_bytes, 1), dtype=torch.uint8, **z)
        self.src_off = torch.zeros(n + 1, dtype=torch.int64, **z)
        self.alph_id = torch.zeros(max(n, 1), dtype=torch.uint8, **z)
        self.dst_off = torch.zeros(n + 1, dtype=torch.int64, **z)
        self.results = torch.empty(max(n, 1), dtype=torch.int64, **z)
        self.workspace = b64.batch_workspace(n, self.device)
        self.dst = None
        self.tile_units = tile_units or 4
        self.use_graph = use_graph
        self.align16 = align16  # output offsets with 16-byte aligned string starts
        self.graph = None

    def _enqueue(self):
        fn = b64.encode_batch if self.op == "encode" else b64.decode_batch
        fn(self.src, self.src_off, self.dst, self.dst_off, self.alphabets, self.alph_id[:self.n],
           self.results, self.tile_units, self.workspace, stream=self.stream)

    def load(self, src: torch.Tensor, src_off: torch.Tensor, alph_id: torch.Tensor | None):
        """Copies a batch into the resident buffers and sizes the output."""
        with torch.cuda.stream(self.stream):
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            self.src[:src.numel()].copy_(src, non_blocking=True)
            self.src_off.copy_(src_off, non_blocking=True)
            if alph_id is not None:
                self.alph_id[:self.n].copy_(alph_id, non_blocking=True)
            else:
                self.alph_id[:self.n].zero_()    # every string takes alphabet 0
            off = b64.batch_offsets(self.src_off, self.alphabets, self.alph_id[:self.n],
                                    decode=self.op == "decode", stream=self.stream,
                                    align16=self.align16)
            self.dst_off.copy_(off, non_blocking=True)
        self.stream.synchronize()
        b64.check_batch_totals(self.src, int(self.src_off[-1]))
        total = int(self.dst_off[-1])
        if self.dst is None or self.dst.numel() < total:
            self.dst = torch.empty(max(total, 1), dtype=torch.uint8, device=self.device)
            self.graph = None
        return total

    def run(self) -> None:
        """Enqueues the batch on the codec's stream. The first call after
        load() runs the launch sequence directly (which also sets the kernels
        up outside any capture) and then records it as a graph, which runs
        nothing; later calls replay the graph. Each call codes the batch once."""
        if not self.use_graph:
            self._enqueue()
            return
        if self.graph is None:
            self._enqueue()
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self._enqueue()
            self.graph = g
            return
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def synchronize(self):
        self.stream.synchronize()
