"""ctypes binding of libb64gpu.so (C ABI in include/b64gpu.h).

Argument marshalling only: every step of encoding and decoding runs in the
library's CUDA kernels. PyTorch supplies device memory and streams. If the
library has not been built, loading raises; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libb64gpu.so")

B64_SUCCESS = 0
B64_ERR_INVALID_ARGUMENT = -1
B64_ERR_CUDA = -2
B64_E_INVAL = -(2**63) + 1
B64_E_CUDA = -(2**63) + 2
B64_E_TIMEOUT = -(2**63) + 3

_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_P, _SZ, _I, _I64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "b64_alphabet_create": (_P, [_P, _I]),
    "b64_alphabet_create_flags": (_P, [_P, _I]),
    "b64_alphabet_flags": (_I, [_P]),
    "b64_alphabet_standard": (_P, []),
    "b64_alphabet_url": (_P, []),
    "b64_alphabet_destroy": (None, [_P]),
    "b64_alphabet_chars": (_I, [_P, _P]),
    "b64_encoded_length": (_SZ, [_SZ, _I]),
    "b64_decoded_max_length": (_SZ, [_SZ]),
    "b64_encode": (_I64, [_P, _SZ, _P, _P, _P]),
    "b64_decode_async": (_I, [_P, _SZ, _P, _P, _P, _P]),
    "b64_decode": (_I64, [_P, _SZ, _P, _P, _P]),
    "b64_batch_workspace_size": (_SZ, [_I64]),
    "b64_encode_batch": (_I, [_P, _P, _I64, _P, _P, _P, _I, _P, _P, _I, _P, _SZ, _P]),
    "b64_decode_batch": (_I, [_P, _P, _I64, _P, _P, _P, _I, _P, _P, _I, _P, _SZ, _P]),
    "b64_batch_offsets": (_I, [_P, _I64, _P, _I, _P, _I, _P, _P]),
    "b64_decode_batch_noalloc": (_I, [_P, _P, _I64, _P, _P, _P, _I, _P, _P, _I, _P]),
    "b64_mime_workspace_size": (_SZ, [_SZ]),
    "b64_mime_decode_async": (_I, [_P, _SZ, _P, _P, _P, _P, _SZ, _P]),
    "b64_mime_batch_workspace_size": (_SZ, [_I64, ctypes.c_uint64]),
    "b64_mime_decode_batch": (_I, [_P, _P, _I64, _P, _P, _P, _I, _P, _P, _P, _SZ, _P]),
    "b64_selftest_wait_timeout": (_I, [_P, ctypes.c_uint64, _P]),
    "b64_server_create": (_P, [_SZ, _I, _SZ, _P, _I]),
    "b64_server_submit": (_I, [_P, ctypes.c_uint64, _I, _I, _P, _SZ, _P, _SZ]),
    "b64_server_submit_many": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "b64_server_poll": (_I, [_P, _P, _I]),
    "b64_server_outstanding": (_I, [_P]),
    "b64_server_batches": (ctypes.c_uint64, [_P]),
    "b64_server_destroy": (None, [_P]),
    "b64_host_codec_create": (_P, [_SZ, _I]),
    "b64_host_codec_device_bytes": (_SZ, [_P]),
    "b64_host_encode": (_I64, [_P, _P, _SZ, _P, _P]),
    "b64_host_decode": (_I64, [_P, _P, _SZ, _P, _P]),
    "b64_host_codec_destroy": (None, [_P]),
    "b64_last_error": (ctypes.c_char_p, []),
    "b64_device_fault_flag": (_I, [_I]),
    "b64_version": (_I, []),
}


class B64Error(RuntimeError):
    pass


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it is missing (build it with build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise B64Error(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1910_05109_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().b64_last_error().decode()


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_u8(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise B64Error(f"{name} must be a CUDA tensor")
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise B64Error(f"{name} must be a contiguous uint8 tensor")
    return t


class Alphabet:
    """A 64-character table plus padding mode (library handle)."""

    def __init__(self, handle: int, owned: bool):
        self.handle = handle
        self._owned = owned
        self._padded = None  # alphabets are immutable: read once

    @classmethod
    def standard(cls) -> "Alphabet":
        return cls(lib().b64_alphabet_standard(), False)

    @classmethod
    def url(cls) -> "Alphabet":
        return cls(lib().b64_alphabet_url(), False)

    @classmethod
    def create(cls, chars: bytes, padded: bool, canonical: bool = False) -> "Alphabet":
        """canonical: decode rejects non-zero unused bits in a partial final group."""
        buf = ctypes.create_string_buffer(bytes(chars), 64)
        h = lib().b64_alphabet_create_flags(buf, (1 if padded else 0) | (2 if canonical else 0))
        if not h:
            raise B64Error(last_error())
        return cls(h, True)

    def chars(self) -> tuple[bytes, bool]:
        buf = ctypes.create_string_buffer(64)
        padded = lib().b64_alphabet_chars(self.handle, buf)
        return buf.raw, bool(padded)

    @property
    def canonical(self) -> bool:
        return bool(lib().b64_alphabet_flags(self.handle) & 2)

    @property
    def padded(self) -> bool:
        if self._padded is None:
            self._padded = self.chars()[1]
        return self._padded

    def __del__(self):
        if getattr(self, "_owned", False) and self.handle and _lib is not None:
            _lib.b64_alphabet_destroy(self.handle)
            self.handle = None


def encoded_length(n: int, padded: bool = True) -> int:
    return lib().b64_encoded_length(n, int(padded))


def decoded_max_length(m: int) -> int:
    return lib().b64_decoded_max_length(m)


def encode(src: torch.Tensor, alphabet: Alphabet | None = None, dst: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Enqueues the encode of ``src``; returns the output view of ``dst``."""
    alphabet = alphabet or Alphabet.standard()
    src = _dev_u8(src, "src")
    n = src.numel()
    out_len = encoded_length(n, alphabet.padded)
    if dst is None:
        dst = torch.empty(max(out_len, 1), dtype=torch.uint8, device=src.device)
    dst = _dev_u8(dst, "dst")
    if dst.numel() < out_len:
        raise B64Error(f"dst holds {dst.numel()} bytes, {out_len} needed")
    r = lib().b64_encode(src.data_ptr(), n, dst.data_ptr(), alphabet.handle, _stream_ptr(stream))
    if r < 0:
        raise B64Error(last_error())
    return dst[:r]


def decode_async(src: torch.Tensor, dst: torch.Tensor, d_result: torch.Tensor,
                 alphabet: Alphabet | None = None, stream=None) -> None:
    """Enqueues a strict decode; d_result (int64, 1 element, on the device)
    receives the length, -(offset+1), or B64_E_TIMEOUT."""
    alphabet = alphabet or Alphabet.standard()
    src, dst = _dev_u8(src, "src"), _dev_u8(dst, "dst")
    if d_result.dtype != torch.int64 or d_result.device.type != "cuda":
        raise B64Error("d_result must be a CUDA int64 tensor")
    m = src.numel()
    if dst.numel() < decoded_max_length(m):
        raise B64Error("dst is smaller than decoded_max_length(len(src))")
    rc = lib().b64_decode_async(src.data_ptr(), m, dst.data_ptr(), alphabet.handle,
                                d_result.data_ptr(), _stream_ptr(stream))
    if rc != B64_SUCCESS:
        raise B64Error(last_error())


def decode(src: torch.Tensor, alphabet: Alphabet | None = None, dst: torch.Tensor | None = None,
           stream=None) -> tuple[int, torch.Tensor]:
    """Strict decode (synchronises the stream). Returns (result, view): result
    is the decoded length or -(offset+1) of the first error."""
    alphabet = alphabet or Alphabet.standard()
    src = _dev_u8(src, "src")
    m = src.numel()
    cap = decoded_max_length(m)
    if dst is None:
        dst = torch.empty(max(cap, 1), dtype=torch.uint8, device=src.device)
    dst = _dev_u8(dst, "dst")
    if dst.numel() < cap:
        raise B64Error(f"dst holds {dst.numel()} bytes, {cap} needed")
    r = lib().b64_decode(src.data_ptr(), m, dst.data_ptr(), alphabet.handle, _stream_ptr(stream))
    if r in (B64_E_INVAL, B64_E_CUDA):
        raise B64Error(last_error())
    if r == B64_E_TIMEOUT:
        raise B64Error("a device wait ran out of time (see device_fault_flag)")
    return int(r), dst[: max(r, 0)]


def device_fault_flag(clear: bool = False) -> int:
    r = lib().b64_device_fault_flag(int(clear))
    if r < 0:
        raise B64Error(last_error())
    return r


# ---------------------------------------------------------------- batches

BATCH_MAX_ALPHABETS = 4


def _alphabet_array(alphabets):
    alphabets = list(alphabets)
    if not 1 <= len(alphabets) <= BATCH_MAX_ALPHABETS:
        raise B64Error(f"need 1..{BATCH_MAX_ALPHABETS} alphabets")
    arr = (ctypes.c_void_p * len(alphabets))(*[a.handle for a in alphabets])
    return arr, len(alphabets)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
        raise B64Error(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def check_batch_counts(n: int, results=None, alph_id=None, dst_off=None,
                       what: str = "string") -> None:
    """Refuses per-string arrays shorter than the batch's n entries (the
    kernels index them by string with no bound): results and alph_id hold n
    entries each, dst_off at least n. Raises B64Error before anything runs."""
    for name, t, need in (("results", results, n), ("alph_id", alph_id, n),
                          ("dst_off", dst_off, n)):
        if t is not None and t.numel() < need:
            raise B64Error(f"{name} holds {t.numel()} entries; the batch has {n} {what}s "
                           f"and needs {need}")


def check_batch_totals(src: torch.Tensor, src_total: int, dst: torch.Tensor | None = None,
                       dst_total: int | None = None) -> None:
    """Refuses buffers smaller than the offsets say (src_off[n] input bytes,
    dst_off[n] output bytes), for callers that already hold those totals on
    the host."""
    if src.numel() < src_total:
        raise B64Error(f"src holds {src.numel()} bytes; src_off[n] is {src_total}")
    if dst is not None and dst_total is not None and dst.numel() < dst_total:
        raise B64Error(f"dst holds {dst.numel()} bytes; dst_off[n] is {dst_total}")


def batch_workspace(n: int, device=None) -> torch.Tensor:
    nbytes = lib().b64_batch_workspace_size(n)
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device or "cuda")


OFFSETS_DECODE = 1
OFFSETS_ALIGN16 = 2


def batch_offsets(src_off: torch.Tensor, alphabets, alph_id: torch.Tensor | None,
                  decode: bool, stream=None, align16: bool = False) -> torch.Tensor:
    """Device int64[n+1]: exclusive scan of per-string output capacities
    (align16: each rounded up to 16 bytes, so outputs start 16-byte aligned)."""
    n = src_off.numel() - 1
    check_batch_counts(n, alph_id=alph_id)
    src_off = _dev(src_off, torch.int64, "src_off")
    arr, na = _alphabet_array(alphabets)
    out = torch.empty(n + 1, dtype=torch.int64, device=src_off.device)
    aid = 0 if alph_id is None else _dev(alph_id, torch.uint8, "alph_id").data_ptr()
    flags = (OFFSETS_DECODE if decode else 0) | (OFFSETS_ALIGN16 if align16 else 0)
    rc = lib().b64_batch_offsets(src_off.data_ptr(), n, arr, na, aid, flags,
                                 out.data_ptr(), _stream_ptr(stream))
    if rc != B64_SUCCESS:
        raise B64Error(last_error())
    return out


def _batch(fn, src, src_off, dst, dst_off, alphabets, alph_id, results, tile_units, workspace,
           stream):
    n = src_off.numel() - 1
    check_batch_counts(n, results, alph_id, dst_off)
    if workspace is not None:
        need = lib().b64_batch_workspace_size(n)
        if workspace.numel() < need:
            raise B64Error(f"workspace holds {workspace.numel()} bytes, {need} needed")
    src = _dev_u8(src, "src")
    dst = _dev_u8(dst, "dst")
    src_off = _dev(src_off, torch.int64, "src_off")
    dst_off = _dev(dst_off, torch.int64, "dst_off")
    results = _dev(results, torch.int64, "results")
    arr, na = _alphabet_array(alphabets)
    aid = 0 if alph_id is None else _dev(alph_id, torch.uint8, "alph_id").data_ptr()
    if workspace is None:
        workspace = batch_workspace(n, src.device)
    rc = fn(src.data_ptr(), src_off.data_ptr(), n, dst.data_ptr(), dst_off.data_ptr(), arr, na,
            aid, results.data_ptr(), int(tile_units), workspace.data_ptr(), workspace.numel(),
            _stream_ptr(stream))
    if rc != B64_SUCCESS:
        raise B64Error(last_error())
    return workspace


def encode_batch(src, src_off, dst, dst_off, alphabets, alph_id=None, results=None,
                 tile_units: int = 0, workspace=None, stream=None):
    """Enqueues a batched encode; returns the results tensor (int64[n])."""
    n = src_off.numel() - 1
    if results is None:
        results = torch.empty(max(n, 1), dtype=torch.int64, device=src.device)
    _batch(lib().b64_encode_batch, src, src_off, dst, dst_off, alphabets, alph_id, results,
           tile_units, workspace, stream)
    return results[:n]


def decode_batch(src, src_off, dst, dst_off, alphabets, alph_id=None, results=None,
                 tile_units: int = 0, workspace=None, stream=None):
    """Enqueues a batched strict decode; returns the results tensor (int64[n])."""
    n = src_off.numel() - 1
    if results is None:
        results = torch.empty(max(n, 1), dtype=torch.int64, device=src.device)
    _batch(lib().b64_decode_batch, src, src_off, dst, dst_off, alphabets, alph_id, results,
           tile_units, workspace, stream)
    return results[:n]


# ---------------------------------------------------------------- MIME

def mime_workspace(m: int, device=None) -> torch.Tensor:
    return torch.empty(max(lib().b64_mime_workspace_size(m), 8), dtype=torch.uint8,
                       device=device or "cuda")


def mime_decode_async(src: torch.Tensor, dst: torch.Tensor, d_result: torch.Tensor,
                      alphabet: Alphabet | None = None, workspace=None, stream=None):
    """Enqueues a whitespace-skipping strict decode; returns the workspace used."""
    alphabet = alphabet or Alphabet.standard()
    src, dst = _dev_u8(src, "src"), _dev_u8(dst, "dst")
    if d_result.dtype != torch.int64 or d_result.device.type != "cuda":
        raise B64Error("d_result must be a CUDA int64 tensor")
    m = src.numel()
    if dst.numel() < decoded_max_length(m):
        raise B64Error("dst is smaller than decoded_max_length(len(src))")
    if workspace is None:
        workspace = mime_workspace(m, src.device)
    rc = lib().b64_mime_decode_async(src.data_ptr(), m, dst.data_ptr(), alphabet.handle,
                                     d_result.data_ptr(), workspace.data_ptr(),
                                     workspace.numel(), _stream_ptr(stream))
    if rc != B64_SUCCESS:
        raise B64Error(last_error())
    return workspace


def mime_decode(src: torch.Tensor, alphabet: Alphabet | None = None, dst=None, workspace=None,
                stream=None) -> tuple[int, torch.Tensor]:
    """Whitespace-skipping strict decode (synchronises). Returns (result, view)."""
    m = src.numel()
    if dst is None:
        dst = torch.empty(max(decoded_max_length(m), 1), dtype=torch.uint8, device=src.device)
    res = torch.empty(1, dtype=torch.int64, device=src.device)
    mime_decode_async(src, dst, res, alphabet, workspace, stream)
    r = int(res.item())
    if r == B64_E_TIMEOUT:
        raise B64Error("a device wait ran out of time (see device_fault_flag)")
    return r, dst[: max(r, 0)]


def _host_u8(t, name: str) -> int:
    """Address of a contiguous uint8 host buffer (CPU tensor or numpy array)."""
    if isinstance(t, torch.Tensor):
        if t.device.type != "cpu" or t.dtype != torch.uint8 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous uint8 CPU tensor")
        return t.data_ptr()
    import numpy as np
    if not isinstance(t, np.ndarray) or t.dtype != np.uint8 or not t.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be a contiguous uint8 array")
    return t.ctypes.data


class HostCodec:
    """Encode / strict decode of host buffers, pieces of piece_bytes copied in,
    coded and copied out with the steps of consecutive pieces overlapped on
    n_streams streams. Page-locked buffers (torch pin_memory) overlap fully."""

    def __init__(self, piece_bytes: int = 0, n_streams: int = 0):
        self._lib = lib()
        self.handle = self._lib.b64_host_codec_create(piece_bytes, n_streams)
        if not self.handle:
            raise B64Error(last_error())

    def device_bytes(self) -> int:
        return int(self._lib.b64_host_codec_device_bytes(self.handle))

    def encode(self, src, dst, alphabet: Alphabet | None = None) -> int:
        a = alphabet or Alphabet.standard()
        n = src.numel() if isinstance(src, torch.Tensor) else src.size
        need = encoded_length(n, a.padded)
        cap = dst.numel() if isinstance(dst, torch.Tensor) else dst.size
        if cap < need:
            raise ValueError(f"dst holds {cap} bytes, needs {need}")
        r = self._lib.b64_host_encode(self.handle, _host_u8(src, "src"), n,
                                      _host_u8(dst, "dst"), a.handle)
        if r < 0:
            raise B64Error(last_error())
        return int(r)

    def decode(self, src, dst, alphabet: Alphabet | None = None) -> int:
        """Returns the decoded length or -(offset+1) of the first bad character."""
        a = alphabet or Alphabet.standard()
        m = src.numel() if isinstance(src, torch.Tensor) else src.size
        need = decoded_max_length(m)
        cap = dst.numel() if isinstance(dst, torch.Tensor) else dst.size
        if cap < need:
            raise ValueError(f"dst holds {cap} bytes, needs {need}")
        r = self._lib.b64_host_decode(self.handle, _host_u8(src, "src"), m,
                                      _host_u8(dst, "dst"), a.handle)
        if r in (B64_E_INVAL, B64_E_CUDA):
            raise B64Error(last_error())
        if r == B64_E_TIMEOUT:
            raise B64Error("a device wait ran out of time (see device_fault_flag)")
        return int(r)

    def close(self):
        if self.handle:
            self._lib.b64_host_codec_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mime_decode_batch(src: torch.Tensor, src_off: torch.Tensor, dst: torch.Tensor,
                      dst_off: torch.Tensor, alphabets, alph_id: torch.Tensor | None = None,
                      results: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Enqueues the whitespace-skipping strict decode of every document;
    returns the device int64 results."""
    n = src_off.numel() - 1
    check_batch_counts(n, results, alph_id, dst_off, what="document")
    src, dst = _dev_u8(src, "src"), _dev_u8(dst, "dst")
    src_off = _dev(src_off, torch.int64, "src_off")
    dst_off = _dev(dst_off, torch.int64, "dst_off")
    arr, na = _alphabet_array(alphabets)
    if results is None:
        results = torch.empty(max(n, 1), dtype=torch.int64, device=src_off.device)
    if workspace is None and n > 0:
        total = int((src_off[-1] - src_off[0]).item())
        size = lib().b64_mime_batch_workspace_size(n, total)
        workspace = torch.empty(max(size, 8), dtype=torch.uint8, device=src_off.device)
    aid = 0 if alph_id is None else _dev(alph_id, torch.uint8, "alph_id").data_ptr()
    rc = lib().b64_mime_decode_batch(
        src.data_ptr() if src.numel() else 0, src_off.data_ptr(), n,
        dst.data_ptr() if dst.numel() else 0, dst_off.data_ptr(), arr, na, aid,
        results.data_ptr(), workspace.data_ptr() if workspace is not None else 0,
        workspace.numel() if workspace is not None else 0, _stream_ptr(stream))
    if rc != B64_SUCCESS:
        raise B64Error(last_error())
    return results[:n]
