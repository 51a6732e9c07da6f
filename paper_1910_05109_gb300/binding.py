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

_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_P, _SZ, _I, _I64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "b64_alphabet_create": (_P, [_P, _I]),
    "b64_alphabet_standard": (_P, []),
    "b64_alphabet_url": (_P, []),
    "b64_alphabet_destroy": (None, [_P]),
    "b64_alphabet_chars": (_I, [_P, _P]),
    "b64_encoded_length": (_SZ, [_SZ, _I]),
    "b64_decoded_max_length": (_SZ, [_SZ]),
    "b64_encode": (_I64, [_P, _SZ, _P, _P, _P]),
    "b64_decode_async": (_I, [_P, _SZ, _P, _P, _P, _P]),
    "b64_decode": (_I64, [_P, _SZ, _P, _P, _P]),
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

    @classmethod
    def standard(cls) -> "Alphabet":
        return cls(lib().b64_alphabet_standard(), False)

    @classmethod
    def url(cls) -> "Alphabet":
        return cls(lib().b64_alphabet_url(), False)

    @classmethod
    def create(cls, chars: bytes, padded: bool) -> "Alphabet":
        buf = ctypes.create_string_buffer(bytes(chars), 64)
        h = lib().b64_alphabet_create(buf, int(padded))
        if not h:
            raise B64Error(last_error())
        return cls(h, True)

    def chars(self) -> tuple[bytes, bool]:
        buf = ctypes.create_string_buffer(64)
        padded = lib().b64_alphabet_chars(self.handle, buf)
        return buf.raw, bool(padded)

    @property
    def padded(self) -> bool:
        return self.chars()[1]

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
    receives the length or -(offset+1)."""
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
    return int(r), dst[: max(r, 0)]


def device_fault_flag(clear: bool = False) -> int:
    r = lib().b64_device_fault_flag(int(clear))
    if r < 0:
        raise B64Error(last_error())
    return r
