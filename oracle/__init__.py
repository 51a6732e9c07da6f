"""Oracle: a plain scalar base64 codec in C, loaded through ctypes.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The GPU library
never imports it and shares no code with it.

What the C file computes, and the passages it follows, is stated in the header
of ``b64_oracle.c`` (Sec. 2 and Table 1 of Mula & Lemire, arXiv:1910.05109,
plus the readings R1-R6 for what the paper leaves open).

Parity status: encode, decode, the strict rules and the batched loops are
pinned by tests under ``tests/test_oracle_*.py``; MIME-mode error offsets are
pinned only by the stated rule R5 and by brute force on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "b64_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Werror", "-shared",
                               "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_encoded_length.restype = ctypes.c_size_t
            lib.oracle_encoded_length.argtypes = [ctypes.c_size_t, ctypes.c_int]
            lib.oracle_encode.restype = ctypes.c_int64
            lib.oracle_encode.argtypes = [P, ctypes.c_size_t, P, P, ctypes.c_int]
            lib.oracle_decode.restype = ctypes.c_int64
            lib.oracle_decode.argtypes = [P, ctypes.c_size_t, P, P, ctypes.c_int, ctypes.c_int]
            lib.oracle_value_of.restype = ctypes.c_int
            lib.oracle_value_of.argtypes = [P, ctypes.c_uint8]
            lib.oracle_standard_alphabet.argtypes = [P]
            lib.oracle_url_alphabet.argtypes = [P]
            lib.oracle_encode_batch.argtypes = [P, P, P, P, P, P, P, ctypes.c_int64, P]
            lib.oracle_decode_batch.argtypes = [P, P, P, P, P, P, P, ctypes.c_int32,
                                                ctypes.c_int64, P]
            _lib = lib
    return _lib


def _u8(buf) -> np.ndarray:
    if isinstance(buf, np.ndarray):
        return np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
    return np.frombuffer(bytes(buf), dtype=np.uint8)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def standard_alphabet() -> bytes:
    out = np.zeros(64, np.uint8)
    _load().oracle_standard_alphabet(_ptr(out))
    return out.tobytes()


def url_alphabet() -> bytes:
    out = np.zeros(64, np.uint8)
    _load().oracle_url_alphabet(_ptr(out))
    return out.tobytes()


def value_of(alphabet: bytes, c: int) -> int:
    a = _u8(alphabet)
    return _load().oracle_value_of(_ptr(a), c)


def encoded_length(n: int, padded: bool = True) -> int:
    return _load().oracle_encoded_length(n, int(padded))


def encode(data, alphabet: bytes | None = None, padded: bool = True) -> np.ndarray:
    """Encodes ``data``; returns the characters as a uint8 array."""
    src = _u8(data)
    alph = _u8(alphabet if alphabet is not None else standard_alphabet())
    out = np.zeros(max(1, encoded_length(src.size, padded)), np.uint8)
    k = _load().oracle_encode(_ptr(src), src.size, _ptr(out), _ptr(alph), int(padded))
    return out[:k]


def decode(text, alphabet: bytes | None = None, padded: bool = True,
           mime: bool = False, canonical: bool = False) -> tuple[int, np.ndarray]:
    """Strict decode. Returns (result, bytes): result is the decoded length
    (>= 0) or -(offset+1) of the first error; bytes is empty on error.
    canonical: also reject non-zero unused bits in a partial final group."""
    src = _u8(text)
    alph = _u8(alphabet if alphabet is not None else standard_alphabet())
    out = np.zeros(max(1, 3 * ((src.size + 3) // 4)), np.uint8)
    flags = int(bool(padded)) | (int(bool(canonical)) << 1)
    r = _load().oracle_decode(_ptr(src), src.size, _ptr(out), _ptr(alph), flags, int(mime))
    return int(r), (out[:r] if r >= 0 else out[:0])


def encode_batch(src: np.ndarray, src_off: np.ndarray, dst_off: np.ndarray,
                 alphabets: bytes, alph_id: np.ndarray, padded: np.ndarray,
                 dst_size: int) -> tuple[np.ndarray, np.ndarray]:
    src = _u8(src)
    src_off = np.ascontiguousarray(src_off, np.int64)
    dst_off = np.ascontiguousarray(dst_off, np.int64)
    alph = _u8(alphabets)
    alph_id = np.ascontiguousarray(alph_id, np.int32)
    padded = np.ascontiguousarray(padded, np.int32)
    n = src_off.size - 1
    dst = np.zeros(max(1, dst_size), np.uint8)
    res = np.zeros(max(1, n), np.int64)
    _load().oracle_encode_batch(_ptr(src), _ptr(src_off), _ptr(dst), _ptr(dst_off), _ptr(alph),
                                _ptr(alph_id), _ptr(padded), n, _ptr(res))
    return dst[:dst_size], res[:n]


def decode_batch(src: np.ndarray, src_off: np.ndarray, dst_off: np.ndarray,
                 alphabets: bytes, alph_id: np.ndarray, padded: np.ndarray,
                 dst_size: int, mime: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Per string: padded[i] carries its flags (bit 0 padded, bit 1 canonical)."""
    src = _u8(src)
    src_off = np.ascontiguousarray(src_off, np.int64)
    dst_off = np.ascontiguousarray(dst_off, np.int64)
    alph = _u8(alphabets)
    alph_id = np.ascontiguousarray(alph_id, np.int32)
    padded = np.ascontiguousarray(padded, np.int32)
    n = src_off.size - 1
    dst = np.zeros(max(1, dst_size), np.uint8)
    res = np.zeros(max(1, n), np.int64)
    _load().oracle_decode_batch(_ptr(src), _ptr(src_off), _ptr(dst), _ptr(dst_off), _ptr(alph),
                                _ptr(alph_id), _ptr(padded), int(mime), n, _ptr(res))
    return dst[:dst_size], res[:n]
