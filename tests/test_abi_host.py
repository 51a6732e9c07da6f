"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/*.h declares, and its host-only logic (alphabet handles,
length helpers, argument checks) behaves as documented."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_1910_05109_gb300 import build
    build.build()
    from paper_1910_05109_gb300 import binding
    return binding.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(b64_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("b64_encode", "b64_decode", "b64_decode_async", "b64_alphabet_create",
                 "b64_alphabet_standard", "b64_alphabet_url", "b64_encoded_length",
                 "b64_decoded_max_length", "b64_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    from paper_1910_05109_gb300 import binding
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in binding.SIGNATURES, f"binding lacks {name}"


def test_lengths(L):
    from paper_1910_05109_gb300 import binding as b
    for n in range(0, 2000):
        assert b.encoded_length(n, True) == 4 * ((n + 2) // 3)
        assert b.encoded_length(n, False) == (4 * n + 2) // 3
        assert b.decoded_max_length(n) == 3 * ((n + 3) // 4)
    big = (1 << 40) + 1
    assert b.encoded_length(big, True) == 4 * ((big + 2) // 3)


def test_builtin_alphabets(L):
    from paper_1910_05109_gb300 import binding as b
    std, padded = b.Alphabet.standard().chars()
    assert padded and std == b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
    url, padded = b.Alphabet.url().chars()
    assert not padded and url == std[:62] + b"-_"


def test_alphabet_create_validation(L):
    from paper_1910_05109_gb300 import binding as b
    std = b.Alphabet.standard().chars()[0]
    a = b.Alphabet.create(std[::-1], True)
    assert a.chars() == (std[::-1], True)
    for bad, why in ((std[:63] + b"A", "twice"), (std[:63] + b"=", "reserved"),
                     (std[:63] + b"\n", "reserved"), (std[:63] + b" ", "reserved"),
                     (std[:63] + b"\x80", "reserved")):
        with pytest.raises(b.B64Error, match=why):
            b.Alphabet.create(bad, True)
    assert L.b64_alphabet_create(None, 1) is None


def test_argument_errors_without_gpu(L):
    from paper_1910_05109_gb300 import binding as b
    std = L.b64_alphabet_standard()
    # Rejected before any CUDA call is made.
    assert L.b64_encode(None, 10, None, std, None) == b.B64_E_INVAL
    assert "NULL" in b.last_error()
    assert L.b64_encode(None, 0, None, std, None) == 0
    assert L.b64_encode(16, 10, 16, None, None) == b.B64_E_INVAL
    assert L.b64_decode_async(None, 4, None, std, None, None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_decode_async(256, 4, 4096, std, 4099, None) == b.B64_ERR_INVALID_ARGUMENT
    assert "aligned" in b.last_error()
    # Overlapping src/dst are refused.
    assert L.b64_encode(4096, 300, 4096 + 100, std, None) == b.B64_E_INVAL
    assert "overlap" in b.last_error()
    assert L.b64_decode_async(4096, 400, 4096 + 100, std, 8, None) == \
        b.B64_ERR_INVALID_ARGUMENT
    # batch tile_units: units 1, 2, 4 or 8, blocks per SM in bits 8..15, the
    # pair-table bit 16; anything else is refused before a launch
    arr = (ctypes.c_void_p * 1)(std)
    for bad in (3, 8 | (1 << 17), -1):
        assert L.b64_encode_batch(256, 512, 4, 1024, 768, arr, 1, None, 2048, bad, 4096, 1 << 20,
                                  None) == b.B64_ERR_INVALID_ARGUMENT
        assert "tile_units" in b.last_error()


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_1910_05109_gb300 import binding as b
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(b.B64Error, match="missing"):
        b.lib()


def test_package_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1910_05109_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "workloads.py" and \
                    "import oracle" not in text, f


def test_alphabet_flags(L):
    from paper_1910_05109_gb300 import binding as b
    std = b.Alphabet.standard().chars()[0]
    a = b.Alphabet.create(std, True, canonical=True)
    assert a.padded and a.canonical
    assert L.b64_alphabet_flags(a.handle) == 3
    c = b.Alphabet.create(std, False, canonical=True)
    assert not c.padded and c.canonical and L.b64_alphabet_flags(c.handle) == 2
    assert L.b64_alphabet_flags(L.b64_alphabet_url()) == 0
    assert L.b64_alphabet_flags(None) == b.B64_ERR_INVALID_ARGUMENT
    buf = ctypes.create_string_buffer(std, 64)
    assert L.b64_alphabet_create_flags(buf, 4) is None      # unknown flag bit
    assert "flag" in b.last_error()
    h = L.b64_alphabet_create(buf, 1)                       # same as flags = padded
    assert L.b64_alphabet_flags(h) == 1
    L.b64_alphabet_destroy(h)


def test_new_entry_points_reject_bad_arguments_without_gpu(L):
    from paper_1910_05109_gb300 import binding as b
    std = L.b64_alphabet_standard()
    arr = (ctypes.c_void_p * 1)(std)
    # batched MIME: n < 0, no alphabets, NULL pointers, workspace too small or misaligned
    assert L.b64_mime_decode_batch(None, None, -1, None, None, arr, 1, None, None, None, 0,
                                   None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_mime_decode_batch(None, None, 4, None, None, None, 0, None, None, None, 0,
                                   None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_mime_decode_batch(None, None, 0, None, None, arr, 1, None, None, None, 0,
                                   None) == b.B64_SUCCESS          # n == 0: nothing to do
    assert L.b64_mime_decode_batch(16, None, 4, 16, 64, arr, 1, None, 128, 256, 4096,
                                   None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_mime_decode_batch(16, 64, 4, 16, 64, arr, 1, None, 128, 260, 4096,
                                   None) == b.B64_ERR_INVALID_ARGUMENT
    assert "aligned" in b.last_error()
    assert L.b64_mime_decode_batch(16, 64, 4, 16, 64, arr, 1, None, 128, 256, 8,
                                   None) == b.B64_ERR_INVALID_ARGUMENT
    assert "workspace" in b.last_error()
    assert L.b64_mime_batch_workspace_size(0, 1000) == 0
    assert L.b64_mime_batch_workspace_size(4, 4096 * 10) == 8 * (5 * 4 + 1 + 10 + 4 + 1)
    # bounded-wait self-test: NULL or misaligned result, limit out of range
    assert L.b64_selftest_wait_timeout(None, 1000, None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_selftest_wait_timeout(12, 1000, None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_selftest_wait_timeout(16, 0, None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_selftest_wait_timeout(16, 3_000_000_000, None) == b.B64_ERR_INVALID_ARGUMENT
    # host codec: NULL codec or alphabet, NULL buffers
    assert L.b64_host_encode(None, 16, 10, 16, std) == b.B64_E_INVAL
    assert L.b64_host_decode(None, 16, 10, 16, std) == b.B64_E_INVAL
    assert L.b64_host_codec_device_bytes(None) == 0
    L.b64_host_codec_destroy(None)
    # serving: a NULL server, a negative count, NULL arrays with n > 0
    assert L.b64_server_submit_many(None, 0, None, None, None, None, None, None,
                                    None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_server_submit_many(16, -1, None, None, None, None, None, None,
                                    None) == b.B64_ERR_INVALID_ARGUMENT
    assert L.b64_server_submit_many(16, 2, 16, 16, 16, None, 16, 16,
                                    16) == b.B64_ERR_INVALID_ARGUMENT
    assert "submit_many" in b.last_error()


def test_binding_rejects_host_and_mistyped_tensors(L):
    """Every wrapper checks its tensors before calling into the library, so a
    CPU tensor or a wrong dtype is an error, never a host-side computation."""
    import torch
    from paper_1910_05109_gb300 import binding as b
    host = torch.zeros(16, dtype=torch.uint8)
    off = torch.zeros(2, dtype=torch.int64)
    res = torch.zeros(1, dtype=torch.int64)
    calls = [
        lambda: b.encode(host),
        lambda: b.decode(host),
        lambda: b.encode(torch.zeros(16, dtype=torch.int32)),
        lambda: b.decode_async(host, host, res),
        lambda: b.mime_decode_async(host, host, res),
        lambda: b.mime_decode(host),
        lambda: b.encode_batch(host, off, host, off, [b.Alphabet.standard()]),
        lambda: b.decode_batch(host, off, host, off, [b.Alphabet.standard()]),
        lambda: b.mime_decode_batch(host, off, host, off, [b.Alphabet.standard()]),
        lambda: b.batch_offsets(off, [b.Alphabet.standard()], None, decode=True),
    ]
    for i, call in enumerate(calls):
        with pytest.raises(b.B64Error):
            call()
    with pytest.raises(b.B64Error, match="1..4"):
        b._alphabet_array([])
    with pytest.raises(b.B64Error, match="1..4"):
        b._alphabet_array([b.Alphabet.standard()] * 5)
    with pytest.raises(ValueError):
        b._host_u8(torch.zeros(4, dtype=torch.int16), "src")


def test_batch_wrappers_refuse_short_per_string_arrays(L):
    """The batched kernels index results, alph_id and dst_off by string with
    no bound of their own, so the wrappers refuse arrays shorter than the
    batch (before any device check, so this runs on the CPU) and the resident
    batch codec refuses an input buffer shorter than src_off[n]."""
    import torch
    from paper_1910_05109_gb300 import binding as b
    n = 10
    buf = torch.zeros(64, dtype=torch.uint8)
    off = torch.zeros(n + 1, dtype=torch.int64)
    alphs = [b.Alphabet.standard()]
    short_res = torch.zeros(n - 1, dtype=torch.int64)
    short_aid = torch.zeros(n - 1, dtype=torch.uint8)
    short_doff = torch.zeros(n - 1, dtype=torch.int64)
    ok_res = torch.zeros(n, dtype=torch.int64)
    for fn in (b.encode_batch, b.decode_batch, b.mime_decode_batch):
        with pytest.raises(b.B64Error, match="results holds 9 entries"):
            fn(buf, off, buf, off, alphs, None, short_res)
        with pytest.raises(b.B64Error, match="alph_id holds 9 entries"):
            fn(buf, off, buf, off, alphs, short_aid, ok_res)
        with pytest.raises(b.B64Error, match="dst_off holds 9 entries"):
            fn(buf, off, buf, short_doff, alphs, None, ok_res)
    with pytest.raises(b.B64Error, match="alph_id holds 9 entries"):
        b.batch_offsets(off, alphs, short_aid, decode=False)
    with pytest.raises(b.B64Error, match="workspace holds 8 bytes"):
        b.decode_batch(buf, off, buf, off, alphs, None, ok_res,
                       workspace=torch.zeros(8, dtype=torch.uint8))
    with pytest.raises(b.B64Error, match="src holds 64 bytes; src_off"):
        b.check_batch_totals(buf, 65)
    with pytest.raises(b.B64Error, match="dst holds 64 bytes; dst_off"):
        b.check_batch_totals(buf, 64, buf, 100)
    b.check_batch_totals(buf, 64, buf, 64)
