"""Exhaustive short strings through the batched decoder, against the oracle.

Every string below is its own batch entry, so the strict rules of Sec. 2 (as
read in the oracle: padding position, length classes, minimum offset) are
applied to each one separately:

- all 16,777,216 strings "XYZ=" (X, Y, Z any byte), standard table, padded:
  this holds every "XY==" and every final group with one pad;
- all 16,777,216 three-character strings, base64url, unpadded (decodes to 2
  bytes, or the first bad offset);
- all 65,536 two-character strings in both modes.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b64():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding
    binding.lib()
    yield binding
    assert binding.device_fault_flag() == 0


def all_strings(width: int, suffix: bytes = b"") -> np.ndarray:
    """Every `width`-byte string (first byte slowest), each followed by suffix."""
    v = np.arange(256 ** width, dtype=np.uint32)
    cols = [((v >> (8 * (width - 1 - k))) & 255).astype(np.uint8) for k in range(width)]
    cols += [np.full(v.size, c, np.uint8) for c in suffix]
    return np.stack(cols, axis=1)


def check_batch(b64, orc, strings: np.ndarray, alphabet, chars: bytes, padded: bool):
    n, w = strings.shape
    text = np.ascontiguousarray(strings).ravel()
    off = np.arange(n + 1, dtype=np.int64) * w
    aid = np.zeros(n, np.int32)
    dst_off = np.arange(n + 1, dtype=np.int64) * ((w + 3) // 4 * 3)
    want_dec, want_res = orc.decode_batch(text, off, dst_off, chars, aid,
                                          np.full(n, int(padded), np.int32), int(dst_off[-1]))
    d_text = torch.from_numpy(text).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_dst_off = torch.from_numpy(dst_off).cuda()
    dst = torch.zeros(int(dst_off[-1]) + 16, dtype=torch.uint8, device="cuda")
    res = b64.decode_batch(d_text, d_off, dst, d_dst_off, [alphabet])
    got_res = res.cpu().numpy()
    bad = np.nonzero(got_res != want_res)[0]
    assert bad.size == 0, [(bytes(strings[i]), int(got_res[i]), int(want_res[i])) for i in bad[:8]]
    # decoded bytes of every accepted string
    ok = np.nonzero(want_res >= 0)[0]
    got = dst[: int(dst_off[-1])].cpu().numpy().reshape(n, -1)
    want = want_dec.reshape(n, -1)
    lens = want_res[ok]
    for k in np.unique(lens):
        rows = ok[lens == k]
        assert np.array_equal(got[rows, :k], want[rows, :k])
    return want_res


def test_every_final_group_with_one_pad(b64, orc):
    res = check_batch(b64, orc, all_strings(3, b"="), b64.Alphabet.standard(),
                      orc.standard_alphabet(), True)
    assert (res == 2).sum() == 64 ** 3        # every XYZ= with X, Y, Z in the table
    assert (res == 1).sum() == 64 ** 2        # XY== (Z is '=')


def test_every_three_characters_unpadded(b64, orc):
    res = check_batch(b64, orc, all_strings(3), b64.Alphabet.url(), orc.url_alphabet(), False)
    assert (res == 2).sum() == 64 ** 3


@pytest.mark.parametrize("padded", [True, False])
def test_every_two_characters(b64, orc, padded):
    alph = b64.Alphabet.standard() if padded else b64.Alphabet.url()
    chars = orc.standard_alphabet() if padded else orc.url_alphabet()
    res = check_batch(b64, orc, all_strings(2), alph, chars, padded)
    if padded:
        # length error at offset 2 when nothing earlier fails: two table
        # characters, a table character then '=', or "=="
        assert (res == -3).sum() == 64 * 64 + 64 + 1
    else:
        assert (res == 1).sum() == 64 * 64
