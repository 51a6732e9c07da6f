"""Exhaustive short strings through the batched decoder, against the oracle.

Every string below is its own batch entry, so the strict rules of Sec. 2 (as
read in the oracle: padding position, length classes, minimum offset) are
applied to each one separately:

- all 16,777,216 strings "XYZ=" (X, Y, Z any byte), standard table, padded:
  this holds every "XY==" and every final group with one pad;
- all 16,777,216 three-character strings, base64url, unpadded (decodes to 2
  bytes, or the first bad offset);
- all 65,536 two-character strings in both modes;
- all 4,294,967,296 four-byte strings, standard padded and base64url
  unpadded: every result against the oracle's result for the string's class
  pattern (quad_classes.py; pinned in test_oracle_quads.py), and the bytes of
  every accepted string against the oracle's decode of it.
"""
import numpy as np
import pytest
import torch

import quad_classes as qc

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


@pytest.mark.parametrize("padded", [True, False])
def test_every_four_byte_string(b64, orc, padded):
    alph = b64.Alphabet.standard() if padded else b64.Alphabet.url()
    chars = orc.standard_alphabet() if padded else orc.url_alphabet()
    table = torch.from_numpy(qc.pattern_table(orc, chars, padded)).cuda()
    cls = torch.from_numpy(qc.byte_classes(chars)).cuda()
    N = 1 << 26                                     # strings per batch; 64 batches
    dev = "cuda"
    off = torch.arange(0, 4 * (N + 1), 4, dtype=torch.int64, device=dev)
    doff = torch.arange(0, 3 * (N + 1), 3, dtype=torch.int64, device=dev)
    dst = torch.empty(3 * N + 16, dtype=torch.uint8, device=dev)
    res = torch.empty(N, dtype=torch.int64, device=dev)
    ws = torch.empty(max(1, b64.lib().b64_batch_workspace_size(N)), dtype=torch.uint8, device=dev)
    s = torch.empty((N, 4), dtype=torch.uint8, device=dev)
    base = torch.arange(N, dtype=torch.int64, device=dev)
    acc_in, acc_out, acc_len = [], [], []
    for c in range(64):
        x = base + (c << 26)                        # string x: bytes x & 255, (x >> 8) & 255, ...
        for i in range(4):
            s[:, i] = ((x >> (8 * i)) & 255).to(torch.uint8)
        b64.decode_batch(s.view(-1), off, dst, doff, [alph], results=res, workspace=ws)
        pat = cls[s[:, 0].long()] + 3 * cls[s[:, 1].long()] + 9 * cls[s[:, 2].long()] + \
            27 * cls[s[:, 3].long()]
        want = table[pat]
        if not torch.equal(res, want):
            i = int(torch.nonzero(res != want)[0])
            raise AssertionError((c, bytes(s[i].cpu().numpy()), int(res[i]), int(want[i])))
        ok = res >= 0
        acc_in.append(s[ok].cpu())
        acc_out.append(dst[:3 * N].view(N, 3)[ok].cpu())
        acc_len.append(res[ok].cpu())
    vin = torch.cat(acc_in).numpy()
    vout = torch.cat(acc_out).numpy()
    vlen = torch.cat(acc_len).numpy()
    n = vin.shape[0]
    assert n == (64 ** 4 + 64 ** 3 + 64 ** 2 if padded else 64 ** 4)
    want_dec, want_res = orc.decode_batch(vin.ravel(), np.arange(n + 1, dtype=np.int64) * 4,
                                          np.arange(n + 1, dtype=np.int64) * 3, chars,
                                          np.zeros(n, np.int32), np.full(n, int(padded), np.int32),
                                          3 * n)
    assert np.array_equal(want_res, vlen)
    want_dec = want_dec.reshape(n, 3)
    for k in np.unique(vlen):
        rows = vlen == k
        assert np.array_equal(vout[rows, :k], want_dec[rows, :k])
