"""Batched MIME decode (many documents, one launch sequence) against the oracle
and against the single-document call.

The first case is the error variant of the 256 MiB MIME workload: 256
documents of 1 MiB of data each, wrapped in 76-character CRLF lines, each
hit by a stray bad byte with p = 0.01 (seed 13, at least one forced),
decoded in one batched call. Then thousands of small documents with random
whitespace, errors, '=' placements and three alphabet modes, starting at any
alignment; a workspace sized for too few bytes; an empty batch.
"""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STD = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
URL = STD[:62] + b"-_"
TILE = 4096  # raw bytes per segment of the decode kernels


@pytest.fixture(scope="module")
def b64():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding
    binding.lib()
    yield binding
    assert binding.device_fault_flag() == 0


def run_batch(b64, docs, alphabets, aid, origin=0):
    """Concatenates the documents (after `origin` junk bytes), decodes them in
    one call; returns (results, per-document outputs, dst offsets)."""
    lens = np.array([d.size for d in docs], np.int64)
    off = (np.concatenate([[0], np.cumsum(lens)]) + origin).astype(np.int64)
    buf = np.concatenate([np.full(origin, ord("*"), np.uint8)] + list(docs)) if docs else \
        np.zeros(origin, np.uint8)
    src = torch.from_numpy(buf).cuda() if buf.size else torch.zeros(1, dtype=torch.uint8,
                                                                       device="cuda")
    d_off = torch.from_numpy(off).cuda()
    dst_off = b64.batch_offsets(d_off, alphabets, None, decode=True)
    dst = torch.full((int(dst_off[-1]) + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    res = b64.mime_decode_batch(src, d_off, dst, dst_off, alphabets,
                                torch.from_numpy(aid).cuda() if aid is not None else None)
    torch.cuda.synchronize()
    host = dst.cpu().numpy()
    ho = dst_off.cpu().numpy()
    assert (host[int(ho[-1]):] == 0xA5).all()
    outs = [host[ho[i]:ho[i + 1]] for i in range(len(docs))]
    return res.cpu().numpy(), outs


def test_config4_documents_batched(b64, orc):
    g = wl.rng(13)
    hit = g.random(256) < 0.01
    if not hit.any():
        hit[int(g.integers(0, 256))] = True
    docs, want = [], []
    for d in range(256):
        text = wl.mime_wrap(orc.encode(wl.random_bytes(1 << 20, 10_000 + d)))
        if hit[d]:
            text[int(g.integers(0, text.size))] = 0xFF
        docs.append(text)
        want.append(orc.decode(text, mime=True))
    res, outs = run_batch(b64, docs, [b64.Alphabet.standard()], None)
    for d in range(256):
        assert res[d] == want[d][0], d
        if res[d] >= 0:
            assert res[d] == 1 << 20
            assert np.array_equal(outs[d][:res[d]], want[d][1]), d
    assert (res < 0).sum() == hit.sum()


def make_docs(orc, count, seed):
    g = wl.rng(seed)
    modes = [(STD, True, False), (URL, False, False), (STD, True, True)]
    docs, aid = [], np.zeros(count, np.uint8)
    for i in range(count):
        a = int(g.integers(0, 3))
        aid[i] = a
        chars, padded, _ = modes[a]
        n = int(g.choice([0, 1, 2, 3, int(g.integers(0, 200)), int(g.integers(0, 20_000))]))
        text = orc.encode(wl.random_bytes(n, seed * 100_000 + i), chars, padded)
        kind = int(g.integers(0, 6))
        if kind == 0:
            text = wl.mime_wrap(text)
        elif kind == 1 and text.size:
            text = wl.insert_spaces(text, seed=seed + i, count=int(g.integers(1, 50)))
        elif kind == 2 and text.size:   # a bad byte or a misplaced '=' anywhere
            text = text.copy()
            text[int(g.integers(0, text.size))] = int(g.choice([0x00, 0x09, 0x3D, 0x7F, 0xC3]))
        elif kind == 3 and text.size:   # non-canonical last character
            t = text.copy()
            k = t.size
            while k and t[k - 1] == ord("="):
                k -= 1
            if k % 4 in (2, 3):
                t[k - 1] = chars[chars.index(bytes([t[k - 1]])) | 1]
            text = wl.mime_wrap(t)
        elif kind == 4:                 # long whitespace runs
            text = np.concatenate([np.frombuffer(b"\r\n" * int(g.integers(0, 3000)), np.uint8),
                                   text, np.frombuffer(b" \r\n", np.uint8)])
        docs.append(np.ascontiguousarray(text, np.uint8))
    return docs, aid, modes


@pytest.mark.parametrize("origin", [0, 7])
def test_mixed_documents_vs_oracle_and_single_calls(b64, orc, origin):
    docs, aid, modes = make_docs(orc, 3000, seed=21 + origin)
    alphs = [b64.Alphabet.standard(), b64.Alphabet.url(),
             b64.Alphabet.create(STD, True, canonical=True)]
    res, outs = run_batch(b64, docs, alphs, aid, origin)
    errors = 0
    for i, text in enumerate(docs):
        chars, padded, canonical = modes[aid[i]]
        want_r, want = orc.decode(text, chars, padded, mime=True, canonical=canonical)
        assert res[i] == want_r, (i, res[i], want_r, bytes(text[:40]))
        if want_r >= 0:
            assert np.array_equal(outs[i][:want_r], want), i
        else:
            errors += 1
        if i % 97 == 0 and text.size:   # same result as the single-document call
            r, out = b64.mime_decode(torch.from_numpy(text).cuda(), alphs[aid[i]])
            assert r == res[i]
            if r >= 0:
                assert np.array_equal(out.cpu().numpy(), outs[i][:r])
    assert errors > 300


def test_small_workspace_and_empty_batch(b64, orc):
    docs = [wl.mime_wrap(orc.encode(wl.random_bytes(50_000, 5 + i))) for i in range(8)]
    lens = np.array([d.size for d in docs], np.int64)
    off = torch.from_numpy(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)).cuda()
    src = torch.from_numpy(np.concatenate(docs)).cuda()
    alph = [b64.Alphabet.standard()]
    dst_off = b64.batch_offsets(off, alph, None, decode=True)
    dst = torch.zeros(int(dst_off[-1]) + 16, dtype=torch.uint8, device="cuda")
    # a workspace computed for far fewer bytes than the documents hold
    size = b64.lib().b64_mime_batch_workspace_size(8, 1000)
    ws = torch.empty(size, dtype=torch.uint8, device="cuda")
    res = b64.mime_decode_batch(src, off, dst, dst_off, alph, workspace=ws)
    assert (res.cpu().numpy() == b64.B64_E_INVAL).all()
    assert int(dst.sum()) == 0                       # nothing written
    res = b64.mime_decode_batch(src, off, dst, dst_off, alph)
    assert (res.cpu().numpy() == 50_000).all()
    # n == 0 enqueues nothing
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    b64.mime_decode_batch(torch.zeros(1, dtype=torch.uint8, device="cuda"), z, dst, z, alph)


def test_line_layout_documents(b64, orc):
    """Documents in the line layout (L from 4 to 1020, CR LF) over several
    segments, next to broken ones (a CR turned into data, a bad byte, a line
    one group longer, LF-only breaks), at odd and even offsets in the batch
    (the line path reads a segment where its copy put it for L >= 16 and, with
    CR LF, an even offset; other segments are moved first)."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    g = wl.rng(31)
    docs = []
    widths = (76, 64, 16, 20, 8, 1020, 76, 64, 36, 4)
    for i in range(60):
        L = widths[i // 6]
        n = int(g.integers(3 * TILE, 40_000))
        t = wl.mime_wrap(orc.encode(wl.random_bytes(n, 9000 + i)), line=L)
        kind = i % 6
        if kind == 1:
            crs = np.nonzero(t == 13)[0]
            t = t.copy()
            t[int(crs[g.integers(0, crs.size)])] = ord("A")
        elif kind == 2:
            t = t.copy()
            t[int(g.integers(0, t.size))] = 0x21
        elif kind == 3:
            p = (L + 2) * int(g.integers(1, t.size // (L + 2) - 1))
            t = np.concatenate([t[:p + L], np.frombuffer(b"QUJD", np.uint8), t[p + L:]])
        elif kind in (4, 5):  # LF-only lines (kind 5 with a CR in one break)
            t = wl.mime_wrap(orc.encode(wl.random_bytes(n, 9000 + i)), line=L, eol=b"\n")
            if kind == 5:
                lfs = np.nonzero(t == 10)[0]
                t = t.copy()
                t[int(lfs[g.integers(0, lfs.size)])] = 13
        docs.append(np.ascontiguousarray(t, np.uint8))
    for origin in (0, 5):
        res, outs = run_batch(b64, docs, [std], None, origin)
        for i, text in enumerate(docs):
            want_r, want = orc.decode(text, chars, True, mime=True)
            assert res[i] == want_r, (origin, i, res[i], want_r)
            if want_r >= 0:
                assert np.array_equal(outs[i][:want_r], want), i


def test_layout_broken_past_the_start_and_recorded_in_a_cuda_graph(b64, orc):
    """Every document shows its line layout in its first bytes; in the second
    batch one of them has a line a group longer in its third segment, which
    only the one-pass kernel can find (it then clears the word that lets the
    counting kernels return at once). The launch chain (a memset, then the
    layout kernel and five programmatic dependents) is recorded once in a CUDA
    graph per batch and replayed twice, each replay against the oracle."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    docs = [wl.mime_wrap(orc.encode(wl.random_bytes(12_000 + 997 * i, 7100 + i)))
            for i in range(8)]
    lines = [docs[5][k:k + 78] for k in range(0, docs[5].size, 78)]
    j = 9000 // 78  # a line of the third segment
    lines[j] = np.concatenate([lines[j][:76], np.frombuffer(b"QUJD", np.uint8), lines[j][76:]])
    broken = docs[:5] + [np.concatenate(lines)] + docs[6:]
    for batch in (docs, broken):
        # odd offsets: origin 3 and the documents' own lengths
        off = np.concatenate([[0], np.cumsum([d.size for d in batch])]).astype(np.int64) + 3
        buf = np.concatenate([np.full(3, ord("*"), np.uint8)] + batch)
        src = torch.from_numpy(buf).cuda()
        d_off = torch.from_numpy(off).cuda()
        dst_off = b64.batch_offsets(d_off, [std], None, decode=True)
        dst = torch.zeros(int(dst_off[-1]), dtype=torch.uint8, device="cuda")
        res = torch.zeros(len(batch), dtype=torch.int64, device="cuda")
        ws = torch.empty(b64.lib().b64_mime_batch_workspace_size(len(batch), int(off[-1] - off[0])),
                         dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        b64.mime_decode_batch(src, d_off, dst, dst_off, [std], None, res, ws, stream=s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b64.mime_decode_batch(src, d_off, dst, dst_off, [std], None, res, ws, stream=s)
        ho = dst_off.cpu().numpy()
        for _ in range(2):
            dst.zero_()
            res.fill_(-7)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            got, out = res.cpu().numpy(), dst.cpu().numpy()
            for i, text in enumerate(batch):
                want_r, want = orc.decode(text, chars, True, mime=True)
                assert got[i] == want_r, (i, got[i], want_r)
                if want_r >= 0:
                    assert np.array_equal(out[ho[i]:ho[i] + want_r], want), i
