"""Host-side helpers that need no GPU: the synthetic input recipes, the
serving driver's host output ring, and the benchmark's clock summary and
kernel-source digest."""
import os

import numpy as np
from conftest import ROOT

from paper_1910_05109_gb300 import serve
from paper_1910_05109_gb300 import workloads as wl


def test_mime_wrap_lines():
    text = np.frombuffer(b"A" * 1000, np.uint8)
    w = wl.mime_wrap(text).tobytes()
    lines = w.split(b"\r\n")
    assert all(len(x) == 76 for x in lines[:-1]) and len(lines[-1]) == 1000 - 76 * 13
    assert not w.endswith(b"\r\n")
    assert wl.mime_wrap(np.zeros(0, np.uint8)).size == 0
    assert wl.mime_wrap(np.frombuffer(b"A" * 76, np.uint8)).tobytes() == b"A" * 76


def test_insert_spaces_keeps_the_data():
    text = np.frombuffer(b"QUJDREVG" * 50, np.uint8)
    w = wl.insert_spaces(text, seed=3, count=100)
    assert w.size == text.size + 100
    kept = w[~np.isin(w, np.frombuffer(b"\r\n ", np.uint8))]
    assert np.array_equal(kept, text)


def test_varlen_lengths_recipe():
    lengths = wl.lognormal_lengths(100_000, 2, 1024, 1.5, 1, 1 << 20)
    assert lengths.min() >= 1 and lengths.max() <= 1 << 20
    assert set(np.unique(lengths % 3)) == {0, 1, 2}          # every padding case occurs
    assert 700 < np.median(lengths) < 1400


def test_poisson_requests_recipe():
    t, ops, sizes, pick = serve.poisson_requests(20_000, 2.0, 4, 5)
    assert 38_000 < t.size < 42_000 and np.all(np.diff(t) >= 0) and t[-1] <= 2.0
    assert 0.57 < ops.mean() < 0.63                          # 60% decode
    assert sizes.min() >= 4 and sizes.max() <= 16 << 20
    assert np.all(sizes[ops == 1] % 4 == 0)                  # whole groups for decode
    assert 30_000 < np.median(sizes) < 55_000                # median about 40 KiB
    assert np.all((pick >= 0) & (pick < 1))


def test_host_ring_wraps_and_releases_in_order():
    ring = serve.HostRing(1000)
    a = ring.take(0, 300)
    b = ring.take(1, 300)
    c = ring.take(2, 300)
    assert (a, b, c) == (0, 320, 640)
    assert ring.take(3, 100) is None                         # full
    ring.release(1)                                          # out of order: nothing freed yet
    assert ring.take(3, 100) is None
    ring.release(0)                                          # frees 0 and 1
    assert ring.take(3, 300) == 0                            # wraps to the front
    assert ring.take(4, 400) is None
    ring.release(2)
    ring.release(3)
    assert not ring.live and ring.take(5, 960) == 0
    assert ring.take(6, 2000) is None                        # larger than the ring


def test_host_ring_full_after_wrap_refuses():
    """After a wrap the newest slot may end exactly where the oldest begins;
    the ring is then full and must not hand out space after that end."""
    ring = serve.HostRing(1024)
    assert ring.take(0, 256) == 0
    assert ring.take(1, 256) == 256
    ring.release(0)                                          # oldest now starts at 256
    assert ring.take(2, 256) == 512
    assert ring.take(3, 256) == 768
    assert ring.take(4, 256) == 0                            # wraps; ends at 256 == oldest start
    assert ring.take(5, 64) is None                          # full: [256, 1024) is live


def test_host_ring_slots_never_overlap():
    g = np.random.default_rng(17)
    ring = serve.HostRing(4096)
    live = {}
    tag = 0
    for _ in range(20_000):
        if live and g.random() < 0.45:
            t = min(live)                                    # release in submission order...
            if g.random() < 0.3 and len(live) > 1:
                t = sorted(live)[1]                          # ...or one out of order
            ring.release(t)
            del live[t]
            continue
        size = int(g.choice([64, 128, 256, 512, 1024, 3000]))
        at = ring.take(tag, size)
        if at is not None:
            span = (size + 63) // 64 * 64
            assert 0 <= at and at + span <= 4096
            for a, s in live.values():
                assert at + span <= a or a + s <= at, (at, span, a, s)
            live[tag] = (at, span)
        tag += 1


def test_clock_sampler_summary_parses_nvidia_smi_lines():
    import bench
    c = bench.ClockSampler("GPU-0")
    c.lines = [
        "2070, 2070, 812.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2040, 2070, 1100.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable
        "garbage",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3, "source": "nvidia-smi"}
    c.lines = []
    assert c.summary()["samples"] == 0 and c.summary()["sm_mhz"] is None


def test_nvml_clock_sampler_summary():
    """The in-process sampler's summary: median SM clock over readable
    samples, the highest maximum clock, and every clock-event reason bit seen
    (power cap 0x4, hardware slowdown 0x8, software thermal 0x20, hardware
    thermal 0x40), named as in the nvidia-smi summary."""
    import bench
    c = bench.NvmlClockSampler("GPU-0")
    c.samples = [(2070, 2070, 0x0, 900_000), (1980, 2070, 0x4, 1_390_000),
                 (2055, 2070, 0x1, 1_000_000), (0, 2070, 0x0, 0)]     # last one unreadable
    s = c.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["source"] == "nvml"
    c.samples = [(1500, 2070, 0x8 | 0x40 | 0x20, 1)]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                      "sw_thermal_slowdown"]
    c.samples = []
    assert c.summary()["samples"] == 0 and c.summary()["sm_mhz"] is None
    assert not bench.NvmlClockSampler("GPU-no-such-device").open()   # no NVML, or no such GPU


def test_kernel_digest_ignores_comments_only(tmp_path, monkeypatch):
    """The digest that ties a committed DRAM-traffic figure to a kernel's
    sources changes with the code and not with its comments."""
    import shutil
    import bench
    src = os.path.join(ROOT, "paper_1910_05109_gb300", "csrc")
    dst = tmp_path / "paper_1910_05109_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in ("b64_encode.cu", "b64_decode.cu", "b64_device.cuh", "b64_internal.h"):
        shutil.copy(os.path.join(src, name), dst / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = {k: bench.source_digest(k) for k in bench.KERNEL_SOURCES}
    enc = dst / "b64_encode.cu"
    text = enc.read_text()
    enc.write_text("// a new first line of comment\n/* and a block\n   comment */\n" +
                   text.replace("// ", "//  ") + "\n\n// trailing note\n")
    assert {k: bench.source_digest(k) for k in bench.KERNEL_SOURCES} == before
    enc.write_text(text.replace("kStages", "kStagez"))
    after = {k: bench.source_digest(k) for k in bench.KERNEL_SOURCES}
    assert after["encode_tma_kernel"] != before["encode_tma_kernel"]
    assert after["decode_body_kernel"] == before["decode_body_kernel"]
    assert bench.code_only('a = "/* x */ // y"; /* z */ b = \'/\'; // w') == \
        'a = "/* x */ // y";   b = \'/\';'


def test_reference_sample_keeps_the_run_near_a_minute():
    import bench
    rate, per_byte = 9e9, 4.67                      # bytes consumed per second / per sample byte
    big = bench.reference_sample_bytes(rate, per_byte, steps=3, warmup=3)
    assert big == (128 << 20) // 3 * 3                # few steps: the 128 MiB cap
    for steps in (100, 1000, 5000):
        s = bench.reference_sample_bytes(rate, per_byte, steps=steps, warmup=5)
        assert s % 3 == 0 and (1 << 20) - 3 <= s <= 128 << 20
        run_s = (steps + 5) * s * per_byte / rate
        assert run_s <= 61 or s == (1 << 20) // 3 * 3
    assert bench.reference_sample_bytes(1e6, per_byte, steps=10_000, warmup=5) == (1 << 20) // 3 * 3


def _unbound_globals(path):
    """Names that a function of the module at `path` reads as globals but that
    neither the module's top level nor the builtins define."""
    import builtins
    import symtable
    top = symtable.symtable(open(path).read(), path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    defined |= set(dir(builtins)) | {"__file__", "__name__", "__doc__"}
    missing = []

    def walk(t):
        for s in t.get_symbols():
            if t.get_type() != "module" and s.is_global() and s.is_referenced() \
                    and s.get_name() not in defined:
                missing.append(f"{t.get_name()}:{s.get_name()}")
        for c in t.get_children():
            walk(c)

    walk(top)
    return missing


def test_python_sources_read_no_unbound_names():
    # the GPU-only branches of bench.py and the package never run on this
    # host; a name read there that nothing defines would only show on the GPU
    pkg = os.path.join(ROOT, "paper_1910_05109_gb300")
    files = [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    files += [os.path.join(pkg, f) for f in sorted(os.listdir(pkg)) if f.endswith(".py")]
    for f in files:
        assert _unbound_globals(f) == [], f
