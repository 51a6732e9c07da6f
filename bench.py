"""Benchmark: base64 encode + strict decode of large single buffers on GB300.

One step = the whole hot path over one batch of input: encode 1 GiB of
uniform random bytes with the standard table, strict-decode the result, then
the same with the base64url table (padded) swapped in at run time. The metric
is input GB/s (bytes consumed by encode plus characters consumed by decode,
per second), next to an on-device D2D memcpy of the same bytes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run, one replica of the workload per GPU
(the buffers are independent; no data-path collective): weak scaling.
`--impl reference` times the oracle (the plain scalar C codec) on the host's
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode/decode input GB/s vs on-device D2D memcpy GB/s; batched p99 latency"
N_BYTES = 1 << 30
SEED = 1
WORKLOAD = ("large single buffer: 1 GiB uniform random bytes (seed 1); encode then strict "
            "decode, standard table then base64url table (padded) swapped at run time")


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


# The source files each profiled kernel is built from.
KERNEL_SOURCES = {
    "encode_tma_kernel": ("b64_encode.cu", "b64_device.cuh"),
    "decode_body_kernel": ("b64_decode.cu", "b64_device.cuh", "b64_internal.h"),
}


def code_only(text: str) -> str:
    """C/C++/CUDA source without its comments, trailing blanks and blank lines
    (string and character literals kept), so that an edit of comments alone
    leaves a kernel's digest unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == "/" and text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif c == "/" and text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def source_digest(kernel: str) -> str:
    """Digest of the code (comments aside) of the files `kernel` is built from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1910_05109_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(d, name), encoding="utf-8") as f:
            h.update(name.encode() + code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str) -> dict | None:
    """DRAM traffic per input byte of `kernel` from the committed ncu summary,
    if it was taken on the kernel's current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    digest = source_digest(kernel)
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(x.split("=", 1) for x in line.split())
        if kv.get("kernel") == kernel and kv.get("sources") == digest:
            return {"bytes_per_input_byte": float(kv["dram_bytes_per_input_byte"])}
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "source": "nvidia-smi"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}


class NvmlClockSampler:
    """SM clock, power and clock-event reasons sampled in-process every
    `interval_s` through NVML's read-only queries (the driver's
    libnvidia-ml, called through ctypes), from a thread, while running.
    Changes no GPU setting."""

    CLOCK_SM = 1
    # clock-event reason bits (nvml.h) -> names used in the bench line
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_id: str, interval_s: float = 0.0005):
        self.gpu_id = gpu_id
        self.interval_s = interval_s
        self.samples: list[tuple[int, int, int, int]] = []   # (sm MHz, max MHz, reasons, mW)
        self._stop = threading.Event()
        self._thread = None
        self._nvml = None
        self._dev = None

    def open(self) -> bool:
        """Loads NVML and finds the device; False if either is unavailable."""
        import ctypes
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return False
            dev = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByUUID(self.gpu_id.encode(), ctypes.byref(dev)) != 0:
                return False
            self._reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            return False
        mx = ctypes.c_uint()
        nv.nvmlDeviceGetMaxClockInfo(dev, self.CLOCK_SM, ctypes.byref(mx))
        self._nvml, self._dev, self._max = nv, dev, mx.value
        self._sm, self._rs, self._pw = ctypes.c_uint(), ctypes.c_ulonglong(), ctypes.c_uint()
        self._power = 0
        return True

    def _sample(self):
        # two queries a sample (SM clock, event reasons); power every 16th
        import ctypes
        nv, dev = self._nvml, self._dev
        if nv.nvmlDeviceGetClockInfo(dev, self.CLOCK_SM, ctypes.byref(self._sm)) != 0:
            return
        self._reasons_fn(dev, ctypes.byref(self._rs))
        if len(self.samples) % 16 == 0:
            nv.nvmlDeviceGetPowerUsage(dev, ctypes.byref(self._pw))
            self._power = self._pw.value
        self.samples.append((self._sm.value, self._max, self._rs.value, self._power))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            self._stop.wait(self.interval_s)

    def __enter__(self):
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._thread.join(timeout=2)
        self._sample()                   # one reading at the end of the region

    def summary(self) -> dict:
        sm = [s[0] for s in self.samples if s[0] > 0]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "source": "nvml"}
        reasons = set()
        for s in self.samples:
            for bit, name in self.REASONS.items():
                if s[2] & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvml",
                "interval_ms": self.interval_s * 1e3,
                "power_w_median": statistics.median(s[3] for s in self.samples) / 1e3}


def clock_sampler(gpu_id: str):
    """In-process NVML sampling where NVML loads, else nvidia-smi's."""
    s = NvmlClockSampler(gpu_id)
    return s if s.open() else ClockSampler(gpu_id)


def gpu_uuid(dev=0) -> str:
    import torch
    u = str(torch.cuda.get_device_properties(dev).uuid)
    return u if u.startswith("GPU-") else f"GPU-{u}"


# ---------------------------------------------------------------- CPU baseline (oracle)

def oracle_pass(data: np.ndarray, threads: int) -> tuple[int, float]:
    """The oracle over one step's work (encode + decode, both tables), with the
    buffer split into `threads` slices at multiples of 3 bytes (each slice's
    encoding is then a whole number of 4-character groups). Returns (input
    bytes consumed, seconds)."""
    import oracle
    tables = (oracle.standard_alphabet(), oracle.url_alphabet())
    n = data.size
    per = max(3, (n // threads) // 3 * 3)
    cuts = list(range(0, n, per)) + [n]
    slices = [data[cuts[i]:cuts[i + 1]] for i in range(len(cuts) - 1)]
    consumed = 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for alph in tables:
            enc = list(ex.map(lambda s: oracle.encode(s, alph, True), slices))
            dec = list(ex.map(lambda e: oracle.decode(e, alph, True), enc))
            assert sum(r for r, _ in dec) == n
            consumed += n + sum(e.size for e in enc)
    return consumed, time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu's, else the platform's)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(data: np.ndarray) -> dict:
    cores = len(os.sched_getaffinity(0))
    consumed, sec = 0, 0.0
    for _ in range(3):
        c, s = oracle_pass(data, cores)
        consumed, sec = consumed + c, sec + s
    one = data[: 64 << 20]
    c1, s1 = oracle_pass(one, 1)
    return {"value": consumed / sec / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": (f"three full steps (1 GiB each; encode+decode, standard and url tables) "
                       f"split over {cores} threads at 3-byte boundaries; {sec:.2f} s wall"),
            "value_1core": c1 / s1 / 1e9,
            "sample_1core": "first 64 MiB of the same buffer, one thread, both tables",
            "cpu": cpu_model()}


# ---------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def emit(obj: dict):
    print(json.dumps(obj), flush=True)


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank_step: float, world_size: int, steps: int, max_ms: float) -> float:
    """Whole-job GB/s: what every rank processed, over the slowest rank's time."""
    return bytes_per_rank_step * world_size * steps / (max_ms / 1e3) / 1e9


# ---------------------------------------------------------------- reference arm

def reference_sample_bytes(consumed_per_s: float, consumed_per_byte: float, steps: int,
                           warmup: int, budget_s: float = 60.0) -> int:
    """Bytes of the 1 GiB buffer one reference step takes: as many as let the
    warm-up and timed steps finish in about budget_s at the probed rate,
    between 1 MiB and 128 MiB, a multiple of 3."""
    per_step_s = budget_s / max(1, steps + warmup)
    want = int(consumed_per_s * per_step_s / consumed_per_byte)
    return max(1 << 20, min(128 << 20, want)) // 3 * 3


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1910_05109_gb300 import workloads as wl
    data = wl.random_bytes(N_BYTES, SEED)
    cores = len(os.sched_getaffinity(0))
    # Each step: a bounded sample (the start of the 1 GiB buffer) of the
    # step's workload, sized from a probe pass so that the run takes about a
    # minute whatever --steps is.
    probe = data[: 16 << 20]
    c, s = oracle_pass(probe, cores)
    sample = data[: reference_sample_bytes(c / s, c / probe.size, args.steps, args.warmup)]
    for _ in range(args.warmup):
        oracle_pass(sample, cores)
    total, sec = 0, 0.0
    for _ in range(args.steps):
        c, s = oracle_pass(sample, cores)
        total += c
        sec += s
    value = total / sec / 1e9
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
          "config": {"workload": WORKLOAD, "bytes": N_BYTES, "sample_bytes": sample.size},
          "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                           "cpu": cpu_model(),
                           "sample": f"first {sample.size} bytes of the 1 GiB buffer per "
                                     f"step, both tables, split over {cores} threads"},
          "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                  "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1910_05109_gb300 import build as gpu_build
    if rank == 0 or ws == 1:
        gpu_build.build()
    if ws > 1:
        dist.barrier()
    from paper_1910_05109_gb300 import binding as b64
    from paper_1910_05109_gb300 import workloads as wl

    n = args.bytes
    data = wl.random_bytes(n, SEED)
    src = torch.from_numpy(data).to(dev)
    std = b64.Alphabet.standard()
    url = b64.Alphabet.create(std.chars()[0][:62] + b"-_", True)
    m = b64.encoded_length(n, True)
    enc = {k: torch.empty(m, dtype=torch.uint8, device=dev) for k in ("std", "url")}
    dec = {k: torch.empty(b64.decoded_max_length(m), dtype=torch.uint8, device=dev)
           for k in ("std", "url")}
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    tables = (("std", std), ("url", url))
    stream = torch.cuda.current_stream()

    def step(ev=None):
        for i, (k, a) in enumerate(tables):
            if ev is not None:
                ev[4 * i].record(stream)
            b64.encode(src, a, enc[k], stream)
            if ev is not None:
                ev[4 * i + 1].record(stream)
                ev[4 * i + 2].record(stream)
            b64.decode_async(enc[k], dec[k], res[i:i + 1], a, stream)
            if ev is not None:
                ev[4 * i + 3].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # Round trip and alphabet swap checked once (not timed).
    assert int(res[0]) == n and int(res[1]) == n
    assert torch.equal(dec["std"][:n], src) and torch.equal(dec["url"][:n], src)
    assert not torch.equal(enc["std"], enc["url"])

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_id if gpu_id.startswith("GPU-") else f"GPU-{gpu_id}"
    with clock_sampler(gpu_id) as clocks:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(K):
            step(evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    ms = start.elapsed_time(stop)
    t_enc = [e[4 * i].elapsed_time(e[4 * i + 1]) for e in evs for i in range(2)]
    t_dec = [e[4 * i + 2].elapsed_time(e[4 * i + 3]) for e in evs for i in range(2)]
    ms = max_over_ranks(ms, dev)
    assert int(res[0]) == n and int(res[1]) == n

    # D2D memcpy of the same bytes (torch copy_ issues cudaMemcpyAsync D2D).
    def memcpy_ms(nbytes: int, reps: int = 20) -> float:
        a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        bb = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        for _ in range(3):
            bb.copy_(a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(reps):
            e0.record(stream)
            bb.copy_(a)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        del a, bb
        return statistics.median(times)

    mc_n, mc_m = memcpy_ms(n), memcpy_ms(m)
    enc_ms, dec_ms = statistics.median(t_enc), statistics.median(t_dec)
    enc_avg, dec_avg = sum(t_enc) / len(t_enc), sum(t_dec) / len(t_dec)

    # End to end through the public API with host buffers: the host codec
    # (b64_host_encode / b64_host_decode) takes page-locked host input,
    # copies it to the device in pieces, codes them and copies the output
    # back, the pieces' copies and kernels overlapped on its streams; both
    # tables, encode then decode of the encoded text. Each call returns when
    # its output is in host memory, so the host clock times the step.
    if args.no_e2e:
        return finish(args, locals())
    h_src = torch.from_numpy(data).pin_memory()
    h_txt = torch.empty(m, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(b64.decoded_max_length(m), dtype=torch.uint8).pin_memory()
    codec = b64.HostCodec(args.piece_bytes, args.host_streams)
    h_res = [0, 0]

    def e2e_step():
        for i, (k, a) in enumerate(tables):
            codec.encode(h_src, h_txt, a)
            h_res[i] = codec.decode(h_txt, h_out, a)

    # Each step timed on the host clock; the median step is reported (the
    # host link is shared with other work on the node, so single steps can
    # stall), the mean and the extremes beside it.
    e2e_steps = max(3, min(10, K // 50))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()  # the ranks' host links are busy at the same time
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = max_over_ranks(statistics.median(e2e_times), dev)  # the slowest rank's median step
    assert h_res == [n, n] and torch.equal(h_out[:n], h_src)
    codec.close()
    del h_src, h_txt, h_out
    return finish(args, locals())


def finish(args, v):
    import torch.distributed as dist
    ws, rank, K, n, m, ms = v["ws"], v["rank"], v["K"], v["n"], v["m"], v["ms"]
    enc_ms, dec_ms, enc_avg, dec_avg = v["enc_ms"], v["dec_ms"], v["enc_avg"], v["dec_avg"]
    mc_n, mc_m, data, clocks = v["mc_n"], v["mc_m"], v["data"], v["clocks"]
    e2e_ms = v.get("e2e_ms")

    step_in = 2 * (n + m)                       # input bytes per step (both tables)
    value = job_throughput(step_in, ws, K, ms)
    pk = peaks()
    enc_alg = n + m                             # algorithmic bytes per encode launch
    dec_alg = m + n                             # per decode call (reads m, writes n)
    dominant = "decode" if dec_avg >= enc_avg else "encode"
    dom_ms = dec_avg if dominant == "decode" else enc_avg
    achieved = (dec_alg if dominant == "decode" else enc_alg) / (dom_ms / 1e3) / 1e9
    kname = "decode_body_kernel" if dominant == "decode" else "encode_tma_kernel"
    tr = profiled_traffic(kname)
    traffic = None
    if tr is not None:
        traffic = tr["bytes_per_input_byte"] * (m if dominant == "decode" else n)

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_BYTES else f"{n} bytes (profiling case)",
                   "bytes": n, "encoded_bytes": m,
                   "tables": ["standard (Table 1)", "base64url, padded"],
                   "l2": "inputs (1 GiB / 1.43 GB) larger than L2; no flush",
                   "parallelism": f"replicas x{ws}"},
        "encode_gbps": n / (enc_ms / 1e3) / 1e9,
        "decode_gbps": m / (dec_ms / 1e3) / 1e9,
        "memcpy_gbps": {"encode_input": n / (mc_n / 1e3) / 1e9,
                        "decode_input": m / (mc_m / 1e3) / 1e9},
        "frac_of_memcpy": {"encode": mc_n / enc_ms, "decode": mc_m / dec_ms},
        "base64_gbps": {"encode": m / (enc_ms / 1e3) / 1e9, "decode": m / (dec_ms / 1e3) / 1e9},
        "dram_gbps": {"encode": enc_alg / (enc_ms / 1e3) / 1e9,
                      "decode": dec_alg / (dec_ms / 1e3) / 1e9,
                      "memcpy": 2 * n / (mc_n / 1e3) / 1e9},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "peak_source": pk["source"], "traffic": traffic},
        "e2e": None if e2e_ms is None else {
            # all ranks' input over the slowest rank's median step, like `value`
            "value": job_throughput(step_in, ws, 1, e2e_ms), "unit": "GB/s",
            "h2d_bytes_per_step": ws * 2 * (n + m), "d2h_bytes_per_step": ws * 2 * (m + n),
            "api": "b64_host_encode + b64_host_decode, page-locked host buffers",
            "step_ms": {"median": e2e_ms, "mean": statistics.mean(v["e2e_times"]),
                        "min": min(v["e2e_times"]), "max": max(v["e2e_times"]),
                        "steps": len(v["e2e_times"])},
            "host_codec": {"piece_bytes": args.piece_bytes or 48 << 20,
                           "streams": args.host_streams or 3}},
        # per step and table: encode; decode = result init, body, tail
        "gpu_launches": 8 * K,
        "clocks": clocks.summary(),
    }
    if ws == 1 and not args.no_workloads:
        out["workloads"] = other_workloads(args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(data)
    if rank == 0:
        emit(out)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- other workloads

# The default run's settings for the other workloads: enough timed calls for
# a few dozen clock samples, the serving stream at its stated rate for 10 s,
# then a short sweep of higher rates for the engine's capacity.
WORKLOAD_MIN_STEPS = 100
SERVE_DURATION_S = 10.0
SERVE_SWEEP = (40_000.0, 80_000.0, 120_000.0, 160_000.0)


def other_workloads(args) -> dict:
    """The batched-strings, MIME and serving workloads, measured after the
    single-buffer step in the same process (one GPU). A workload that fails
    is reported with its error instead of its figures."""
    import copy
    import traceback
    wargs = copy.copy(args)
    wargs.steps = max(args.steps, WORKLOAD_MIN_STEPS)
    wargs.warmup = max(args.warmup, 3)
    out = {}
    for name, fn in (("batch", lambda: batch_workload(wargs)),
                     ("mime", lambda: mime_workload(wargs)),
                     ("serve", lambda: serve_workload(wargs, args.rate, SERVE_DURATION_S,
                                                      SERVE_SWEEP))):
        try:
            out[name] = fn()
            out[name]["steps"] = wargs.steps if name != "serve" else out[name]["requests"]
        except Exception as e:  # reported, not hidden: the figures are then absent
            out[name] = {"error": f"{type(e).__name__}: {e}",
                         "trace": traceback.format_exc(limit=3)}
    return out


# ---------------------------------------------------------------- batched workload

def batch_workload(args) -> dict:
    """100,000 strings (lognormal lengths, median 1 KiB, sigma 1.5, 1 B..1 MiB,
    seed 2), 50/50 standard-padded / url-unpadded (seed 13): one persistent
    launch sequence per batch (CUDA-graph replay, autotuned tile) against one
    launch per string, identical output required. Returns the measurements."""
    import torch
    from paper_1910_05109_gb300 import autotune
    from paper_1910_05109_gb300 import binding as b64
    from paper_1910_05109_gb300 import build as gpu_build
    from paper_1910_05109_gb300 import workloads as wl
    from paper_1910_05109_gb300.batch import BatchCodec

    gpu_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    data, off = wl.varlen_strings(args.strings, seed=2, median=1024, sigma=1.5, lo=1, hi=1 << 20)
    aid = wl.bernoulli(args.strings, seed=13).astype(np.uint8)
    n = args.strings
    alphs = [b64.Alphabet.standard(), b64.Alphabet.url()]
    d_src = torch.from_numpy(data).to(dev)
    d_off = torch.from_numpy(off).to(dev)
    d_aid = torch.from_numpy(aid).to(dev)
    total_in = int(off[-1])

    align16 = args.batch_layout == "align16"
    # the strings' encoded lengths (packed output offsets)
    enc_len = b64.batch_offsets(d_off, alphs, d_aid, decode=False)
    enc_len = enc_len[1:] - enc_len[:-1]
    total_enc = int(enc_len.sum())

    def time_codec(codec, steps):
        for _ in range(max(args.warmup, 3)):
            codec.run()
        codec.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(codec.stream)
        for _ in range(steps):
            codec.run()
        e1.record(codec.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {}
    texts = None
    clocks = clock_sampler(gpu_uuid(dev)).__enter__()   # sampled over both ops' timed loops
    for op in ("encode", "decode"):
        if op == "encode":
            src, src_off = d_src, d_off
        else:
            src, src_off = texts
        codec = BatchCodec(op, n, src.numel(), alphs, dev, align16=align16)
        cap = codec.load(src, src_off, d_aid)
        # output offsets (b64_batch_offsets), timed on their own
        with torch.cuda.stream(codec.stream):
            for _ in range(3):
                b64.batch_offsets(codec.src_off, alphs, codec.alph_id[:n], decode=op == "decode",
                                  stream=codec.stream)
            o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            o0.record(codec.stream)
            for _ in range(10):
                b64.batch_offsets(codec.src_off, alphs, codec.alph_id[:n], decode=op == "decode",
                                  stream=codec.stream)
            o1.record(codec.stream)
        o1.synchronize()
        offsets_ms = o0.elapsed_time(o1) / 10
        if args.tile_units:
            units, timings = args.tile_units, {}
        else:
            units, timings = autotune.best_units(op, codec.src, codec.src_off, codec.dst,
                                                 codec.dst_off, alphs, codec.alph_id[:n])
        codec.tile_units = units
        batch_ms = time_codec(codec, args.steps)
        with torch.cuda.stream(codec.stream):
            codec.dst.zero_()   # the bytes between aligned strings stay zero
        codec.run()
        codec.synchronize()
        res = codec.results[:n].clone()
        batch_out = codec.dst[:cap].clone()
        in_bytes = src.numel()
        # the same batch with packed output offsets (the other layout), for comparison
        pcodec = BatchCodec(op, n, src.numel(), alphs, dev, tile_units=units, align16=False)
        pcap = pcodec.load(src, src_off, d_aid)
        packed_ms = time_codec(pcodec, args.steps)
        # algorithmic bytes: the strings read, their encoded / decoded bytes written
        alg = in_bytes + (total_enc if op == "encode" else total_in)
        roof = {"bound": "hbm", "achieved": alg / (batch_ms / 1e3) / 1e9,
                "peak": peaks()["hbm_gbs"], "unit": "GB/s", "traffic_alg_bytes": alg}
        roof["frac"] = roof["achieved"] / roof["peak"]
        packed = {"batch_ms": packed_ms, "input_gbps": in_bytes / (packed_ms / 1e3) / 1e9,
                  "roofline_frac": alg / (packed_ms / 1e3) / 1e9 / roof["peak"]}
        if op == "encode":
            assert torch.equal(res, enc_len)
            texts = (pcodec.dst[:pcap].clone(), pcodec.dst_off.clone())   # packed text
        else:
            assert torch.equal(res, d_off[1:] - d_off[:-1])
        assert torch.equal(pcodec.results[:n], res)
        del pcodec

        if args.no_per_string:
            out[op] = {"batch_ms": batch_ms, "input_gbps": in_bytes / (batch_ms / 1e3) / 1e9,
                       "roofline": roof, "tile_units": units,
                       "tile": autotune.describe(units), "autotune_ms": timings,
                       "offsets_ms": offsets_ms, "packed_offsets": packed}
            continue
        # One launch per string through the single-buffer calls.
        hoff = codec.src_off.cpu().numpy()
        hdo = codec.dst_off.cpu().numpy()
        haid = aid
        per_dst = torch.zeros_like(batch_out)
        per_res = torch.zeros(n, dtype=torch.int64, device=dev)
        stream = torch.cuda.current_stream()

        def per_string():
            for i in range(n):
                a, b_ = int(hoff[i]), int(hoff[i + 1])
                if op == "encode":
                    if b_ > a:
                        b64.encode(src[a:b_], alphs[haid[i]], per_dst[int(hdo[i]):int(hdo[i + 1])],
                                   stream)
                else:
                    b64.decode_async(src[a:b_], per_dst[int(hdo[i]):int(hdo[i + 1])],
                                     per_res[i:i + 1], alphs[haid[i]], stream)

        per_string()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        per_string()
        e1.record(stream)
        e1.synchronize()
        eager_ms = (time.perf_counter() - t0) * 1e3
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.graph(g, stream=gs):
            stream_saved = stream
            stream = gs
            per_string()
            stream = stream_saved
        with torch.cuda.stream(gs):              # replay() launches on the current stream
            g.replay()
            torch.cuda.synchronize()
            e0.record(gs)
            g.replay()
            e1.record(gs)
        e1.synchronize()
        graph_ms = e0.elapsed_time(e1)
        if op == "encode":
            # both outputs start from zeros, and neither call writes between strings
            identical = bool(torch.equal(per_dst, batch_out))
        else:
            # same results; decoded bytes compared string by string (a string's
            # capacity can exceed its decoded length)
            identical = bool(torch.equal(per_res, res))
            hres = res.cpu().numpy()
            pb, bb = per_dst.cpu().numpy(), batch_out.cpu().numpy()
            for i in range(n):
                o = int(hdo[i])
                if not np.array_equal(pb[o:o + hres[i]], bb[o:o + hres[i]]):
                    identical = False
                    break
        del g
        out[op] = {"batch_ms": batch_ms, "input_gbps": in_bytes / (batch_ms / 1e3) / 1e9,
                   "roofline": roof, "tile_units": units, "tile": autotune.describe(units),
                   "autotune_ms": timings,
                   "offsets_ms": offsets_ms,
                   "per_string_eager_ms": eager_ms, "per_string_graph_ms": graph_ms,
                   "speedup_vs_eager": eager_ms / batch_ms,
                   "speedup_vs_graph": graph_ms / batch_ms, "identical_output": identical,
                   "packed_offsets": packed,
                   "launches_per_batch": 2 if op == "encode" else 3}
    clocks.__exit__(None, None, None)
    step_ms = out["encode"]["batch_ms"] + out["decode"]["batch_ms"]
    step_in = total_in + texts[0].numel()
    return {"value": step_in / (step_ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": step_ms,
            "config": {"workload": f"{n} strings, lognormal lengths (median 1 KiB, sigma 1.5, "
                                   "1 B..1 MiB, seed 2), 50/50 standard-padded / url-unpadded",
                       "input_bytes": total_in, "encoded_bytes": int(texts[0].numel()),
                       "output_offsets": ("b64_batch_offsets with B64_OFFSETS_ALIGN16 (16-byte "
                                          "aligned string starts); packed offsets timed beside"
                                          if align16 else "b64_batch_offsets, packed"),
                       "l2": f"batch input and output ({total_in / 1e6:.0f} MB + "
                             f"{int(texts[0].numel()) / 1e6:.0f} MB) larger than L2; no flush"},
            "encode": out["encode"], "decode": out["decode"], "clocks": clocks.summary(),
            # per step: encode results + tile kernel; decode tile + finalize kernel
            "gpu_launches": 4 * args.steps}


def run_batch(args):
    r = batch_workload(args)
    emit({"metric": METRIC, "workload": "batched varlen strings", "value": r["value"],
          "unit": r["unit"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": r["config"],
          "encode": r["encode"], "decode": r["decode"], "clocks": r["clocks"],
          "gpu_launches": r["gpu_launches"]})


# ---------------------------------------------------------------- MIME workload

# The kernels of one MIME decode call, and how many launches it makes.
MIME_KERNELS = ("mime decode call (mime_status_init_kernel, mime_onepass_kernel; "
                "mime_count_kernel, mime_scan_kernel, mime_decode_kernel, which return at once "
                "when the line layout holds; mime_finalize_kernel)")
MIME_LAUNCHES_PER_CALL = 6

def mime_workload(args) -> dict:
    """256 MiB of seed-3 random bytes, encoded with the standard table and
    wrapped as 76-character lines with CRLF (367,332,730 bytes), decoded with
    CR/LF/space skipped; against a D2D memcpy of the same bytes. Returns the
    measurements."""
    import torch
    from paper_1910_05109_gb300 import binding as b64
    from paper_1910_05109_gb300 import build as gpu_build
    from paper_1910_05109_gb300 import workloads as wl

    gpu_build.build()
    torch.cuda.set_device(0)
    n = args.mime_bytes
    data = wl.random_bytes(n, 3)
    d = torch.from_numpy(data).cuda()
    text = wl.mime_wrap(b64.encode(d, b64.Alphabet.standard()).cpu().numpy())
    src = torch.from_numpy(text).cuda()
    m = src.numel()
    dst = torch.empty(b64.decoded_max_length(m), dtype=torch.uint8, device="cuda")
    res = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = b64.mime_workspace(m)
    std = b64.Alphabet.standard()
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        b64.mime_decode_async(src, dst, res, std, ws)
    torch.cuda.synchronize()
    assert int(res.item()) == n and torch.equal(dst[:n], d)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clock_sampler(gpu_uuid()) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            b64.mime_decode_async(src, dst, res, std, ws)
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cp = torch.empty_like(src)
    for _ in range(3):
        cp.copy_(src)
    e0.record(stream)
    for _ in range(20):
        cp.copy_(src)
    e1.record(stream)
    e1.synchronize()
    mc = e0.elapsed_time(e1) / 20
    # The same data as 256 documents of n / 256 bytes each (wrapped separately),
    # decoded in one batched call (b64_mime_decode_batch).
    per = n // 256
    docs = [wl.mime_wrap(b64.encode(d[i * per:(i + 1) * per], std).cpu().numpy())
            for i in range(256)]
    doff = torch.from_numpy(np.concatenate([[0], np.cumsum([x.size for x in docs])])
                            .astype(np.int64)).cuda()
    dsrc = torch.from_numpy(np.concatenate(docs)).cuda()
    ddoff = b64.batch_offsets(doff, [std], None, decode=True)
    ddst = torch.empty(int(ddoff[-1]) + 16, dtype=torch.uint8, device="cuda")
    dres = torch.empty(256, dtype=torch.int64, device="cuda")
    dws = torch.empty(b64.lib().b64_mime_batch_workspace_size(256, dsrc.numel()),
                      dtype=torch.uint8, device="cuda")
    for _ in range(3):
        b64.mime_decode_batch(dsrc, doff, ddst, ddoff, [std], None, dres, dws)
    torch.cuda.synchronize()
    assert (dres == per).all()
    e0.record(stream)
    for _ in range(args.steps):
        b64.mime_decode_batch(dsrc, doff, ddst, ddoff, [std], None, dres, dws)
    e1.record(stream)
    e1.synchronize()
    docs_ms = e0.elapsed_time(e1) / args.steps
    del dsrc, ddst, dws
    pk = peaks()
    dram = (m + n) / (ms / 1e3) / 1e9
    return {"value": m / (ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "config": {"workload": f"{n} random bytes (seed 3), standard table, 76-char lines "
                                   "+ CRLF, no trailing CRLF", "input_bytes": m,
                       "output_bytes": n,
                       "l2": f"input and output ({m / 1e6:.0f} MB + {n / 1e6:.0f} MB) larger "
                             "than L2; no flush"},
            "memcpy_gbps": m / (mc / 1e3) / 1e9, "frac_of_memcpy": mc / ms,
            # the whole call (count, scan, decode and finalize kernels) against the
            # bytes it must move: the wrapped input read, the decoded bytes written
            "roofline": {"bound": "hbm", "kernel": MIME_KERNELS, "achieved": dram,
                         "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": dram / pk["hbm_gbs"],
                         "peak_source": pk["source"], "traffic": None},
            "clocks": clocks.summary(),
            "documents_batched": {"documents": 256, "bytes_each": per,
                                  "input_bytes": int(doff[-1]), "ms": docs_ms,
                                  "input_gbps": int(doff[-1]) / (docs_ms / 1e3) / 1e9},
            "gpu_launches": MIME_LAUNCHES_PER_CALL * args.steps}


def run_mime(args):
    r = mime_workload(args)
    emit({"metric": METRIC, "workload": "MIME line-wrapped decode", "value": r["value"],
          "unit": r["unit"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": r["config"],
          **{k: r[k] for k in ("memcpy_gbps", "frac_of_memcpy", "roofline", "clocks",
                               "documents_batched", "gpu_launches")}})


# ---------------------------------------------------------------- Table 2 sizes

def run_table2(args):
    """Decode (and encode) at the sizes of the paper's Table 2 files (141,020;
    247,222; 2,357; 34,904,444 bytes of binary data; random bytes stand in,
    as the codec is content-insensitive). Per size: the base64 text of the
    data is decoded from device memory, one call at a time (eager launches)
    and as 100 calls recorded in a CUDA graph; GB/s counts base64 bytes, the
    paper's unit, beside a D2D memcpy of the same text. Everything fits in
    L2 except the largest size."""
    import torch
    from paper_1910_05109_gb300 import binding as b64
    from paper_1910_05109_gb300 import build as gpu_build
    from paper_1910_05109_gb300 import workloads as wl

    gpu_build.build()
    torch.cuda.set_device(0)
    std = b64.Alphabet.standard()
    stream = torch.cuda.Stream()
    rows = []
    launches = 0
    clocks = clock_sampler(gpu_uuid()).__enter__()   # sampled over every size's timed calls
    for name, n in (("lena.jpg", 141_020), ("mandril.jpg", 247_222), ("google logo png", 2_357),
                    ("large.zip", 34_904_444)):
        data = torch.from_numpy(wl.random_bytes(n, 2)).cuda()
        text = b64.encode(data, std)
        torch.cuda.synchronize()
        m = text.numel()
        dst = torch.empty(b64.decoded_max_length(m), dtype=torch.uint8, device="cuda")
        enc = torch.empty_like(text)
        res = torch.zeros(1, dtype=torch.int64, device="cuda")
        reps = 200 if n < (1 << 20) else 50

        def timed(fn, k):
            with torch.cuda.stream(stream):
                for _ in range(5):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(k):
                    fn()
                e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / k

        dec_ms = timed(lambda: b64.decode_async(text, dst, res, std, stream), reps)
        enc_ms = timed(lambda: b64.encode(data, std, enc, stream), reps)
        assert int(res.item()) == n and torch.equal(dst[:n], data) and torch.equal(enc, text)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            b64.decode_async(text, dst, res, std, stream)
            stream.synchronize()
            with torch.cuda.graph(g, stream=stream):
                for _ in range(100):
                    b64.decode_async(text, dst, res, std, stream)
        graph_ms = timed(g.replay, max(2, reps // 100)) / 100
        ge = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(ge, stream=stream):
                for _ in range(100):
                    b64.encode(data, std, enc, stream)
        enc_graph_ms = timed(ge.replay, max(2, reps // 100)) / 100
        cp = torch.empty_like(text)
        mc_ms = timed(lambda: cp.copy_(text), reps)
        per_dec = 1 if m <= (512 << 10) else 3  # one launch up to 512 KiB, else init, body, tail
        g_reps = max(2, reps // 100)
        launches += per_dec * (reps + 100 * g_reps) + (reps + 100 * g_reps)  # timed calls
        rows.append({"file": name, "bytes": n, "base64_bytes": m,
                     "decode_gbps": m / (dec_ms / 1e3) / 1e9,
                     "decode_graph_gbps": m / (graph_ms / 1e3) / 1e9,
                     "encode_gbps": m / (enc_ms / 1e3) / 1e9,
                     "encode_graph_gbps": m / (enc_graph_ms / 1e3) / 1e9,
                     "memcpy_gbps": m / (mc_ms / 1e3) / 1e9,
                     "decode_us": dec_ms * 1e3, "decode_graph_us": graph_ms * 1e3})
    clocks.__exit__(None, None, None)
    big = rows[-1]
    emit({"metric": METRIC, "workload": "paper Table 2 sizes", "value": big["decode_gbps"],
          "unit": "GB/s (base64 bytes, decode, 34,904,444-byte case)", "n_gpus": 1, "steps": 0,
          "warmup": 5, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u8", "data": "synthetic (random bytes at the files' sizes)",
          "config": {"workload": "Table 2 sizes", "l2": "all but the largest case fit in L2"},
          "sizes": rows, "clocks": clocks.summary(), "gpu_launches": launches})


# ---------------------------------------------------------------- serving workload

def serve_payloads(b64, wl):
    """The payload pools: 1 GiB of seed-5 random bytes (encode requests) and
    its standard encoding (decode requests)."""
    import torch
    raw = wl.random_bytes(1 << 30, 5)
    d_raw = torch.from_numpy(raw).cuda()
    text = b64.encode(d_raw, b64.Alphabet.standard()).cpu().numpy()
    del d_raw
    return [(raw, 1), (text, 4)]


def serve_once(b64, serve, pools, rate: float, duration: float, streams: int) -> dict:
    """One open-loop run at `rate` req/s for `duration` s through a fresh
    engine (4 GiB device budget): latency percentiles, throughput, and the
    length of every result checked."""
    arrivals, ops, sizes, pick = serve.poisson_requests(rate, duration, 4, 5)
    srv = serve.Server(4 << 30, [b64.Alphabet.standard()], n_streams=streams)
    try:
        import torch
        with clock_sampler(gpu_uuid(torch.cuda.current_device())) as clocks:
            lat, results, wall, _ = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                        8 << 30)
        batches = srv.batches()
    finally:
        srv.close()
    n = arrivals.size
    want = np.where(ops == 0, (sizes + 2) // 3 * 4, sizes // 4 * 3)   # no padding in payloads
    in_bytes = int(sizes.sum())
    return {"rate_req_per_s": rate, "duration_s": duration, "requests": n,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3),
            "aggregate_gbps": in_bytes / wall / 1e9,
            "offered_gbps": in_bytes / duration / 1e9,
            "achieved_req_per_s": n / wall, "wall_s": wall, "batches": batches,
            "results_correct": int((results == want).sum()),
            "results_checked": "output length of every request",
            "clocks": clocks.summary(),
            # per batch: encode results + tile kernel, or decode tile + finalize kernel
            "gpu_launches": 2 * batches}


SERVE_P99_BOUND_MS = 5.0


def serve_workload(args, rate: float, duration: float, sweep=()) -> dict:
    """Poisson arrivals (mean `rate` req/s, seed 4) over `duration` seconds,
    60% decode / 40% encode, sizes clip(lognormal(10.62, 2.0), 100 B, 16 MiB)
    (seed 5), served under a 4 GiB device budget with continuous batching;
    latency = arrival -> result back on the host. `sweep`: further rates, run
    for --sweep-duration seconds each, to find the engine's capacity (the
    highest rate whose p99 stays within SERVE_P99_BOUND_MS)."""
    import torch
    from paper_1910_05109_gb300 import binding as b64
    from paper_1910_05109_gb300 import build as gpu_build
    from paper_1910_05109_gb300 import serve
    from paper_1910_05109_gb300 import workloads as wl

    gpu_build.build()
    torch.cuda.set_device(0)
    pools = serve_payloads(b64, wl)
    main = serve_once(b64, serve, pools, rate, duration, args.streams)
    main["config"] = {"workload": f"Poisson {rate:.0f} req/s for {duration:.0f} s, 60% "
                                  "decode / 40% encode, sizes clip(lognormal(10.62, 2.0), 100 B, "
                                  "16 MiB), 4 GiB device budget, continuous batching",
                      "requests": main["requests"], "streams": args.streams}
    if sweep:
        rows = [serve_once(b64, serve, pools, r, args.sweep_duration, args.streams)
                for r in sweep]
        keep = ("rate_req_per_s", "requests", "p50_ms", "p99_ms", "max_ms", "aggregate_gbps",
                "offered_gbps", "achieved_req_per_s", "results_correct")
        main["serve_sweep"] = [{k: row[k] for k in keep} for row in rows]
        ok = [row["rate_req_per_s"] for row in rows + [main]
              if row["p99_ms"] <= SERVE_P99_BOUND_MS and row["results_correct"] == row["requests"]]
        main["capacity"] = {"p99_bound_ms": SERVE_P99_BOUND_MS,
                            "highest_rate_within_bound": max(ok) if ok else None,
                            "sweep_duration_s": args.sweep_duration}
    return main


def run_serve(args):
    rates = [float(x) for x in args.rates.split(",") if x] if args.rates else []
    r = serve_workload(args, args.rate, args.duration, rates)
    emit({"metric": METRIC, "workload": "serving loop", "value": r["p99_ms"],
          "unit": "ms (p99 latency)", "n_gpus": 1, "steps": r["requests"], "warmup": 0,
          "ms_per_step": r["wall_s"] / r["requests"] * 1e3, "higher_is_better": False,
          "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
          **{k: v for k, v in r.items() if k not in ("requests", "wall_s")}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--piece-bytes", type=int, default=0,
                    help="host codec piece size for the e2e leg (0 = library default)")
    ap.add_argument("--host-streams", type=int, default=0,
                    help="host codec streams for the e2e leg (0 = library default)")
    ap.add_argument("--bytes", type=int, default=N_BYTES,
                    help="input size (default 1 GiB; smaller sizes are for profiling)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "mime", "table2"],
                    help="single: the 1 GiB single-buffer step (default); batch: 100,000 "
                         "strings in one launch sequence vs one launch per string; serve: "
                         "Poisson request stream through the continuous-batching engine")
    ap.add_argument("--strings", type=int, default=100_000)
    ap.add_argument("--rate", type=float, default=20_000.0)
    ap.add_argument("--duration", type=float, default=30.0)
    ap.add_argument("--rates", default="",
                    help="serve workload: comma-separated further rates (req/s) to sweep")
    ap.add_argument("--sweep-duration", type=float, default=3.0,
                    help="serve workload: seconds per sweep rate")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default run: skip the batch, MIME and serving measurements")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--mime-bytes", type=int, default=256 << 20)
    ap.add_argument("--tile-units", type=int, default=0,
                    help="batch workload: fixed tile size instead of the autotuner's")
    ap.add_argument("--no-per-string", action="store_true",
                    help="batch workload: skip the one-launch-per-string comparison")
    ap.add_argument("--batch-layout", default="align16", choices=["align16", "packed"],
                    help="batch workload: output offsets (16-byte aligned string starts, or "
                         "packed); the other layout is timed beside")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "mime":
        run_mime(args)
    elif args.workload == "table2":
        run_table2(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
