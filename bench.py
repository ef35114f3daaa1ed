"""Benchmark of gbsa on one GB300: input MB/s suffix-sorted, the HBM roofline
fraction, batched against per-text builds, and serving p50/p99.

Default run (one JSON line; one step = one whole suffix-array build through
the C-ABI, inputs resident in HBM when the timed region starts):

- headline: a single DNA-like text of n = 2^31 bytes over {A,C,G,T}, an
  order-3 Markov chain with a seeded random transition table plus 5% of
  positions covered by copied segments of 1-100 KiB; uint32 SA. The text
  (2 GiB) and the working set (about 143 GB) exceed the 129 MB L2, so no
  flush is needed between steps. `e2e` is the same metric through
  sa_build_host (pinned host text in, host SA out, copies timed).
- "cfg2": a single text of n = 2^28 bytes, a 1 MiB Zipf(1.1) base over the
  bytes 1..255 repeated 256 times with 0.1% substitutions per copy, with
  the paths beside the hot path on the same text (BWT, LCP, DC3, DC7,
  prefix doubling using sorting, a-fold rounds).
- "batched": 4096 uniform-DNA texts with log-uniform lengths in
  [1 KiB, 4 MiB] in one sa_build_batched launch sequence, against 4096
  per-text builds on the same stream.
- "serving": Poisson arrivals at 100, 1000 and 2000 requests/s, sizes
  log-uniform in [10 KiB, 64 MiB], half uniform DNA, half i.i.d. Zipf
  bytes, admission by a 100 GB device budget: p50/p99 latency and MB/s.

Every build runs with the library's own parameter choice (the autotuner's
table shipped beside libgbsa.so); the line records the values used.

  python bench.py [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload suite|plain|batched|serving|<extra>] [--n N]

--impl reference times the CPU oracle (oracle/, prefix doubling with
discarding, one host core) on a bounded sample of the headline workload.
Under torchrun with N > 1 processes each rank runs an independent replica
of the headline (the single-text build does not shard); rank 0 prints the
line, the nested workloads run at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEAD = {"recipe": "markov", "seed": 3001, "n": 1 << 31,
        "workload": "single text n=2^31 bytes DNA-like {A,C,G,T}: order-3 Markov chain with a "
                    "seeded random transition table plus 5% of positions covered by copied "
                    "segments of 1-100 KiB; uint32 SA"}
CFG2 = {"recipe": "zipf_repeats", "seed": 2001, "n": 1 << 28,
        "workload": "single text n=2^28 bytes: 1 MiB Zipf(1.1) base over bytes 1..255 x256 "
                    "copies, 0.1% substitutions per copy; uint32 SA"}
CPU_SAMPLE_N = 1 << 23
REF_STEP_N = 1 << 20
FALLBACK_HBM_GBS = 6800.0
SERVE_DEFAULT_RATES = (100, 1000, 2000)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def max_over_ranks(value: float, distributed: bool) -> float:
    """The largest of every rank's value (the slowest replica's time); the
    value itself on a single process. Runs on the gloo group, host side."""
    if not distributed:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(n_per_rank: int, world: int, ms: float) -> float:
    """Whole-job input MB/s: every rank built its own n-character text in at
    most ms milliseconds."""
    return n_per_rank * world / (ms * 1e-3) / 1e6


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gbsa_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {"onesweep": "k_sort.cu", "refine": "k_refine.cu", "rename": "k_rename.cu",
                  "bucket": "k_bucket.cu",
                  "scatter": "k_refine.cu", "apply": "k_refine.cu", "pack": "k_pack.cu"}


def kernel_source_hash(kernel: str):
    """First 16 hex digits of the SHA-256 over the kernel's source file and
    the two headers every kernel includes."""
    csrc = os.path.join(ROOT, "paper_1610_03007_gb300", "csrc")
    h = hashlib.sha256()
    for name in (KERNEL_SOURCES[kernel], "common.cuh", "launch.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """Measured DRAM bytes per algorithmic byte of `kernel` on `workload`
    ("markov" or "zipf"), from its committed ncu summary, if the kernel's
    sources are unchanged since it was captured (else None)."""
    if kernel not in KERNEL_SOURCES:
        return None
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        text = f.read()
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    m_r = re.search(r"dram_bytes_per_algorithmic_byte:\s*([0-9.]+)", text)
    if not (m_sha and m_r) or m_sha.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_r.group(1))


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it ("model name" on x86; the ARM
    implementer and part numbers on Arm servers, 0x41/0xd4f = Neoverse V2)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return (f"{platform.machine()} CPU implementer {fields.get('CPU implementer', '?')} "
                f"part {fields['CPU part']}")
    return platform.machine()


def host_text(recipe: str, seed: int, n: int) -> np.ndarray:
    """The seeded recipe text, cached under the temporary directory by
    (recipe, seed, n) so that later runs on the same machine skip the
    generation (the 2^31-byte Markov text takes ~17 s to draw)."""
    import gen
    path = os.path.join(tempfile.gettempdir(), f"gbsa_text_{recipe}_{seed}_{n}.u8")
    if os.path.exists(path) and os.path.getsize(path) == n:
        return np.fromfile(path, dtype=np.uint8)
    t = gen.text(recipe, seed, n)
    try:
        tmp = path + f".{os.getpid()}"
        t.tofile(tmp)
        os.replace(tmp, path)
    except OSError:
        pass
    return t


def cpu_baseline():
    """The oracle as it stands, one host core, on a bounded sample: the
    headline recipe at n = 2^23."""
    import gen
    import oracle
    t = gen.text(HEAD["recipe"], HEAD["seed"], CPU_SAMPLE_N)
    o = oracle.get()
    t0 = time.perf_counter()
    o.pd_sa(t)
    dt = time.perf_counter() - t0
    return {"value": CPU_SAMPLE_N / dt / 1e6, "unit": "MB/s", "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"the headline recipe (order-3 Markov DNA with 5% copies) at n=2^23, one "
                      f"prefix-doubling-with-discarding build, {dt:.1f} s on "
                      f"{os.cpu_count()} visible host cores (1 used)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import gen
    import oracle
    o = oracle.get()
    t = gen.text(HEAD["recipe"], HEAD["seed"], REF_STEP_N)
    for _ in range(args.warmup):
        o.pd_sa(t)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.pd_sa(t)
    dt = (time.perf_counter() - t0) / args.steps
    value = REF_STEP_N / dt / 1e6
    sample = ("each step: the CPU oracle (prefix doubling with discarding, 1 core) on the "
              "headline recipe (order-3 Markov DNA with 5% copies) at n=2^20")
    line = {"metric": "input MB/s suffix-sorted", "value": value, "unit": "MB/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": HEAD["workload"] + " (sampled at n=2^20 for the CPU oracle)",
                       "n": REF_STEP_N},
            "cpu_baseline": {"value": value, "unit": "MB/s", "cores": 1, "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": sample},
            "e2e": {"value": value, "unit": "MB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _kernel_table(kern, steps):
    return {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
                "bytes_per_step": v["bytes"] / steps,
                "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
            for k, v in kern.items() if v["launches"]}


def _roofline(kern, workload):
    """The dominant kernel (most event time) against the measured copy
    bandwidth: algorithmic bytes per launch / event time per launch."""
    hbm, peak_kind = peaks()
    dname, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    ratio = ncu_traffic(dname, workload)
    avg_bytes = d["bytes"] / max(d["launches"], 1)
    return {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm,
            "traffic": ratio * avg_bytes if ratio is not None else None,
            "peak_kind": peak_kind, "bytes_per_launch": avg_bytes,
            "ms_per_launch": d["ms"] / max(d["launches"], 1)}


def measure_single(cfg, steps, warmup, local, pg=None, clocks=False, h0_chars=0, sort_items=0,
                   refine_shape=0):
    """K timed builds of one seeded text resident in HBM, with the library's
    per-launch CUDA events (sa_options.profile) on the same stream; returns
    the timings, the per-kernel table and the device text/workspace."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    n = cfg["n"]
    t_host = host_text(cfg["recipe"], cfg["seed"], n)
    dev = torch.device("cuda", local)
    text = torch.from_numpy(t_host).to(dev)
    ws = torch.empty(gbsa.workspace_bytes(n), dtype=torch.uint8, device=dev)
    sa = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    lib = gbsa.load()

    def step(profile):
        st = gbsa.Stats()
        opt = gbsa.Options(profile=1 if profile else 0, h0_chars=h0_chars, sort_items=sort_items,
                           refine_shape=refine_shape)
        rc = lib.sa_build_ex(text.data_ptr(), n, sa.data_ptr(), None, ws.data_ptr(), ws.numel(),
                             gbsa.ctypes.byref(opt), gbsa.ctypes.byref(st), stream.cuda_stream)
        if rc != 0:
            raise RuntimeError(f"sa_build_ex failed: {gbsa.status_string(rc)}")
        return st.to_dict()

    for _ in range(max(warmup, 0)):
        step(False)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if clocks else None
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern, launches, bytes_model = {}, 0, 0
    ev0.record(stream)
    for _ in range(steps):
        st = step(True)
        launches += st["launches"]
        bytes_model += st["bytes_model"]
        for k, v in st["kernels"].items():
            a = kern.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0})
            a["ms"] += v["ms"]
            a["launches"] += v["launches"]
            a["bytes"] += v["bytes"]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, pg is not None)
    return {"ms": ms, "kern": kern, "launches": launches, "bytes_model": bytes_model,
            "stats": st, "clocks": sampler.stop() if sampler else None,
            "t_host": t_host, "text": text, "ws": ws, "sa": sa}


def measure_e2e(t_host, steps):
    """sa_build_host from pinned host text to pinned host SA, copies inside
    the timed region (wall clock around the calls; each call returns after
    its result is in host memory)."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    n = t_host.size
    h_text = torch.from_numpy(t_host).pin_memory()
    h_sa = torch.empty(n, dtype=torch.int32).pin_memory()
    gbsa.sa_build_host_ptr(h_text.data_ptr(), n, h_sa.data_ptr())
    torch.cuda.synchronize()
    calls = []
    t0 = time.perf_counter()
    for _ in range(steps):
        t1 = time.perf_counter()
        gbsa.sa_build_host_ptr(h_text.data_ptr(), n, h_sa.data_ptr())
        calls.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) / steps * 1e3
    gbsa.pool_trim(0)
    # The copies alone, between the same pinned buffers and the device (not
    # part of the value: they say how much of it the host link takes).
    d_text = torch.empty(n, dtype=torch.uint8, device="cuda")
    d_sa = torch.empty(n, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    d_text.copy_(h_text, non_blocking=True)
    ev[1].record()
    ev[2].record()
    h_sa.copy_(d_sa, non_blocking=True)
    ev[3].record()
    torch.cuda.synchronize()
    h2d_ms, d2h_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    del h_text, h_sa, d_text, d_sa
    torch.cuda.empty_cache()
    return {"value": n / (e2e_ms * 1e-3) / 1e6, "unit": "MB/s", "h2d_bytes_per_step": n,
            "d2h_bytes_per_step": 4 * n, "ms_per_step": e2e_ms, "steps": steps,
            "ms_per_call": [round(c, 2) for c in calls],
            "copies_alone": {"h2d_ms": h2d_ms, "h2d_GBps": n / (h2d_ms * 1e-3) / 1e9,
                             "d2h_ms": d2h_ms, "d2h_GBps": 4 * n / (d2h_ms * 1e-3) / 1e9}}


def cfg2_extras(m, steps):
    """The paths beside the hot path on the configuration-2 text, each timed
    alone with CUDA events on the launching stream (outside the timed build
    steps): BWT and LCP of the built SA, DC3, DC7, prefix doubling using
    sorting, and the build with a-fold rounds."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    lib = gbsa.load()
    text, ws, sa_dev = m["text"], m["ws"], m["sa"]
    n = text.numel()
    dev = text.device
    stream = torch.cuda.current_stream()
    st = stream.cuda_stream
    hbm, _ = peaks()

    def timed(call, reps, warm=1):
        for _ in range(warm):
            call()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(reps):
            call()
        b1.record(stream)
        torch.cuda.synchronize()
        return b0.elapsed_time(b1) / reps

    def ok(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed: {rc}")

    bwt_buf = torch.empty(n + 1, dtype=torch.uint8, device=dev)
    prim = torch.zeros(1, dtype=torch.int64, device=dev)
    bwt_ms = timed(lambda: ok(lib.sa_bwt(text.data_ptr(), n, sa_dev.data_ptr(),
                                         bwt_buf.data_ptr(), prim.data_ptr(), st), "sa_bwt"), 5, 3)
    del bwt_buf
    lcp_buf = torch.empty(n, dtype=torch.int32, device=dev)
    lcp_ws = torch.empty(int(lib.sa_lcp_workspace_bytes(n)), dtype=torch.uint8, device=dev)
    lcp_ms = timed(lambda: ok(lib.sa_lcp(text.data_ptr(), n, sa_dev.data_ptr(), lcp_buf.data_ptr(),
                                         lcp_ws.data_ptr(), lcp_ws.numel(), st), "sa_lcp"), 3)
    del lcp_buf, lcp_ws
    out = torch.empty(n, dtype=torch.int32, device=dev)
    dc3_ms = timed(lambda: ok(lib.sa_build_dc3(text.data_ptr(), n, out.data_ptr(), None, st),
                              "sa_build_dc3"), 2)
    dc7_ms = timed(lambda: ok(lib.sa_build_dc7(text.data_ptr(), n, out.data_ptr(), None, st),
                              "sa_build_dc7"), 2)
    pds_ms = timed(lambda: ok(lib.sa_build_pd_sort(text.data_ptr(), n, out.data_ptr(), None, 0,
                                                   None, st), "sa_build_pd_sort"), 1)
    del out
    mult = {"2": {"ms": m["ms"], "rounds": m["stats"]["rounds"]}}
    for a in (3, 4):
        rounds = []
        ms = timed(lambda: rounds.append(gbsa.sa_build_ex(text, workspace=ws,
                                                          multiplier=a)[2]["rounds"]), 2)
        mult[str(a)] = {"ms": ms, "rounds": rounds[-1]}
    for v in mult.values():
        v["value"] = n / (v["ms"] * 1e-3) / 1e6
    torch.cuda.empty_cache()
    gbsa.pool_trim(0)
    mb = lambda ms: n / (ms * 1e-3) / 1e6  # noqa: E731
    return {
        "bwt": {"ms": bwt_ms, "bytes_per_row": 6, "gbs": 6.0 * (n + 1) / (bwt_ms * 1e-3) / 1e9,
                "frac": 6.0 * (n + 1) / (bwt_ms * 1e-3) / 1e9 / hbm},
        "lcp": {"ms": lcp_ms, "bytes_per_position": 30, "gbs": 30.0 * n / (lcp_ms * 1e-3) / 1e9,
                "frac": 30.0 * n / (lcp_ms * 1e-3) / 1e9 / hbm},
        "dc3": {"ms": dc3_ms, "value": mb(dc3_ms), "unit": "MB/s"},
        "dc7": {"ms": dc7_ms, "value": mb(dc7_ms), "unit": "MB/s"},
        "pd_sort": {"ms": pds_ms, "value": mb(pds_ms), "unit": "MB/s",
                    "note": "prefix doubling using sorting, no discarding"},
        "multiplier": {"by_a": mult, "unit": "MB/s",
                       "note": "a-fold rounds (Prefix Quadrupling)"},
    }


def single_report(m, cfg, steps, world):
    hbm, _ = peaks()
    ms = m["ms"]
    n = cfg["n"]
    path_gbs = m["bytes_model"] / steps / (ms * 1e-3) / 1e9
    st = m["stats"]
    return {
        "value": replicas_value(n, world, ms), "unit": "MB/s", "ms_per_step": ms, "steps": steps,
        "config": {"workload": cfg["workload"], "n": n, "seed": cfg["seed"],
                   "rounds": st["rounds"], "params": st["params"],
                   "active_per_round": st["active"], "groups_per_round": st["groups"]},
        "roofline": _roofline(m["kern"], "markov" if cfg["recipe"] == "markov" else "zipf"),
        "path_roofline": {"bytes_per_step": m["bytes_model"] / steps, "achieved_gbs": path_gbs,
                          "frac_measured": path_gbs / hbm, "frac_8tbs": path_gbs / 8000.0},
        "kernels": _kernel_table(m["kern"], steps),
        "gpu_launches": m["launches"],
    }


def run_suite(args):
    """The default run: the headline (configuration 3) line with the other
    workloads nested in it."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    gbsa.load()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    head = dict(HEAD)
    if args.n:
        head["n"] = args.n
        head["workload"] += f" (n overridden to {args.n})"
    # End to end first, in the fresh process: the library pool then takes
    # device memory nothing else has used (re-growing it onto ~150 GB that
    # the caching allocator just returned measured 1.7x slower builds).
    e2e = measure_e2e(host_text(head["recipe"], head["seed"], head["n"]),
                      max(1, min(args.steps, 3)))
    m = measure_single(head, args.steps, args.warmup, local, pg, clocks=True)
    rep = single_report(m, head, args.steps, world)
    for k in ("text", "ws", "sa", "t_host"):
        del m[k]
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    line = {
        "metric": "input MB/s suffix-sorted", "value": rep["value"], "unit": "MB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": rep["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(rep["config"], l2="inputs larger than L2 (2 GiB text, ~143 GB working "
                                         "set); no flush",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": rep["roofline"], "path_roofline": rep["path_roofline"],
        "kernels": rep["kernels"], "e2e": e2e, "gpu_launches": rep["gpu_launches"],
        "clocks": m["clocks"],
    }
    if world == 1 and not args.headline_only:
        c2 = dict(CFG2)
        m2 = measure_single(c2, max(1, min(args.steps, 5)), 2, local)
        r2 = single_report(m2, c2, max(1, min(args.steps, 5)), 1)
        if not args.build_only:
            r2.update(cfg2_extras(m2, args.steps))
        for k in ("text", "ws", "sa"):
            del m2[k]
        torch.cuda.empty_cache()
        gbsa.pool_trim(0)
        line["cfg2"] = r2
        line["batched"] = run_batched(args, emit=False)
        torch.cuda.empty_cache()
        gbsa.pool_trim(0)
        line["serving"] = run_serving(args, emit=False)
        gbsa.pool_trim(0)
        line["gpu_launches"] += r2["gpu_launches"] + line["batched"]["gpu_launches"]
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline() if (world == 1 and not args.no_cpu) else None
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()


def run_plain(args):
    """One single-text workload alone (--recipe, --n; default: the
    configuration-2 text), its own line."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    gbsa.load()
    cfg = dict(CFG2 if args.recipe == "zipf_repeats" else HEAD)
    if args.recipe not in ("zipf_repeats", "markov"):
        cfg = {"recipe": args.recipe, "seed": 1001, "n": 1 << 20,
               "workload": f"{args.recipe} recipe"}
    if args.n:
        cfg["n"] = args.n
        cfg["workload"] += f" (n = {args.n})"
    if args.h0:
        cfg["workload"] += f" ({args.h0} characters per initial key)"
    if args.sort_items:
        cfg["workload"] += f" ({args.sort_items} keys per thread in the radix passes)"
    if args.refine_shape:
        cfg["workload"] += f" (refine tile shape {args.refine_shape})"
    m = measure_single(cfg, args.steps, args.warmup, local, clocks=True, h0_chars=args.h0,
                       sort_items=args.sort_items, refine_shape=args.refine_shape)
    rep = single_report(m, cfg, args.steps, 1)
    if not args.build_only and cfg["recipe"] == "zipf_repeats":
        rep.update(cfg2_extras(m, args.steps))
    rep.update({"metric": "input MB/s suffix-sorted", "clocks": m["clocks"],
                "warmup": args.warmup, "higher_is_better": True, "data": "synthetic"})
    print(json.dumps(rep), flush=True)


BATCH_SEED = 4001
BATCH_COUNT = 4096
BATCH_LO, BATCH_HI = 1 << 10, 4 << 20


def run_batched(args, emit=True):
    """Workload 4: 4096 uniform-DNA texts with log-uniform lengths in
    [1 KiB, 4 MiB] (about 2 GB in total), one SA per text. One step = one
    sa_build_batched launch sequence over all texts; compared with per-text
    sa_build calls on the same GPU and stream."""
    import torch

    import gen
    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    lib = gbsa.load()
    count = args.batch_count or BATCH_COUNT
    flat, off = gen.batch(BATCH_SEED, count, BATCH_LO, BATCH_HI)
    N = int(off[-1])
    dev = torch.device("cuda", local)
    texts = torch.from_numpy(flat).to(dev)
    sa = torch.empty(N, dtype=torch.int32, device=dev)
    ws = torch.empty(int(lib.sa_batched_workspace_bytes(off.ctypes.data, count)),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(profile=False):
        return gbsa.sa_build_batched(texts, off, sa_out=sa, workspace=ws, stats=True,
                                     profile=profile)
    for _ in range(max(min(args.warmup, 3), 1)):
        step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern, launches = {}, 0
    e0.record(stream)
    for _ in range(steps):
        _, st = step(profile=True)
        launches += st["launches"]
        for k, v in st["kernels"].items():
            a = kern.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0})
            a["ms"] += v["ms"]
            a["launches"] += v["launches"]
            a["bytes"] += v["bytes"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del ws
    torch.cuda.empty_cache()
    # Per-text plain launches: the same texts through sa_build_ex, one call
    # each, with one workspace sized for the longest text (the library's
    # parameters for each text's own size class).
    lens = np.diff(off).astype(np.int64)
    wsp = torch.empty(gbsa.workspace_bytes(int(lens.max())), dtype=torch.uint8, device=dev)
    views = [(int(off[k]), int(lens[k])) for k in range(count)]
    for a_, l_ in views[:8]:
        gbsa.sa_build_ex(texts[a_:a_ + l_], workspace=wsp)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for a_, l_ in views:
        if l_:
            lib.sa_build_ex(texts.data_ptr() + a_, l_, sa.data_ptr() + 4 * a_, None,
                            wsp.data_ptr(), wsp.numel(), None, None, stream.cuda_stream)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    del wsp, texts, sa
    out = {"metric": "input MB/s suffix-sorted (batched)", "value": N / (ms * 1e-3) / 1e6,
           "unit": "MB/s", "ms_per_step": ms, "steps": steps,
           "config": {"workload": f"{count} uniform-DNA texts, lengths log-uniform in "
                                  f"[1 KiB, 4 MiB], one SA per text", "total_bytes": N,
                      "seed": BATCH_SEED, "rounds": st["rounds"], "params": st["params"]},
           "per_text_plain": {"value": N / (plain_ms * 1e-3) / 1e6, "unit": "MB/s",
                              "ms": plain_ms, "calls": count},
           "speedup_vs_per_text": plain_ms / ms,
           "roofline": _roofline(kern, "batched"),
           "kernels": _kernel_table(kern, steps),
           "gpu_launches": launches}
    if emit:
        print(json.dumps(out), flush=True)
    return out


SERVE_SEED = 5001
SERVE_RATES = (10, 30, 100, 300, 1000, 2000)
SERVE_LO, SERVE_HI = 10 << 10, 64 << 20


def run_serving(args, emit=True):
    """Workload 5: Poisson arrivals of SA builds at each offered rate (rate
    0: a burst, every request submitted at once), sizes log-uniform in
    [10 KiB, 64 MiB] (--serve-max lowers the top), a fair coin choosing uniform DNA or
    i.i.d. Zipf(1.1) bytes; continuous batching under a 100 GB device budget
    (sa_server_*). Each request's text is a slice of one of two 64 MiB
    buffers drawn from those two distributions (same statistics as a fresh
    draw, without generating ~1.5 GB of text per rate)."""
    import torch

    import gen
    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    gbsa.load()
    count = args.requests or 200
    pools = [torch.from_numpy(gen.text("dna", SERVE_SEED, SERVE_HI)).pin_memory(),
             torch.from_numpy(gen.text("zipf", SERVE_SEED + 1, SERVE_HI)).pin_memory()]
    views = [p.numpy() for p in pools]
    default_rates = SERVE_RATES if emit else SERVE_DEFAULT_RATES
    rates = [float(r) for r in (args.rates.split(",") if args.rates else default_rates)]
    # Pinned result buffers, as a serving client would hand the server (a
    # pageable destination turns each result copy into a staged one): one
    # arena large enough for the largest rate's requests, carved per request.
    hi = args.serve_max or SERVE_HI
    if not SERVE_LO < hi <= SERVE_HI:
        raise SystemExit(f"--serve-max must lie in ({SERVE_LO}, {SERVE_HI}]")
    streams = {}
    for lam in rates:
        arr, sizes, kinds = gen.request_stream(SERVE_SEED + int(lam), count, lam or 1.0,
                                               SERVE_LO, hi)
        streams[lam] = (arr if lam > 0 else np.zeros_like(arr), sizes, kinds)
    arena_n = max(int(np.sum(v[1])) for v in streams.values())
    arena = torch.empty(arena_n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    out_rates = []
    with gbsa.Server(budget_bytes=100 * 10**9, slots=args.slots,
                     merge_requests=args.merge_requests) as srv:
        # Warm-up: module, streams, and the library's memory pool grown to
        # one largest request per slot, as a server that has been running a
        # while holds it (growing the pool inside a timed rate would charge
        # one-time device allocations to the requests then in flight).
        for t in [srv.submit(views[k % 2][: 1 << 20]) for k in range(8)]:
            srv.wait(t)
        for t in [srv.submit(views[k % 2]) for k in range(args.slots)]:
            srv.wait(t)
        for lam in rates:
            arr, sizes, kinds = streams[lam]
            outs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
            tickets = []
            st0 = srv.stats()
            t0 = time.perf_counter()
            for k in range(count):
                delay = t0 + float(arr[k]) - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                n = int(sizes[k])
                start = (k * 2654435761) % (SERVE_HI - n + 1)
                tickets.append(srv.submit(views[int(kinds[k])][start:start + n],
                                          out=arena[outs[k]:outs[k] + n]))
            infos = [srv.wait(t)[1] for t in tickets]
            lat = np.array([i["latency_s"] for i in infos]) * 1e3
            span = max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos)
            total = float(np.sum(sizes))
            st = srv.stats()
            out_rates.append({"offered_rps": lam, "requests": count,
                              "p50_ms": float(np.percentile(lat, 50)),
                              "p99_ms": float(np.percentile(lat, 99)),
                              "mean_ms": float(lat.mean()),
                              "throughput_MBps": total / span / 1e6,
                              "achieved_rps": count / span,
                              "input_MB": total / 1e6,
                              "peak_in_flight": st["peak_in_flight"],
                              "builds": st["builds"] - st0["builds"],
                              "merged_requests": st["merged"] - st0["merged"],
                              "peak_GB_in_use": st["peak_bytes_in_use"] / 1e9})
    del arena, pools
    line = {"metric": "serving latency p50/p99 (ms) and input MB/s per offered rate",
            "unit": "ms", "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "Poisson arrivals (rate 0: a burst, every request "
                                   "submitted at once), sizes log-uniform "
                                   f"[10 KiB, {hi / 2**20:g} MiB], "
                                   "50/50 uniform DNA / Zipf(1.1) bytes, 100 GB budget",
                       "host_buffers": "texts and results in pinned host memory",
                       "slots": args.slots, "requests_per_rate": count, "seed": SERVE_SEED,
                       "merge_requests": max(args.merge_requests, 1)},
            "rates": out_rates}
    if emit:
        print(json.dumps(line), flush=True)
    return line


EXTRA_CALLS = ("bwt", "lcp", "dc3", "dc7", "pd_sort", "quad")


def run_extra(args):
    """One of the paths beside the hot path, alone, on the configuration-2
    text (or --n characters of its recipe): W untimed calls, K calls timed
    with CUDA events on the launching stream. bwt and lcp take the SA from
    one sa_build outside the timed calls; quad is sa_build_ex with
    multiplier 4."""
    import torch

    import gen
    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build

    _build.build()
    lib = gbsa.load()
    n = args.n or CFG2["n"]
    dev = torch.device("cuda", 0)
    text = torch.from_numpy(gen.text("zipf_repeats", CFG2["seed"], n)).to(dev)
    stream = torch.cuda.current_stream()
    out = torch.empty(n + 1, dtype=torch.int32, device=dev)
    st = stream.cuda_stream
    kind = args.workload
    if kind in ("bwt", "lcp"):
        sa = gbsa.sa_build(text)
        prim = torch.zeros(1, dtype=torch.int64, device=dev)
        lws = torch.empty(int(lib.sa_lcp_workspace_bytes(n)), dtype=torch.uint8, device=dev)

    def call():
        if kind == "bwt":
            rc = lib.sa_bwt(text.data_ptr(), n, sa.data_ptr(), out.data_ptr(), prim.data_ptr(), st)
        elif kind == "lcp":
            rc = lib.sa_lcp(text.data_ptr(), n, sa.data_ptr(), out.data_ptr(), lws.data_ptr(),
                            lws.numel(), st)
        elif kind == "dc3":
            rc = lib.sa_build_dc3(text.data_ptr(), n, out.data_ptr(), None, st)
        elif kind == "dc7":
            rc = lib.sa_build_dc7(text.data_ptr(), n, out.data_ptr(), None, st)
        elif kind == "pd_sort":
            rc = lib.sa_build_pd_sort(text.data_ptr(), n, out.data_ptr(), None, 0, None, st)
        else:
            gbsa.sa_build_ex(text, multiplier=4)
            rc = 0
        if rc != 0:
            raise RuntimeError(f"{kind} failed: {rc}")

    for _ in range(max(args.warmup, 0)):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    line = {"metric": "input MB/s", "value": n / (ms * 1e-3) / 1e6, "unit": "MB/s",
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{kind} on the repeated-Zipf recipe (Zipf(1.1) base over "
                                   f"bytes 1..255 x256 copies, 0.1% substitutions), n={n}",
                       "seed": CFG2["seed"]}}
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="suite",
                    choices=["suite", "plain", "batched", "serving"] + list(EXTRA_CALLS))
    ap.add_argument("--recipe", default="zipf_repeats",
                    help="plain workload: zipf_repeats (configuration 2), markov (3), dna, ...")
    ap.add_argument("--requests", type=int, default=0, help="requests per rate (serving)")
    ap.add_argument("--rates", default="",
                    help="comma-separated offered rates (serving; 0 = a burst: every request "
                         "submitted at once)")
    ap.add_argument("--slots", type=int, default=16, help="server slots (serving)")
    ap.add_argument("--serve-max", type=int, default=0,
                    help="largest request in bytes (serving; 0 = 64 MiB)")
    ap.add_argument("--merge-requests", type=int, default=0,
                    help="most queued small requests one build takes (serving; 0 or 1 = "
                         "none merged, the library default)")
    ap.add_argument("--batch-count", type=int, default=0, help="texts in the batched workload")
    ap.add_argument("--n", type=int, default=0, help="override the text length (testing)")
    ap.add_argument("--h0", type=int, default=0,
                    help="plain workload: characters per initial key (0: the library's choice), "
                         "e.g. to profile a smaller text with the full-size key width")
    ap.add_argument("--sort-items", type=int, default=0,
                    help="plain workload: keys per thread of the radix passes (8, 12, 16; "
                         "0: the library's choice)")
    ap.add_argument("--refine-shape", type=int, default=0,
                    help="plain workload: refine tile shape 1-4 (0: the library's choice)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--headline-only", action="store_true",
                    help="suite: the headline line without the nested workloads")
    ap.add_argument("--build-only", action="store_true",
                    help="configuration 2: skip the BWT, LCP, DC3, DC7, sorting-variant and "
                         "multiplier calls (a launch list of the builds alone)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload in EXTRA_CALLS:
        run_extra(args)
    elif args.workload == "plain":
        run_plain(args)
    else:
        run_suite(args)


if __name__ == "__main__":
    main()
