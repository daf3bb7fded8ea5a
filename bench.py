"""Benchmark: build + lookup of a cascading-bit-array MPHF on one GB300.

Headline workload (one step): build the function over N = 1e10 distinct
64-bit keys (SplitMix64 outputs 0..N-1 of stream 4, generated on the device:
80 GB resident in HBM), gamma = 2, L = 25, then answer Q = 1e9 lookups of
member keys drawn uniformly at random (torch's generator, seed 5).  Keys,
queries and level arrays are far larger than L2, so no flush is needed
between steps.

value     = N / (time of one step) in Mkeys/s over all ranks (weak scaling:
            each rank builds its own function over its own N keys); the
            step's build and lookup rates are reported beside it.
e2e       = the same step through the host-buffer C-ABI entry point
            mphf_build_lookup_host (keys and queries in pinned host memory,
            the indices back to pinned memory), host<->device copies inside
            the timed region; measured when the host has the memory for it.
roofline  = the step's dominant kernel: its algorithmic bytes per launch over
            its event-timed duration, against the measured HBM copy bandwidth.
ceilings  = random sector loads and random atomics, measured in this run by
            the library's ceiling kernels; the lookup and fill bounds use them.
plain_1e8 = the N = 1e8 configuration (build + all N lookups, shuffled) as a
            secondary block, with its gamma sweep and storage layouts.
cpu_baseline / --impl reference = the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

UNIT = "Mkeys/s"
C3_N, C3_Q, C3_KEY_SEED, C3_QUERY_SEED = 10**10, 10**9, 4, 5
C2_N, C2_KEY_SEED, C2_QUERY_SEED = 10**8, 2, 3


def metric_name(N: int, Q: int) -> str:
    return f"build+lookup Mkeys/s (N={N:.0e} keys built + Q={Q:.0e} member lookups per step, " \
           f"gamma=2, L=25; value = N / step time)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=float, default=C3_N, help="keys of the headline step")
    p.add_argument("--q", type=float, default=C3_Q, help="member lookups of the headline step")
    p.add_argument("--gamma", type=float, default=2.0)
    p.add_argument("--levels", type=int, default=25)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the N = 1e8 block")
    p.add_argument("--no-sweep", action="store_true", help="skip timing gamma = 1 and 5 (1e8)")
    p.add_argument("--no-batched", action="store_true", help="skip the 4096-set batched build")
    p.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    p.add_argument("--no-partitioned", action="store_true",
                   help="skip the partitioned-form block (1e9 keys in 8 parts)")
    p.add_argument("--no-ceilings", action="store_true", help="skip the ceiling kernels")
    p.add_argument("--serve-seconds", type=float, default=3.0)
    p.add_argument("--no-layouts", action="store_true",
                   help="skip timing the lookup in the other storage layouts")
    p.add_argument("--profile-batched", action="store_true",
                   help="only the 4096-set batched build: autotune, then two builds (for ncu)")
    return p.parse_args()


# ----------------------------------------------------------------------- utils
def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (every rank's step time counts: the slowest
    rank sets the job's time).  One all-reduce; no collective for world == 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput in Mkeys/s: all ranks' keys over the slowest rank's time."""
    return world * n_per_rank / (ms_max / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- CPU baselines
def host_cpu() -> dict:
    """The host the CPU oracle runs on: logical cores and the processor name."""
    name, part = None, None
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1",
                 "0xd0c": "Arm Neoverse N1", "0xd49": "Arm Neoverse N2",
                 "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "hardware", "cpu model") and name is None:
                name = line.split(":", 1)[1].strip()
            if k == "cpu part" and part is None:
                part = line.split(":", 1)[1].strip().lower()
    except OSError:
        pass
    if name is None and part is not None:
        name = arm_parts.get(part, f"Arm CPU part {part}")
    import platform
    return {"nproc": os.cpu_count(), "cpu": name or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_baseline(n_sample: int, q_sample: int, key_seed: int, gamma: float, levels: int,
                 what: str):
    """The CPU oracle, as it stands, on a bounded sample of the workload: a
    build over the first n_sample keys of the key stream, then q_sample
    lookups of its members drawn at random."""
    import oracle
    from paper_1702_03154_gb300 import inputs
    keys = inputs.splitmix64_keys(n_sample, key_seed)
    q = keys[inputs.sample_indices(n_sample, q_sample, 17)]
    t0 = time.perf_counter()
    h = oracle.build(keys, gamma=gamma, levels=levels, seed=0)
    t1 = time.perf_counter()
    h.lookup(q)
    t2 = time.perf_counter()
    # the sample's step scaled like the workload's: n_sample keys built + q_sample looked up
    return {"value": n_sample / (t2 - t0) / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(), "seconds": t2 - t0,
            "sample": f"{what}: build over the first {n_sample:.0e} keys of the key stream + "
                      f"{q_sample:.0e} random member lookups (gamma={gamma:g}, L={levels}); "
                      f"build {t1 - t0:.2f} s, lookup {t2 - t1:.2f} s, single-threaded C; "
                      f"value = keys built / (build + lookup time)"}


def workload_config(N: int, Q: int, gamma: float, L: int, rank: int = 0) -> dict:
    """The `config` of the bench line (the same for both arms)."""
    seed = C3_KEY_SEED if N == C3_N else C2_KEY_SEED
    return {"workload": f"plain large MPHF: N={N:.0e} distinct uint64 keys (SplitMix64 outputs "
                        f"0..N-1 of stream {seed + rank}, generated on the device, "
                        f"{8 * N / 1e9:.0f} GB in HBM), gamma={gamma:g}, L={L}; build, bits/key, "
                        f"then Q={Q:.0e} random member lookups",
            "N": N, "Q": Q, "gamma": gamma, "levels": L,
            "l2": (f"keys ({8 * N / 1e9:.1f} GB) and queries ({8 * Q / 1e9:.1f} GB) far larger "
                   "than L2; no flush" if 8 * min(N, Q) > 129e6 else
                   "inputs smaller than L2 (a reduced test size, not the bench workload)")}


def run_reference(args):
    """The oracle, timed on this host's cores on bounded samples of the
    headline workload (one sample per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    N, Q = int(args.n), int(args.q)
    n_sample, q_sample = 2_000_000, max(1, int(2_000_000 * Q / N))
    per_step, r = [], None
    for _ in range(args.warmup):
        cpu_baseline(n_sample, q_sample, C3_KEY_SEED, args.gamma, args.levels, "warm-up")
    for _ in range(args.steps):
        r = cpu_baseline(n_sample, q_sample, C3_KEY_SEED, args.gamma, args.levels,
                         "sample of the headline workload")
        per_step.append(r["seconds"])
    ms = 1e3 * float(np.mean(per_step))
    val = n_sample / (ms / 1e3) / 1e6
    line = {"impl": "reference", "metric": metric_name(N, Q), "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": workload_config(N, Q, args.gamma, args.levels),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": r["sample"], "host": r["host"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------- algorithmic bytes
# Unbucketed path: a level whose hit/collision array (2 bits a position)
# exceeds 64 MiB is grouped by slab before its fill (coarse and fine
# multisplit into fixed-capacity ranges, shared-memory fill and compaction);
# smaller levels fill with L2 atomics.
GROUP_MIN_AC_BYTES = 64 << 20


def kernel_bytes(h, name: str, n_queries: int) -> int:
    """Algorithmic DRAM bytes of all launches of one kernel in one build (or
    the step's lookup), from the level sizes: every pass over a level's keys
    reads each key once (8 B) and every pass that moves keys writes each once;
    A_d is written once (m_d / 8 B).  Moving F_0 into position buckets reads
    and writes every key; a lookup reads its key and writes its index."""
    sizes = h.level_sizes()          # n_0 .. n_last, n_fb
    lv = h.levels()                  # (n_d, m_d, off_d, s_d)
    nd = sizes[:-1]
    path = h.build_path
    if name == "lookup":
        return 16 * n_queries
    if path == 1:
        if name == "partition":
            return 16 * sizes[0]
        if name == "fill_buckets":
            return sum(8 * n + m // 8 for (n, m, _, _) in lv)
        if name == "compact_buckets":
            return sum(8 * nd[d] + 8 * sizes[d + 1] for d in range(len(nd)))
        return 0
    grouped = [d for d, (n, m, _, _) in enumerate(lv) if m // 4 > GROUP_MIN_AC_BYTES]
    if name == "slab_count":
        return sum(8 * nd[d] for d in grouped)
    if name == "slab_scatter":     # coarse slabs, then fine slabs: read + write twice
        return sum(32 * nd[d] for d in grouped)
    if name == "fine_fill":
        return sum(8 * nd[d] + lv[d][1] // 8 for d in grouped)
    if name == "compact":
        return sum(8 * nd[d] + 8 * sizes[d + 1] for d in range(len(nd)))
    if name == "extract":          # hit/collision array read, A_d written
        return sum(lv[d][1] // 4 + lv[d][1] // 8 for d in range(len(nd)) if d not in grouped)
    return 0


def build_stream_bytes(h) -> int:
    """The method's streamed bytes for one build (per key-visit: 8 B read by
    ArrayFill, 8 B read by the compaction, 8 B written per survivor), A
    written once, and the rank structure (A read, counters written)."""
    sizes = h.level_sizes()
    nd = sizes[:-1]
    M = h.total_bits
    return sum(16 * n for n in nd) + 8 * sum(sizes[1:-1]) + M // 8 + M // 8 + M // 64


# ---------------------------------------------------------------- ceilings
def measure_ceilings():
    """Random-access ceilings of this GPU, measured here with the library's
    ceiling kernels (median of 3 launches after one warm-up): 32-byte and
    8-byte loads and 64-bit atomic ORs over a 48 MB array (L2-resident), and
    32-byte loads over an 8 GB array (HBM)."""
    import torch

    from paper_1702_03154_gb300 import mphf
    out = {}
    l2buf = torch.zeros(48 << 17, dtype=torch.int64, device="cuda")          # 48 MB
    hbm = torch.zeros(1 << 30, dtype=torch.int64, device="cuda")              # 8 GB
    cases = [("l2_loads32", "loads", l2buf, 32, 4 << 30),
             ("l2_loads8", "loads", l2buf, 8, 4 << 30),
             ("l2_atomics", "atomics", l2buf, 8, 2 << 30),
             ("l2_atomics_ret", "atomics_ret", l2buf, 8, 2 << 30),
             ("hbm_loads32", "loads", hbm, 32, 2 << 30)]
    for name, kind, buf, width, n in cases:
        ts, done = [], 0
        for i in range(4):
            done, ms = mphf.ceiling(kind, buf, n, seed=i + 1, width=width)
            if i:
                ts.append(ms)
        ms = float(np.median(ts))
        out[name] = {"g_per_s": round(done / (ms / 1e3) / 1e9, 1), "ops": int(done),
                     "ms": round(ms, 4), "array_bytes": buf.numel() * 8,
                     "gbs_accessed": round(done * (width if kind == "loads" else 8)
                                           / (ms / 1e3) / 1e9, 1)}
    # streaming copy HBM -> HBM over 2 x 8 GB (read + write bytes counted)
    dst = torch.empty_like(hbm)
    ts = []
    for i in range(4):
        ms = mphf.ceiling_copy(hbm, dst)
        if i:
            ts.append(ms)
    ms = float(np.median(ts))
    out["hbm_copy"] = {"gbs": round(2 * hbm.numel() * 8 / (ms / 1e3) / 1e9, 1),
                       "ms": round(ms, 4), "array_bytes": hbm.numel() * 8,
                       "note": "cross-check of the roofline peak, which is MEASURED_PEAKS.json's "
                               "hbm_gbs"}
    del l2buf, hbm, dst
    torch.cuda.empty_cache()
    out["source"] = ("measured in this run (mphf_ceiling_random_loads / _atomics / _copy, "
                     "CUDA events)")
    return out


# ----------------------------------------------------------- timed regions
def time_steps(step, steps, warmup, stream, world, local, barrier):
    """Warm-up, then `steps` timed steps bracketed by barrier + synchronize,
    with the library's per-kernel profile and launch count over the region."""
    import torch

    from paper_1702_03154_gb300 import mphf
    last = None
    for _ in range(warmup):
        if last is not None:
            last.free()
        last = step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    mphf.profile_report()
    mphf.profile_enable(True)
    launches0 = mphf.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        if last is not None:
            last.free()
        last = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = mphf.launch_count() - launches0
    mphf.profile_enable(False)
    prof = mphf.profile_report()
    ms = ev0.elapsed_time(ev1) / steps
    clk = clocks.stop()
    return last, ms, prof, launches, clk


def kernel_table(h, prof, steps, n_queries):
    total_ms = sum(v[1] for v in prof.values()) or 1.0
    kernels = {}
    for name, (cnt, tot) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        b = kernel_bytes(h, name, n_queries) * steps
        kernels[name] = {"launches": cnt, "total_ms": round(tot, 4),
                         "share": round(tot / total_ms, 4),
                         "gbs": round(b / (tot / 1e3) / 1e9, 1) if tot and b else None}
    return kernels


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per unit of
# work, from ncu captures of the kernels (their commands are kept with the
# profile summaries),
# keyed by the kernel and, for the lookup, by where A lives (HBM or L2).
# `src` lists the source files the kernel is built from and `sha` their SHA-1
# at capture time: when any of them changes the counters no longer describe
# the kernel and traffic is null.  Units: a "grouped key-visit" is one key of
# a level grouped by slab (the unbucketed path's levels past 64 MiB of
# hit/collision bits); a "query" one looked-up key; a "key" one key of F_0.
_HDR = ["common.cuh", "fastbuild.cuh", "sector.cuh"]
NCU_TRAFFIC = {
    "slab_scatter": {"src": ["build.cu"] + _HDR, "sha": "3e970480a42b", "unit": "grouped key-visit",
                     "bytes_per_unit": 35.19,
                     "note": "3e8-key capture (level 0 grouped: 24 launches of 4 builds, 42.23 GB "
                             "over 1.2e9 grouped key-visits), scaled by grouped key-visits"},
    "fine_fill": {"src": ["build.cu"] + _HDR, "sha": "3e970480a42b", "unit": "grouped key-visit",
                  "bytes_per_unit": 14.52,
                  "note": "3e8-key capture (20 launches of 4 builds, 17.43 GB over 1.2e9 "
                          "grouped key-visits), scaled by grouped key-visits"},
    "lookup@hbm": {"src": ["lookup.cu"] + _HDR, "sha": "590bc6e40776", "unit": "query",
                   "bytes_per_unit": 114.8,
                   "note": "3e8-key function (A 140 MB, above L2), 3e7 random member queries x 4 "
                           "launches, 13.78 GB"},
    "lookup@l2": {"src": ["lookup.cu"] + _HDR, "sha": "590bc6e40776", "unit": "query",
                  "bytes_per_unit": 16.25,
                  "note": "3e7-key function (A 14 MB, in L2), 3e7 random member queries x 2 "
                          "launches, 0.975 GB"},
    "partition": {"src": ["fastbuild.cu"] + _HDR, "sha": "5f73b2a05ed5", "unit": "key",
                  "bytes_per_unit": 18.21, "note": "3e7-key builds (3 launches, 1.639 GB)"},
    "compact_buckets": {"src": ["fastbuild.cu"] + _HDR, "sha": "5f73b2a05ed5", "unit": "key",
                        "bytes_per_unit": 23.34,
                        "note": "3e7-key builds (3 builds, 26 launches, 2.101 GB), per key of F_0"},
}
L2_BYTES = 126 << 20


def traffic_units(h, name: str, n_queries: int):
    """(key into NCU_TRAFFIC, units one step's launches of `name` process)."""
    if name == "lookup":
        return ("lookup@hbm" if h.device_bytes() > L2_BYTES else "lookup@l2"), n_queries
    if name in ("slab_scatter", "fine_fill"):
        lv = h.levels()
        return name, sum(n for (n, m, _, _) in lv if m // 4 > GROUP_MIN_AC_BYTES)
    return name, h.level_sizes()[0]


def traffic_for(h, name: str, n_queries: int, launches_per_step: float):
    key, units = traffic_units(h, name, n_queries)
    rec = NCU_TRAFFIC.get(key)
    if not rec:
        return None, "no ncu capture of this kernel"
    hsh = hashlib.sha1()
    for f in rec["src"]:
        hsh.update(open(os.path.join(ROOT, "paper_1702_03154_gb300", "csrc", f), "rb").read())
    if hsh.hexdigest()[:12] != rec["sha"]:
        return None, "kernel source changed since its ncu capture"
    per_launch = rec["bytes_per_unit"] * units / launches_per_step
    return per_launch, (f"DRAM read+write per launch: {rec['bytes_per_unit']} B per "
                        f"{rec['unit']} x {units:.4g} a step / {launches_per_step:g} launches; "
                        f"{rec['note']}")


def dominant_roofline(h, prof, steps, n_queries, peak, peak_kind):
    """roofline block of the kernel with the most time in the timed region."""
    if not prof:
        return None
    name, (cnt, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    b = kernel_bytes(h, name, n_queries) * steps
    ach = b / (tot / 1e3) / 1e9 if tot else 0.0
    tr, tnote = traffic_for(h, name, n_queries, cnt / steps)
    return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
            "unit": "GB/s", "frac": round(ach / peak, 4),
            "traffic": round(tr, 1) if tr else None, "traffic_note": tnote,
            "per_launch_algorithmic_bytes": round(b / cnt, 1),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json), of measured",
            "launches_per_step": cnt / steps, "avg_launch_ms": tot / cnt,
            "share_of_kernel_time": round(tot / (sum(v[1] for v in prof.values()) or 1), 4)}


# ------------------------------------------------------- headline (1e10)
def host_mem_available() -> int:
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_headline(args, stream, world, rank, local, barrier, ceil):
    """Build over N keys + Q random member lookups per step (N = 1e10,
    Q = 1e9 by default).  Returns the fields of the bench line."""
    import torch

    from paper_1702_03154_gb300 import mphf
    N, Q = int(args.n), int(args.q)
    gamma, L = args.gamma, args.levels
    keys = mphf.keygen(N, C3_KEY_SEED + rank)                     # resident in HBM
    sel = torch.randint(0, N, (Q,), device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(C3_QUERY_SEED))
    q = keys[sel]
    del sel
    out = torch.empty(Q, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    def step():
        h = mphf.MPHF.build(keys, gamma=gamma, levels=L, seed=0)
        h.lookup(q, out=out)
        return h

    last, ms, prof, launches, clk = time_steps(step, args.steps, args.warmup, stream, world,
                                               local, barrier)
    # build / lookup split (separately timed, outside the main region)
    tb, tl = [], []
    for _ in range(2):
        last.free()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        last = mphf.MPHF.build(keys, gamma=gamma, levels=L, seed=0)
        e1.record(stream)
        last.lookup(q, out=out)
        e2.record(stream)
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
        tl.append(e1.elapsed_time(e2))
    t_build, t_look = float(np.median(tb)), float(np.median(tl))
    ms_max = max_over_ranks(ms, world)
    peak, peak_kind = measured_peaks()
    sizes = last.level_sizes()
    probes = sum(last.level_sizes()[:last.num_levels]) * Q / N  # mean levels probed x Q

    res = {"ms_max": ms_max, "ms": ms, "launches": launches, "clocks": clk,
           "build_ms": round(t_build, 3), "lookup_ms": round(t_look, 3),
           "build_mkeys_s": round(N / (t_build / 1e3) / 1e6, 1),
           "lookup_mkeys_s": round(Q / (t_look / 1e3) / 1e6, 1),
           "kernels": kernel_table(last, prof, args.steps, Q),
           "roofline": dominant_roofline(last, prof, args.steps, Q, peak, peak_kind),
           "structure": {"levels": last.num_levels, "bits_per_key": round(last.bits_per_key(), 4),
                         "level_sizes": sizes[:8], "fallback": last.num_fallback,
                         "build_path": last.build_path,
                         "device_bytes_per_key": round(last.device_bytes() / N, 4)}}
    # The build as a whole against HBM: the method's streamed bytes per
    # key-visit (read for the fill, read for the compaction, survivors
    # written) over the build time.
    sb = build_stream_bytes(last)
    res["build_roofline"] = {"bound": "hbm", "algorithmic_bytes": sb,
                             "achieved": round(sb / (t_build / 1e3) / 1e9, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(sb / (t_build / 1e3) / 1e9 / peak, 4),
                             "model": "per key-visit 8 B fill read + 8 B compaction read + 8 B per "
                                      "survivor written; A written once; rank structure reads A "
                                      "and writes its counters"}
    # The lookup against its own bound: each query streams 16 B and probes
    # ~e^{1/gamma} random 32-byte sectors of A, HBM-resident at this size.
    lk = {"bound": "hbm_random_sectors", "probes_per_query": round(probes / Q, 4),
          "achieved_probes_g_s": round(probes / (t_look / 1e3) / 1e9, 2),
          "hbm_gbs_sector_bytes": round((16 * Q + 32 * probes) / (t_look / 1e3) / 1e9, 1)}
    if ceil and "hbm_loads32" in ceil:
        pk = ceil["hbm_loads32"]["g_per_s"]
        lk.update({"peak_probes_g_s": pk, "frac": round(probes / (t_look / 1e3) / 1e9 / pk, 4),
                   "peak_source": "random 32-byte loads over an 8 GB array, measured in this run"})
    res["lookup_roofline"] = lk
    res["last"] = last
    res["keys"], res["q"], res["out"] = keys, q, out
    return res


def e2e_headline(args, res, world, barrier):
    """The headline step through mphf_build_lookup_host: keys and queries in
    pinned host memory, indices back to pinned host memory, copies inside
    the timed region.  Needs ~(8 N + 16 Q) bytes of host memory per rank."""
    import torch

    from paper_1702_03154_gb300 import mphf
    N, Q = int(args.n), int(args.q)
    local_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
    need = (8 * N + 16 * Q) * local_ranks
    avail = host_mem_available()
    if avail < 1.25 * need:
        return {"value": None, "unit": UNIT,
                "skipped": f"host memory: {avail / 2**30:.0f} GiB available, "
                           f"{1.25 * need / 2**30:.0f} GiB needed for pinned keys, queries and "
                           f"indices of {local_ranks} rank(s)"}
    keys, q = res.pop("keys"), res.pop("q")
    res.pop("out")
    res["last"].free()
    t0 = time.perf_counter()
    kh = torch.empty(N, dtype=torch.int64, pin_memory=True)
    kh.copy_(keys)
    qh = torch.empty(Q, dtype=torch.int64, pin_memory=True)
    qh.copy_(q)
    oh = torch.empty(Q, dtype=torch.int64, pin_memory=True)
    t_pin = time.perf_counter() - t0
    del keys, q
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ov = oh.numpy().view(np.uint64)

    def one_call():
        h, _ = mphf.MPHF.build_lookup_host(kh, qh, out=ov, gamma=args.gamma, levels=args.levels,
                                           seed=0)
        h.free()

    # the host link as this process sees it now: one plain copy of the keys
    # to the device (the e2e step moves the same bytes first)
    dk = torch.empty(N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dk.copy_(kh, non_blocking=True)
    torch.cuda.synchronize()
    h2d_s = time.perf_counter() - t0
    del dk
    torch.cuda.empty_cache()
    warm = []
    for _ in range(2):   # warm-up: the first calls also fill the allocation pool
        t0 = time.perf_counter()
        one_call()
        torch.cuda.synchronize()
        warm.append((time.perf_counter() - t0) * 1e3)
    barrier()
    reps = max(3, min(args.steps, 5))
    per_rep = []
    for _ in range(reps):
        t0 = time.perf_counter()
        one_call()
        torch.cuda.synchronize()
        per_rep.append((time.perf_counter() - t0) * 1e3)
    barrier()
    e_max = max_over_ranks(float(np.median(per_rep)), world)
    del kh, qh, oh
    return {"value": job_value(N, world, e_max), "unit": UNIT,
            "h2d_bytes_per_step": 8 * N + 8 * Q, "d2h_bytes_per_step": 8 * Q,
            "ms_per_step": e_max, "reps": reps, "statistic": "median of the reps (wall clock)",
            "rep_ms": [round(x, 1) for x in per_rep], "warmup_ms": [round(x, 1) for x in warm],
            "h2d_keys_gbs": round(8 * N / h2d_s / 1e9, 1),
            "api": "mphf_build_lookup_host (queries copied while the levels are built), "
                   "pinned host buffers", "pin_and_fill_s": round(t_pin, 2)}


# --------------------------------------------------- secondary: N = 1e8
def run_plain(args, stream, rank, ceil):
    """The N = 1e8 configuration: build + lookup of all N keys in shuffled
    order (median of 5 after 2), its kernels, the lookup against the in-run
    L2 ceiling, the storage layouts and the gamma sweep."""
    import torch

    from paper_1702_03154_gb300 import mphf
    N, gamma, L = C2_N, 2.0, 25
    keys = mphf.keygen(N, C2_KEY_SEED + rank)
    perm = torch.randperm(N, device="cuda",
                          generator=torch.Generator(device="cuda").manual_seed(C2_QUERY_SEED))
    q = keys[perm]
    del perm
    out = torch.empty(N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()

    def one(g):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        h = mphf.MPHF.build(keys, gamma=g, levels=L, seed=0)
        ev[1].record(stream)
        h.lookup(q, out=out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        return h, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    for _ in range(2):
        one(gamma)[0].free()
    mphf.profile_report()
    mphf.profile_enable(True)
    tb, tl, reps = [], [], 5
    for i in range(reps):
        h, b, lk = one(gamma)
        tb.append(b)
        tl.append(lk)
        if i < reps - 1:
            h.free()
    mphf.profile_enable(False)
    prof = mphf.profile_report()
    b_ms, l_ms = float(np.median(tb)), float(np.median(tl))
    peak, peak_kind = measured_peaks()
    res = {"workload": f"N={N:.0e} SplitMix64 keys (stream {C2_KEY_SEED + rank}), gamma=2, L=25; "
                       "build + lookup of all N in shuffled order",
           "build_ms": round(b_ms, 4), "lookup_ms": round(l_ms, 4),
           "step_mkeys_s": round(N / ((b_ms + l_ms) / 1e3) / 1e6, 1),
           "build_mkeys_s": round(N / (b_ms / 1e3) / 1e6, 1),
           "lookup_mkeys_s": round(N / (l_ms / 1e3) / 1e6, 1),
           "kernels": kernel_table(h, prof, reps, N),
           "roofline": dominant_roofline(h, prof, reps, N, peak, peak_kind),
           "structure": {"levels": h.num_levels, "bits_per_key": round(h.bits_per_key(), 4),
                         "level_sizes": h.level_sizes()[:8], "fallback": h.num_fallback}}
    sb = build_stream_bytes(h)
    res["build_roofline"] = {"bound": "hbm", "achieved": round(sb / (b_ms / 1e3) / 1e9, 1),
                             "peak": peak, "unit": "GB/s",
                             "frac": round(sb / (b_ms / 1e3) / 1e9 / peak, 4)}
    if ceil and "l2_loads32" in ceil:
        probes = float(sum(h.level_sizes()[:h.num_levels]))
        ach = probes / (l_ms / 1e3) / 1e9
        pk = ceil["l2_loads32"]["g_per_s"]
        res["l2_probe"] = {"kernel": "lookup", "bound": "l2_random_sector_loads",
                           "achieved": round(ach, 1), "peak": pk, "unit": "G loads/s",
                           "frac": round(ach / pk, 4), "probes_per_query": round(probes / N, 4),
                           "peak_source": "random 32-byte loads over a 48 MB array, measured in "
                                          "this run"}
    by_layout = {}
    for nbytes in (() if args.no_layouts else (64, 8, 32)):
        h.set_layout(nbytes)
        tt = []
        for _ in range(3):
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record(stream)
            h.lookup(q, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            tt.append(e0.elapsed_time(e1))
        by_layout[f"{nbytes}B"] = {"lookup_ms": round(float(np.median(tt)), 4),
                                   "device_bytes_per_key": round(h.device_bytes() / N, 4)}
    res["lookup_by_layout"] = by_layout
    h.free()
    if not args.no_sweep:
        sweep = {}
        for g2 in (1.0, 5.0):
            tb, tl = [], []
            for i in range(3):
                h, b, lk = one(g2)
                if i:
                    tb.append(b)
                    tl.append(lk)
                bpk = h.bits_per_key()
                h.free()
            b2, l2 = float(np.median(tb)), float(np.median(tl))
            sweep[f"gamma={g2:g}"] = {"build_ms": round(b2, 3), "lookup_ms": round(l2, 3),
                                      "build_mkeys_s": round(N / b2 / 1e3, 1),
                                      "lookup_mkeys_s": round(N / l2 / 1e3, 1),
                                      "step_mkeys_s": round(N / (b2 + l2) / 1e3, 1),
                                      "bits_per_key": round(bpk, 4)}
        res["gamma_sweep"] = sweep
    del keys, q, out
    torch.cuda.empty_cache()
    return res


def run_batched(args, stream):
    """4096 key sets, sizes log-uniform in [1e3, 1e6] (seed 7), gamma = 2, L = 25:
    one batched build (recorded level loop, autotuned bucket width) vs the
    same sets built one by one with mphf_build; then all keys looked up in one
    multi-function launch."""
    import torch

    from paper_1702_03154_gb300 import inputs, mphf
    S = 4096
    sizes = inputs.log_uniform_sizes(S, 1e3, 1e6, 7)
    off = inputs.set_offsets(sizes)
    total = int(off[-1])
    keys = mphf.keygen(total, 7)
    torch.cuda.synchronize()
    tune_ms = mphf.autotune_batched(keys, off, gamma=2.0, levels=25, seed=0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times, wraps = [], []
    launches = 0
    import ctypes
    L = mphf.lib()
    offh = np.ascontiguousarray(off, dtype=np.uint64)
    for rep in range(4):
        l0 = mphf.launch_count()
        arr = (ctypes.c_void_p * S)()
        # the C-ABI call alone, timed on its stream; the Python wrappers of
        # the 4096 handles are made after the second event (timed apart)
        ev[0].record(stream)
        rc = L.mphf_build_batched_host_offsets(keys.data_ptr(), offh.ctypes.data, S, 2.0, 25, 0,
                                               ctypes.c_void_p(stream.cuda_stream), arr)
        ev[1].record(stream)
        torch.cuda.synchronize()
        assert rc == mphf.OK, rc
        w0 = time.perf_counter()
        hs = [mphf.MPHF(ctypes.c_void_p(arr[i])) for i in range(S)]
        wraps.append((time.perf_counter() - w0) * 1e3)
        if rep:
            times.append(ev[0].elapsed_time(ev[1]))
            launches = mphf.launch_count() - l0
        if rep < 3:
            del hs
    t_b = float(np.median(times))
    # the same sets, one mphf_build each
    ev[0].record(stream)
    singles = [mphf.MPHF.build(keys[int(off[i]):int(off[i + 1])], gamma=2.0, levels=25, seed=0)
               for i in range(S)]
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_p = ev[0].elapsed_time(ev[1])
    del singles
    # every key of every set, one multi-function launch
    out = torch.empty_like(keys)
    ks = [keys[int(off[i]):int(off[i + 1])] for i in range(S)]
    os_ = [out[int(off[i]):int(off[i + 1])] for i in range(S)]
    mphf.lookup_multi(hs, ks, os_)
    torch.cuda.synchronize()
    mphf.profile_report()
    mphf.profile_enable(True)
    mphf.lookup_multi(hs, ks, os_)       # kernel time from its own events
    torch.cuda.synchronize()
    mphf.profile_enable(False)
    t_l = mphf.profile_report()["lookup_multi"][1]
    paths = {}
    for h in hs:
        paths[h.build_path] = paths.get(h.build_path, 0) + 1
    # the method's streamed bytes of all sets (the same model as the plain
    # build's build_roofline) over the batched build's time
    peak, peak_kind = measured_peaks()
    sb = sum(build_stream_bytes(h) for h in hs if h.N)
    roof = {"bound": "hbm", "algorithmic_bytes": sb,
            "achieved": round(sb / (t_b / 1e3) / 1e9, 1), "peak": peak, "unit": "GB/s",
            "frac": round(sb / (t_b / 1e3) / 1e9 / peak, 4),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json), of measured"}
    res = {"sets": S, "keys": total, "gamma": 2.0, "levels": 25,
           "batched_build_ms": round(t_b, 3), "batched_build_mkeys_s": round(total / t_b / 1e3, 1),
           "batched_build_api": "mphf_build_batched_host_offsets (C ABI), CUDA events around the call",
           "python_handle_wrap_ms": round(float(np.median(wraps)), 3),
           "per_set_build_ms": round(t_p, 3), "per_set_build_mkeys_s": round(total / t_p / 1e3, 1),
           "speedup_vs_per_set": round(t_p / t_b, 2),
           "lookup_all_ms": round(t_l, 3), "lookup_mkeys_s": round(total / t_l / 1e3, 1),
           "autotune_best_ms": round(tune_ms, 3),
           "autotune_choice": mphf.batched_tuning(S, total),
           "kernels_per_batched_build": int(launches), "build_roofline": roof,
           "handles_by_path": {str(k): v for k, v in sorted(paths.items())}}
    del hs, keys, out
    torch.cuda.empty_cache()
    return res


def run_partitioned(args, stream):
    """The partitioned form on this GPU: 1e9 keys (stream 13) routed by a
    seeded hash into K = 8 parts, one function a part built one after
    another (mphf_build_partitioned; with one part per rank this is the
    8-GPU form, each rank building one part), then the 1e9 keys looked up in
    shuffled order (mphf_part_lookup: each key's function from its part
    hash).  Median of 3."""
    import torch

    from paper_1702_03154_gb300 import mphf
    N, K = 10**9, 8
    keys = mphf.keygen(N, 13)
    q = keys[torch.randperm(N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(14))]
    out = torch.empty_like(q)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tb, tl = [], []
    last = None
    for rep in range(4):
        if last is not None:
            del last
        ev[0].record(stream)
        last = mphf.PartitionedMPHF.build(keys, K, 21, gamma=2.0, levels=25, seed=0)
        ev[1].record(stream)
        last.lookup(q, out=out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if rep:
            tb.append(ev[0].elapsed_time(ev[1]))
            tl.append(ev[1].elapsed_time(ev[2]))
    b_ms, l_ms = float(np.median(tb)), float(np.median(tl))
    sizes = np.diff(last.offsets.astype(np.int64))
    res = {"workload": f"N=1e9 SplitMix64 keys (stream 13), K={K} parts by a seeded hash "
                       "(one function a part, built one after another on this GPU; the "
                       "8-GPU form gives each rank one part), gamma=2, L=25; then all keys "
                       "looked up in shuffled order, each with its part's function",
           "build_ms": round(b_ms, 3), "build_mkeys_s": round(N / b_ms / 1e3, 1),
           "lookup_ms": round(l_ms, 3), "lookup_mkeys_s": round(N / l_ms / 1e3, 1),
           "part_keys_min_max": [int(sizes.min()), int(sizes.max())],
           "statistic": "median of 3 after one warm-up, CUDA events"}
    del last, keys, q, out
    torch.cuda.empty_cache()
    return res


def run_serving(args, stream):
    """256 resident functions, sizes log-uniform in [1e4, 1e7] (seed 11), gamma = 2;
    open-loop Poisson lookups (batch sizes log-uniform in [1, 1e6] of member keys)
    plus 1% build requests of 1e5-1e7 keys, at 50% and 90% of the measured
    capacity of the multi-function lookup."""
    import torch

    from paper_1702_03154_gb300 import inputs, mphf
    H = 256
    sizes = inputs.log_uniform_sizes(H, 1e4, 1e7, 11)
    off = inputs.set_offsets(sizes)
    total = int(off[-1])
    keys = mphf.keygen(total, 11)
    hs = mphf.build_batched(keys, off, gamma=2.0, levels=25, seed=0)
    ks = [keys[int(off[i]):int(off[i + 1])] for i in range(H)]
    build_keys = mphf.keygen(10_000_000, 12)
    resident_bytes = sum(h.device_bytes() for h in hs)
    # capacity: back-to-back launches of requests drawn like the load (mean batch)
    rng = np.random.default_rng(2)
    reqs = []
    while sum(r[2] for r in reqs) < 2e8:
        i = int(rng.integers(H))
        b = int(np.exp(rng.uniform(0, np.log(1e6))))
        b = min(b, int(sizes[i]))
        o = int(rng.integers(0, int(sizes[i]) - b + 1))
        reqs.append((i, o, b))
    out = torch.empty(1 << 23, dtype=torch.int64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    batch, keys_in = [], 0
    groups = []
    for r in reqs:
        batch.append(r)
        keys_in += r[2]
        if keys_in >= (1 << 22):
            groups.append(batch)
            batch, keys_in = [], 0
    if batch:
        groups.append(batch)
    nk = 0
    mphf.profile_report()
    mphf.profile_enable(True)
    for g in groups:
        ring = 0
        ho, ko, oo = [], [], []
        for (i, o, b) in g:
            ho.append(hs[i])
            ko.append(ks[i][o:o + b])
            oo.append(out[ring:ring + b])
            ring += b
            nk += b
        mphf.lookup_multi(ho, ko, oo)
    torch.cuda.synchronize()
    mphf.profile_enable(False)
    cap_keys_s = nk / (mphf.profile_report()["lookup_multi"][1] / 1e3)
    mean_batch = float(np.mean([r[2] for r in reqs]))
    # cost of a build request: builds of log-uniform size in [1e5, 1e7], one at a time
    bsz = [int(np.exp(x)) for x in rng.uniform(np.log(1e5), np.log(1e7), 12)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in bsz:
        mphf.MPHF.build(build_keys[:n], gamma=2.0, levels=25, seed=0).free()
    torch.cuda.synchronize()
    build_cost = (time.perf_counter() - t0) / len(bsz)
    # capacity of the mix (99 lookups : 1 build), in arrivals per second
    per_arrival = 0.99 * mean_batch / cap_keys_s + 0.01 * build_cost
    res = {"functions": H, "resident_keys": total, "resident_bytes": int(resident_bytes),
           "lookup_capacity_mkeys_s": round(cap_keys_s / 1e6, 1),
           "mean_batch_keys": round(mean_batch, 1), "build_request_ms": round(build_cost * 1e3, 3),
           "mix_capacity_req_s": round(1.0 / per_arrival, 1),
           "load_definition": "fraction of the capacity of the 99:1 lookup/build mix, measured "
                              "back to back before the run",
           "server": {"max_batch_keys": 1 << 22, "max_inflight": 3, "build_workers": 1},
           "loads": {}}
    # one build worker: two concurrent builds keep every SM busy for the span
    # of their kernels and the lookups' p99 doubles (measured: 0.79 vs 0.45 ms
    # at 90% load; without builds it is 0.07 ms)
    srv = mphf.Server(max_batch_keys=1 << 22, max_batch_reqs=4096, max_inflight=3,
                      build_workers=1, mem_reserve=8 << 30)
    ring_out = torch.empty(1 << 24, dtype=torch.int64, device="cuda")
    # warm-up (not reported): first-use work of the server and of the build
    # path (lookup descriptors, pool growth) stays out of the measured loads
    srv.loadgen(hs, ks, rate_hz=0.5 / per_arrival, duration_s=min(1.0, args.serve_seconds),
                bmin=1, bmax=1e6, out=ring_out, build_frac=0.01, build_keys=build_keys, nbmin=1e5,
                nbmax=1e7, gamma=2.0, seed=7)
    for load in (0.5, 0.9):
        rate = load / per_arrival
        r = srv.loadgen(hs, ks, rate_hz=rate, duration_s=args.serve_seconds, bmin=1, bmax=1e6,
                        out=ring_out, build_frac=0.01, build_keys=build_keys, nbmin=1e5, nbmax=1e7,
                        gamma=2.0, seed=int(load * 100))
        lat = r["latencies"] * 1e3
        res["loads"][f"{int(load * 100)}%"] = {
            "offered_req_s": round(rate, 1), "lookups": r["lookups"], "builds": r["builds"],
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mkeys_s": round(r["keys"] / r["elapsed"] / 1e6, 1),
            "parts_ms": {k: {q: round(v[q] * 1e3, 4) for q in ("p50", "p99")}
                         for k, v in r["parts"].items()}}
    srv.close()
    del hs, keys, build_keys, out, ring_out
    torch.cuda.empty_cache()
    return res




def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1702_03154_gb300 import mphf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    N, Q = int(args.n), int(args.q)
    ceil = None if args.no_ceilings else measure_ceilings()
    res = run_headline(args, stream, world, rank, local, barrier, ceil)
    value = job_value(N, world, res["ms_max"])
    e2e = None
    if not args.no_e2e:
        e2e = e2e_headline(args, res, world, barrier)
    for k in ("keys", "q", "out"):
        res.pop(k, None)
    last = res.pop("last")
    last.free()
    del last
    torch.cuda.empty_cache()
    mphf.pool_trim()  # the 1e10 scratch cached by the library, back for the blocks below

    plain = None if args.no_plain else run_plain(args, stream, rank, ceil)
    batched = None if args.no_batched else run_batched(args, stream)
    serving = None if args.no_serving else run_serving(args, stream)
    partitioned = None if args.no_partitioned else run_partitioned(args, stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(10_000_000, max(1, int(10_000_000 * Q / N)), C3_KEY_SEED, args.gamma,
                           args.levels, "sample of the headline workload")
        cpu.pop("seconds", None)

    if rank == 0:
        line = {"metric": metric_name(N, Q), "value": round(value, 1), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["ms_max"], 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": workload_config(N, Q, args.gamma, args.levels, rank),
                "build_mkeys_s": res["build_mkeys_s"], "lookup_mkeys_s": res["lookup_mkeys_s"],
                "build_ms": res["build_ms"], "lookup_ms": res["lookup_ms"],
                "structure": res["structure"], "clocks": res["clocks"], "e2e": e2e,
                "gpu_launches": int(res["launches"]), "roofline": res["roofline"],
                "build_roofline": res["build_roofline"], "lookup_roofline": res["lookup_roofline"],
                "kernels": res["kernels"], "ceilings": ceil, "cpu_baseline": cpu}
        if plain:
            line["plain_1e8"] = plain
        if batched:
            line["batched"] = batched
        if serving:
            line["serving"] = serving
        if partitioned:
            line["partitioned"] = partitioned
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profile_batched():
    """The batched workload alone, for a profiler: the 4096 sets of the batched
    bench line, autotuned, then built twice."""
    import torch

    from paper_1702_03154_gb300 import inputs, mphf
    off = inputs.set_offsets(inputs.log_uniform_sizes(4096, 1e3, 1e6, 7))
    keys = mphf.keygen(int(off[-1]), 7)
    mphf.autotune_batched(keys, off, gamma=2.0, levels=25, seed=0)
    for _ in range(2):
        hs = mphf.build_batched(keys, off, gamma=2.0, levels=25, seed=0)
        torch.cuda.synchronize()
        del hs




def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_batched:
        profile_batched()
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
