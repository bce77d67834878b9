#!/usr/bin/env python3
"""Benchmark of the GB300 comparison sort.

Workload (one "step"): sort the four 2^24-key int32 arrays of the benchmark
configuration -- uniform random, strictly descending, nearly sorted (1% of
positions exchanged) and few unique (16 values) -- all drawn from seed 1.
Each array is restored from a pristine device copy and L2 is flushed (a
512 MiB write, larger than the 129 MB L2) before every sort; only the sorts
are timed, with CUDA events on the sorting stream.

Printed: one JSON line with the metric (Gkeys/s), the per-kernel HBM roofline
of the dominant kernel measured live, the end-to-end number through the
host-buffer entry point, the CPU oracle baseline, clocks and launch count.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU; the sort does not shard).
--impl reference times the CPU oracle (the paper's mergesort, single thread)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gkeys/s at 2^24–2^28 int32, % of HBM roofline; learned/batched vs plain"
N_KEYS = 1 << 24
CLASSES = ("uniform", "reversed", "nearly_sorted", "few_unique")
SEED = 1
FLUSH_BYTES = 512 << 20
CPU_SAMPLE = 1 << 22          # keys of each array one reference-arm step sorts


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 2^24..2^28 size sweep")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the pairs / learned / batched measurements")
    ap.add_argument("--profile-case", type=int, default=0, metavar="LOG2N",
                    help="for ncu: sort a uniform int32 array of 2^LOG2N keys twice (warm-up + one) and exit")
    ap.add_argument("--profile-form", choices=["keys", "learned", "batched"], default="keys",
                    help="with --profile-case: the learned sort of 2^LOG2N lognormal float32 keys, or the "
                         "batched sort of 200,000 arrays (LOG2N ignored), instead of the key sort")
    ap.add_argument("--profile-config", type=int, default=-1,
                    help="with --profile-form batched: this launch configuration instead of tuning")
    ap.add_argument("--profile-pairs", action="store_true",
                    help="with --profile-case: a stable uint64-key + uint32-payload sort instead")
    ap.add_argument("--classes", action="store_true",
                    help="time the paper's parametrised input classes (Section 2) at 2^24 int32 and exit")
    ap.add_argument("--profile-class", default="uniform",
                    choices=["uniform", "reversed", "nearly_sorted", "few_unique"],
                    help="with --profile-case (key sort): the int32 input class")
    return ap.parse_args()


NOMINAL_HBM_GBS = 8000.0          # the nominal ~8 TB/s of GB300's HBM3e, reported beside the measured peak


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _ncu_traffic(kernel_tag: str, scale: float = 1.0):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary (times
    `scale`, for a summary taken on a smaller array whose traffic grows with
    the keys), or None if the summary is missing or the kernel's sources
    changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    src = b""
    for fn in ("sr_kernels.cuh", "sr_device.cuh"):
        with open(os.path.join(ROOT, "paper_1609_04471_gb300", "csrc", fn), "rb") as f:
            src += f.read()
    if hashlib.sha256(src).hexdigest()[:16] != h.group(1)[:16]:
        return None
    return int(int(m.group(1)) * scale)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def _max_over_ranks(x: float, device) -> float:
    """The maximum of x over the ranks of the default process group (x itself
    when there is none or it has one rank): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(keys_per_rank: int, ranks: int, ms: float) -> float:
    """Whole-job throughput in Gkeys/s: every rank's keys over the job's time."""
    return keys_per_rank * ranks / (ms / 1e3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(arrays, sample=None, algos=("merge", "quick")):
    """The oracle's two sorts (single-threaded C: the natural mergesort and the
    hybrid quicksort) on the arrays of the workload (their first `sample` keys
    if given), pinned to host core 0 while they run; returns
    {algo: (Gkeys/s, seconds, keys)}."""
    import oracle
    oracle.build()
    try:
        old = os.sched_getaffinity(0)
        os.sched_setaffinity(0, {sorted(old)[0]})
    except (AttributeError, OSError):
        old = None
    out = {}
    try:
        for algo in algos:
            keys = 0
            t0 = time.perf_counter()
            for a in arrays:
                part = a if sample is None else a[:sample]
                oracle.sort_keys(part, algo)
                keys += part.size
            dt = time.perf_counter() - t0
            out[algo] = (keys / dt / 1e9, dt, keys)
    finally:
        if old is not None:
            os.sched_setaffinity(0, old)
    return out


def _cpu_model():
    """The host CPU's model name (lscpu's, else /proc/cpuinfo's)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _config():
    return {"workload": "sort 4 arrays of 2^24 int32 keys (uniform, strictly descending, "
                        "nearly sorted 1% exchanges, few unique 16 values), seed 1",
            "n": N_KEYS, "arrays": 4, "l2": "flushed before every timed sort (512 MiB write)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import sortrace_inputs as si
    arrays = [si.int32_input(k, N_KEYS, SEED) for k in CLASSES]
    for _ in range(args.warmup):
        _cpu_baseline(arrays, CPU_SAMPLE, ("merge",))
    times = []
    keys = 0
    for _ in range(args.steps):
        v, dt, keys = _cpu_baseline(arrays, CPU_SAMPLE, ("merge",))["merge"]
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = keys / (ms / 1e3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": _config(),
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {CPU_SAMPLE} keys of each of the 4 arrays per step",
                         "cpu": _cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _gen_arrays():
    import sortrace_inputs as si
    return [si.int32_input(k, N_KEYS, SEED) for k in CLASSES]


def run_ours(args):
    import numpy as np
    import torch
    import paper_1609_04471_gb300 as sr

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    sr.load()
    peak, peak_kind = _peaks()

    arrays = _gen_arrays()
    pristine = [torch.from_numpy(a).to(dev) for a in arrays]
    work = [torch.empty_like(p) for p in pristine]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(step, timed, prof):
        ms = []
        for c in range(len(CLASSES)):
            work[c].copy_(pristine[c])
            flush.fill_(step & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if prof is not None:
                sr.profile_begin()
            e0.record(stream)
            sr.sort_keys(work[c])
            e1.record(stream)
            if prof is not None:
                k = sr.profile_end()
                st = sr.stats()
                prof.append((c, k, st))
            ms.append((e0, e1))
        return ms

    for w in range(args.warmup):
        one_step(w, False, None)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = sr.launch_count()
    events = []
    wall0 = time.perf_counter()
    for step in range(args.steps):                   # timed region: the headline number
        events.append(one_step(step, True, None))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = sr.launch_count() - launches0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    prof = []
    for step in range(args.steps):                   # same steps again, every launch bracketed by events
        one_step(step, True, prof)
    torch.cuda.synchronize()
    clk = clocks.stop()

    per_class_ms = [0.0] * len(CLASSES)
    for evs in events:
        for c, (e0, e1) in enumerate(evs):
            per_class_ms[c] += e0.elapsed_time(e1)
    per_class_ms = [m / args.steps for m in per_class_ms]
    ms_step = _max_over_ranks(sum(per_class_ms), dev)
    keys_step = N_KEYS * len(CLASSES)
    value = _job_value(keys_step, ws, ms_step)

    # live roofline of each kernel kind over the timed region
    kinds = {}
    path_bytes = 0
    work_merges = 0
    merge_ms_work = 0.0
    for c, k, st in prof:
        path_bytes += st["bytes_moved"]
        for name, (n_l, t_ms) in k.items():
            a = kinds.setdefault(name, [0, 0.0])
            a[0] += n_l
            a[1] += t_ms
        if st["input_class"] == 0:
            done = st["passes_planned"] - st["passes_skipped"]
            if done == st["passes_planned"]:
                work_merges += k["merge"][0]
                merge_ms_work += k["merge"][1]
    dominant = max(kinds.items(), key=lambda kv: kv[1][1])[0]
    merge_bytes_launch = 2 * N_KEYS * 4            # read + write of every key
    achieved = merge_bytes_launch / (merge_ms_work / work_merges / 1e3) / 1e9 if work_merges else None
    timed_region = {
        "where": "the timed region (4 x 2^24 int32, uniform array's merge steps); input and output of a "
                 "step fit the 129 MB L2 together, so part of each step's traffic is L2 hits",
        "achieved": achieved, "frac": (achieved / peak) if achieved else None,
        "frac_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
        "avg_launch_ms": merge_ms_work / work_merges if work_merges else None,
        "launches_timed": work_merges, "algorithmic_bytes_per_launch": merge_bytes_launch,
        "traffic": _ncu_traffic("merge_step_2p24_int32"),
    }
    roofline = {
        "bound": "hbm", "kernel": "merge step (k_merge: 2-way, the fan-in of 4-byte keys alone)",
        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
        "peak_kind": peak_kind, "frac_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
        "nominal_peak": NOMINAL_HBM_GBS, "algorithmic_bytes_per_launch": merge_bytes_launch,
        "traffic": timed_region["traffic"], "where": timed_region["where"],
        "avg_launch_ms": merge_ms_work / work_merges if work_merges else None,
        "launches_timed": work_merges,
        "dominant_by_time": dominant,
        "path_bytes_per_step": path_bytes / args.steps,
        "path_frac": (path_bytes / args.steps) / (ms_step / 1e3) / 1e9 / peak,
        "path_frac_nominal": (path_bytes / args.steps) / (ms_step / 1e3) / 1e9 / NOMINAL_HBM_GBS,
        "lower_bound_frac": (2 * 4 * keys_step) / (ms_step / 1e3) / 1e9 / peak,
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in kinds.items() if v[0]},
        "timing": "per-launch events in a second pass over the same steps; value comes from the unbracketed pass",
    }

    # end to end through the host-buffer entry point (pinned host memory): the
    # step's four arrays are queued on four streams, so one array's copies
    # overlap another's sort; the step ends when all four are back in host memory
    # (sr_sort_keys_host_many, one pipelined call, measured the same or slower)
    host = [torch.from_numpy(a).pin_memory() for a in arrays]
    host_src = [h.clone().pin_memory() for h in host]
    streams = [torch.cuda.Stream() for _ in CLASSES]
    for c in range(len(CLASSES)):
        sr.sort_keys_host(host[c].numpy())
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for step in range(args.steps):
        for c in range(len(CLASSES)):
            host[c].copy_(host_src[c])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in range(len(CLASSES)):
            sr.sort_keys_host_async(host[c], stream=streams[c])
        for st_ in streams:
            st_.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = _max_over_ranks(e2e_ms / args.steps, dev)
    e2e = {"value": _job_value(keys_step, ws, e2e_ms), "unit": "Gkeys/s",
           "h2d_bytes_per_step": 4 * keys_step, "d2h_bytes_per_step": 4 * keys_step,
           "ms_per_step": e2e_ms,
           "api": "sr_sort_keys_host_async on four streams (one per array), host clock from the first "
                  "call to the last stream's completion"}

    sweep = None
    if not args.no_sweep:
        sweep = _sweep(sr, torch, dev, stream, peak)
        # headline roofline out of L2: the merge steps of the 2^28 sort (2 GiB
        # in, 2 GiB out per step), each launch timed with CUDA events on the
        # sorting stream; the timed region's L2-assisted figure stays beside it
        big = sweep.get("2^28", {}).get("kernels", {})
        m28 = big.get("merge")
        if m28:
            roofline.update({
                "achieved": m28["achieved_gbs"], "frac": m28["frac"], "frac_nominal": m28["frac_nominal"],
                "algorithmic_bytes_per_launch": m28["bytes_per_launch"], "avg_launch_ms": m28["avg_launch_ms"],
                "launches_timed": m28["launches"],
                "where": "2^28 uniform int32 sort of the size sweep (2 GiB per step in and out, far above L2), "
                         "every launch bracketed by CUDA events on the sorting stream",
                "traffic": _ncu_traffic("merge_step_2p26_int32", scale=4),
                "traffic_note": "dram read + write bytes of one k_merge launch at 2^26 (ncu, "
                                "profiles/merge_step_2p26_int32.md) times 4, the keys of a 2^28 launch",
                "timed_region_2p24_l2_assisted": timed_region,
                "other_kernels_2p28": {kname: big[kname] for kname in ("block_sort", "detect") if kname in big},
            })
    forms = None
    if not args.no_forms and rank == 0:
        forms = _forms(sr, torch, dev, stream, peak)
        forms["classes_2^24_int32"] = _classes(sr, torch)

    cpu = None
    if rank == 0:
        cb = _cpu_baseline(arrays)
        v, dt, keys = cb["merge"]
        vq, dtq, _ = cb["quick"]
        cpu = {"value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole workload: the 4 arrays of 2^24 keys ({keys} keys); "
                         f"mergesort {dt:.2f} s, quicksort {dtq:.2f} s",
               "algorithm": "natural mergesort (mer6 techniques, Section 3)",
               "quicksort_value": vq, "quicksort_algorithm": "hybrid quicksort (hyb2, Section 4)",
               "cpu": _cpu_model(), "nproc": os.cpu_count()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": dict(_config(), parallelism="replicas" if ws > 1 else "single-gpu",
                           per_class_ms=dict(zip(CLASSES, per_class_ms)), wall_s_timed_region=wall),
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clk,
        }
        if sweep is not None:
            line["sweep"] = sweep
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def _sweep(sr, torch, dev, stream, peak, reps=3):
    """Uniform int32 at 2^24..2^28 (prefixes of one 2^28 draw): Gkeys/s and the
    fraction of the HBM roofline on the passes model and on the 1 read + 1
    write lower bound."""
    import sortrace_inputs as si
    big = torch.from_numpy(si.uniform_i32(1 << 28, SEED)).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for lg in range(24, 29):
        n = 1 << lg
        x = torch.empty(n, dtype=torch.int32, device=dev)
        best = None
        for r in range(reps + 1):
            x.copy_(big[:n])
            flush.fill_(r)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sr.sort_keys(x)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        st = sr.stats()
        # the same sort once more with every launch bracketed by CUDA events on
        # the sorting stream: per-kernel time, hence each kernel's own roofline
        x.copy_(big[:n])
        flush.fill_(0x5A)
        torch.cuda.synchronize()
        sr.profile_begin()
        sr.sort_keys(x)
        k = sr.profile_end()
        kern = {}
        # merge and block sort: bytes of one launch over its average time; the
        # scan: the keys read once over the time of the whole kind (the scan
        # and the few-distinct-keys sampling kernels it launches with)
        for name, per_key, per_call in (("merge", 8, False), ("block_sort", 8, False), ("detect", 4, True)):
            launches, t_ms = k.get(name, (0, 0.0))
            if launches:
                avg = t_ms if per_call else t_ms / launches
                gbs = per_key * n / (avg / 1e3) / 1e9
                kern[name] = {"launches": launches, "avg_launch_ms" if not per_call else "ms_per_call": avg,
                              "bytes_per_launch" if not per_call else "bytes_per_call": per_key * n,
                              "achieved_gbs": gbs, "frac": gbs / peak, "frac_nominal": gbs / NOMINAL_HBM_GBS}
        out[f"2^{lg}"] = {"ms": best, "gkeys_s": n / (best / 1e3) / 1e9,
                          "passes_frac": st["bytes_moved"] / (best / 1e3) / 1e9 / peak,
                          "passes_frac_nominal": st["bytes_moved"] / (best / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                          "lower_bound_frac": 8 * n / (best / 1e3) / 1e9 / peak,
                          "bytes_moved": st["bytes_moved"], "merge_steps": st["passes_planned"],
                          "kernels": kern,
                          "kernel_ms": {name: round(v[1], 4) for name, v in k.items() if v[0]}}
        del x
    return out


def run_profile_case(args):
    """A small, fixed case for ncu captures: one warm-up sort, then one sort."""
    import numpy as np
    import torch
    import paper_1609_04471_gb300 as sr
    import sortrace_inputs as si
    torch.cuda.set_device(0)
    n = 1 << args.profile_case
    if args.profile_pairs:
        k, v = si.pairs_u64_zipf(n, SEED)
        src_k = torch.from_numpy(k.view(np.int64)).cuda()
        src_v = torch.from_numpy(v.view(np.int32)).cuda()
        for _ in range(2):
            xk, xv = src_k.clone(), src_v.clone()
            sr.sort_pairs(xk, xv, key_type=sr.KEY_U64)
    elif args.profile_form == "learned":
        src = torch.from_numpy(si.lognormal_f32(n, SEED)).cuda()
        for _ in range(2):
            x = src.clone()
            sr.sort_keys_learned(x)
    elif args.profile_form == "batched":
        from paper_1609_04471_gb300 import autotune
        keys, off, _ = si.segmented_i32(200_000, SEED)
        src = torch.from_numpy(keys).cuda()
        toff = torch.from_numpy(off).cuda()
        best = args.profile_config
        if best < 0:
            best = autotune.select_best(autotune.time_configs(src, toff, sr.KEY_I32, reps=1, warmup=0))
        for _ in range(2):
            x = src.clone()
            sr.sort_segmented_cfg(x, toff, best)
    else:
        src = torch.from_numpy(si.int32_input(args.profile_class, n, SEED)).cuda()
        for _ in range(2):
            x = src.clone()
            sr.sort_keys(x)
    torch.cuda.synchronize()
    st = sr.stats()
    print(json.dumps({"profile_case": args.profile_case, "pairs": bool(args.profile_pairs),
                      "form": args.profile_form, "class": args.profile_class, "input_class": st["input_class"],
                      "bytes_moved": st["bytes_moved"],
                      "passes_planned": st["passes_planned"], "passes_skipped": st["passes_skipped"], "ok": True}))


def _classes(sr, torch, reps=5):
    """The paper's input classes with a parameter k (Section 2) at 2^24 int32
    keys: per class the sort time (median of `reps` after 3 warm-ups, L2
    flushed, input restored untimed), the path the call took and the merge
    steps it skipped.  Every output is compared with numpy's sort of the same
    keys (the parity tests compare them with the oracle)."""
    import numpy as np
    import sortrace_inputs as si
    n = 1 << 24
    classes = {
        "random": lambda: si.uniform_i32(n, SEED),
        "k-limited, k=12": lambda: si.k_limited(n, 12, SEED),
        "k-equal teeth, k=8": lambda: si.k_equal_teeth(n, 8),
        "k-even teeth, k=8": lambda: si.k_even_teeth(n, 8),
        "k-sharp teeth, k=8": lambda: si.k_sharp_teeth(n, 8),
        "k-shuffled teeth, k=8": lambda: si.k_shuffled_teeth(n, 8, SEED),
        "k-distance, k=256": lambda: si.k_distance(n, 256, SEED),
        "k-exchange, k=n/100": lambda: si.k_exchange(n, n // 100, SEED),
    }
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {}
    for name, gen in classes.items():
        a = gen()
        src = torch.from_numpy(a).cuda()
        x = torch.empty_like(src)
        ts = []
        for r in range(3 + reps):
            x.copy_(src)
            flush.fill_(r & 0xFF)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sr.sort_keys(x)
            e1.record()
            torch.cuda.synchronize()
            if r >= 3:
                ts.append(e0.elapsed_time(e1))
        ok = bool(np.array_equal(x.cpu().numpy(), np.sort(a)))
        st = sr.stats()
        ms = float(np.median(ts))
        out[name] = {"ms": round(ms, 4), "gkeys_s": round(n / (ms / 1e3) / 1e9, 2), "ok": ok,
                     "input_class": st["input_class"], "runs": st["runs"],
                     "passes_planned": st["passes_planned"], "passes_skipped": st["passes_skipped"],
                     "bytes_moved": st["bytes_moved"]}
        del src, x
    return out


def run_classes(args):
    import torch
    import paper_1609_04471_gb300 as sr
    torch.cuda.set_device(0)
    sr.load()
    out = _classes(sr, torch)
    print(json.dumps({"classes": out, "n": 1 << 24, "key": "int32", "data": "synthetic (Section 2 generators)"}))


def _timed(torch, stream, fn, restore, reps):
    """Best device time (ms) of fn() over reps runs, each after restore()
    (the restore is not timed) and an L2 flush."""
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    best = None
    for r in range(reps + 1):
        restore()
        flush.fill_(r & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    return best


def _forms(sr, torch, dev, stream, peak):
    """The other forms of the sort on their own workloads:
    pairs    2^28 stable uint64-key + uint32-payload sort (half uniform, half
             Zipf 1.1 over 2^20 values);
    learned  2^27 float32 keys of the lognormal mixture, learned partition
             against the plain sort on the same input (and the untrained
             quantile start and the model-free equal-width ablation, the latter
             also under its own best bucket-sort configuration);
    batched  200,000 int32 arrays (lognormal lengths, median 512, four
             classes), the segmented sort under the autotuner's configuration
             replayed from a captured CUDA graph,
             against one plain sort call per array (on the first 2,000 arrays,
             scaled per key)."""
    import numpy as np
    import sortrace_inputs as si
    out = {}
    # pairs
    k, v = si.pairs_u64_zipf(1 << 28, SEED)
    pk = torch.from_numpy(k.view(np.int64)).to(dev)
    pv = torch.from_numpy(v.view(np.int32)).to(dev)
    del k, v
    wk, wv = torch.empty_like(pk), torch.empty_like(pv)
    ms = _timed(torch, stream, lambda: sr.sort_pairs(wk, wv, key_type=sr.KEY_U64),
                lambda: (wk.copy_(pk), wv.copy_(pv)), 2)
    st = sr.stats()
    n = 1 << 28
    out["pairs_2^28_u64_u32"] = {"ms": ms, "gkeys_s": n / (ms / 1e3) / 1e9,
                                 "passes_frac": st["bytes_moved"] / (ms / 1e3) / 1e9 / peak,
                                 "passes_frac_nominal": st["bytes_moved"] / (ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                                 "lower_bound_frac": 24 * n / (ms / 1e3) / 1e9 / peak}
    del pk, pv, wk, wv
    torch.cuda.empty_cache()
    # learned vs plain
    a = si.lognormal_f32(1 << 27, SEED)
    src = torch.from_numpy(a).to(dev)
    del a
    x = torch.empty_like(src)
    n = 1 << 27
    plain = _timed(torch, stream, lambda: sr.sort_keys(x), lambda: x.copy_(src), 3)
    learned = _timed(torch, stream, lambda: sr.sort_keys_learned(x), lambda: x.copy_(src), 3)
    stl = sr.stats()
    untrained = _timed(torch, stream, lambda: sr.sort_keys_learned(x, model=sr.MODEL_UNTRAINED),
                       lambda: x.copy_(src), 2)
    stu = sr.stats()
    ew = _timed(torch, stream, lambda: sr.sort_keys_learned(x, model=sr.MODEL_EQUAL_WIDTH), lambda: x.copy_(src), 2)
    ste = sr.stats()
    # the ablation under its own best bucket-sort configuration, for a fair comparison
    ew_cfg = {c["index"]: _timed(torch, stream,
                                 lambda: sr.sort_keys_learned(x, model=sr.MODEL_EQUAL_WIDTH, bucket_config=c["index"] + 1),
                                 lambda: x.copy_(src), 1)
              for c in sr.segmented_configs(sr.KEY_F32) if c["strategy"] == 1}
    out["learned_2^27_f32_lognormal"] = {
        "plain_ms": plain, "learned_ms": learned, "untrained_ms": untrained, "equal_width_ms": ew,
        "equal_width_best_ms": min(ew_cfg.values()),
        "equal_width_best_bucket_config": min(ew_cfg, key=ew_cfg.get),
        "plain_gkeys_s": n / (plain / 1e3) / 1e9, "learned_gkeys_s": n / (learned / 1e3) / 1e9,
        "learned_over_plain": plain / learned,
        "fallback": stl["fallback"], "model_loss": stl["model_loss"], "model_loss_untrained": stu["model_loss"],
        "bucket_imbalance": stl["bucket_imbalance"], "bucket_imbalance_equal_width": ste["bucket_imbalance"],
        "max_bucket": stl["max_bucket"]}
    del src, x
    torch.cuda.empty_cache()
    # batched segmented vs per-array: the autotuner times every launch
    # configuration on this batch (untimed here), the winner is captured in a
    # CUDA graph and replayed
    from paper_1609_04471_gb300 import autotune
    keys, off, _ = si.segmented_i32(200_000, SEED)
    n = int(off[-1])
    src = torch.from_numpy(keys).to(dev)
    toff = torch.from_numpy(off).to(dev)
    x = torch.empty_like(src)
    cand = autotune.time_configs(src, toff, sr.KEY_I32, reps=2)
    best = autotune.select_best(cand)
    cfgs = {c["index"]: c for c in sr.segmented_configs(sr.KEY_I32)}
    x.copy_(src)
    sr.sort_segmented_cfg(x, toff, best)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            sr.sort_segmented_cfg(x, toff, best)
    torch.cuda.synchronize()
    graph_ms = _timed(torch, stream, g.replay, lambda: x.copy_(src), 3)
    sts = sr.stats()
    eager_ms = _timed(torch, stream, lambda: sr.sort_segmented_cfg(x, toff, best), lambda: x.copy_(src), 3)
    default_ms = _timed(torch, stream, lambda: sr.sort_segmented_ex(x, toff), lambda: x.copy_(src), 3)
    sample = 2000
    views = [x[int(off[i]):int(off[i + 1])] for i in range(sample)]
    sample_keys = int(off[sample])

    def per_array():
        for v in views:
            sr.sort_keys(v)
    per_ms = _timed(torch, stream, per_array, lambda: x.copy_(src), 2)
    # the same keys as one array in one plain call (a different output: one
    # sorted array instead of 200,000), for scale
    one_ms = _timed(torch, stream, lambda: sr.sort_keys(x), lambda: x.copy_(src), 2)
    out["batched_200k_arrays_i32"] = {
        "keys": n, "graph_ms": graph_ms, "eager_ms": eager_ms,
        "graph_gkeys_s": n / (graph_ms / 1e3) / 1e9,
        "per_array_sample_arrays": sample, "per_array_sample_keys": sample_keys, "per_array_ms": per_ms,
        "per_array_gkeys_s": sample_keys / (per_ms / 1e3) / 1e9,
        "batched_over_per_array": (n / graph_ms) / (sample_keys / per_ms),
        "one_plain_call_ms": one_ms, "one_plain_call_gkeys_s": n / (one_ms / 1e3) / 1e9,
        "batched_over_one_plain_call": one_ms / graph_ms,
        "big_segments": sts["big_segments"],
        "autotuned": {"config": best,
                      "shape": {k: cfgs[best][k] for k in ("strategy", "sort_threads", "pack_items",
                                                           "tile_items", "fan_in", "ladder")},
                      "candidates_ms": {str(c): round(v, 4) for c, v in sorted(cand.items())},
                      "default_config_ms": default_ms}}
    del g
    return out


def main():
    args = _args()
    if args.classes:
        run_classes(args)
        return
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
