#!/usr/bin/env python
"""Throughput benchmark of the GB300 Wally server path.

One step = one whole batch of the workload (default: the full-scale batch,
3.2M x 192 database in 1,800 clusters, 500,000 real queries plus the
negative-binomial fakes of every client) evaluated end to end on the device:
grouping by cluster, inputs to NTT form, g-1 baby-step rotations, the grouped
plaintext x ciphertext products, h-1 giant-step rotations, outputs to
coefficient form.  Inputs are resident in HBM when the timed region starts
(they are far larger than L2: a 2,048-client pool of submissions and the
~91 GB encoded database).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank evaluates its own copy of the batch (independent
replicas; weak scaling; the only collectives are the timing barrier and the
max-over-ranks of the step time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted similarity QPS @3.2M×192, 500k batch, 1 GB300 (bit-exact); p50/p99 latency"


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- recorded ncu traffic

KERNEL_SOURCES = ["paper_2406_06761_gb300/csrc/kernels.cu", "paper_2406_06761_gb300/csrc/common.cuh",
                  "paper_2406_06761_gb300/csrc/kernels.hpp"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, items_per_launch: float | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary in
    profiles/ (a launch of 1,024 items), scaled to `items_per_launch` items
    (the key-switch kernels' traffic grows in proportion to the items), or
    None when that capture was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}_1024_items.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_source_sha256") != kernel_source_hash():
        return None
    try:
        b = float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None
    return b if items_per_launch is None else b / 1024.0 * items_per_launch


# ---------------------------------------------------------------- algorithmic work

def modmuls_per_kind(L: int, N: int, log_n: int, ks_count: int, mac_pairs: int, g: int, h: int) -> dict:
    """64-bit modular multiplications the method performs, per kernel kind,
    for `ks_count` key switches and `mac_pairs` (query, chunk) products: an
    NTT of N points is N/2 log2 N butterflies (one product each) plus N for the
    inverse's N^-1; a key switch is L inverse NTTs (digits), L^2 NTTs (digits
    into the other moduli) + 2(L+1)L key products + 2 inverse NTTs (ModDown
    residue mod P), then 2L NTTs + 2LN P^-1 products; a (query, chunk)
    product is g*h*2*L*N multiply-accumulates."""
    ntt = N // 2 * log_n
    return {
        "ks_a": ks_count * L * (ntt + N),
        "ks_b": ks_count * ((L * L) * ntt + 2 * (ntt + N) + 2 * (L + 1) * L * N),
        "ks_c": ks_count * (2 * L * ntt + 2 * L * N),
        "mac": mac_pairs * g * h * 2 * L * N,
    }


# ---------------------------------------------------------------- the oracle arm

_ORACLE_PREP = {}


def _oracle_prepare(workload: str, seed: int = 0) -> dict:
    """The oracle's inputs for a bounded sample of the workload (built once):
    the cluster the first query names, encoded; one client submission per
    host core; the single-thread latency of one query."""
    key = (workload, seed)
    if key in _ORACLE_PREP:
        return _ORACLE_PREP[key]
    import numpy as np
    import oracle as O
    from paper_2406_06761_gb300 import workload as W
    w = W.WORKLOADS[workload]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    cores = os.cpu_count() or 1
    sizes = W.cluster_sizes(w, seed)
    ids, is_real = W.query_mix(w, sizes, seed)
    c0 = int(ids[0])
    rows = np.cumsum(sizes) - sizes
    emb = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound, seed)
    m0, pt0 = O.encode_cluster(prm, emb[rows[c0]:rows[c0] + sizes[c0]])
    cl = [(m0, O.ptxt_to_ntt(prm, m0, pt0))]
    cr = W.client_randomness(cores, prm.N, prm.q, prm.P, seed, index=999)
    qv = W.query_vectors(cores, w.dim, w.entry_bound, seed, index=999)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(cores)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qv[i], cr.enc_a[i], cr.enc_e[i]) for i in range(cores)])
    t0 = time.perf_counter()
    O.eval_batch(prm, cl, np.zeros(1, np.uint32), cts[:1], keys[:1], nthreads=1)
    single = time.perf_counter() - t0
    prep = dict(prm=prm, cores=cores, cl=cl, cts=cts, keys=keys, single=single, m0=m0,
                config={"workload": workload, "queries": int(len(ids)), "real_queries": int(is_real.sum()),
                        "clusters": int(len(sizes)), "embeddings": int(sizes.sum()), "N": prm.N, "L": prm.L,
                        "d": prm.d, "g": prm.g, "h": prm.h})
    _ORACLE_PREP[key] = prep
    return prep


def oracle_sample_qps(workload: str, seconds: float, seed: int = 0) -> dict:
    """Time the CPU oracle on a bounded sample of the workload's queries, on
    every host core.  Returns {value, unit, cores, sample, kind}."""
    import numpy as np
    import oracle as O
    p = _oracle_prepare(workload, seed)
    prm, cores, single = p["prm"], p["cores"], p["single"]
    per_round = single * 1.15  # all cores busy: a little slower per query
    rounds = max(1, int(seconds / per_round))
    n = rounds * cores
    sel = np.arange(n) % cores
    t0 = time.perf_counter()
    O.eval_batch(prm, p["cl"], np.zeros(n, np.uint32), p["cts"][sel], p["keys"][sel], nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} queries of the {workload} workload (N={prm.N}, L={prm.L}, one {p['m0']}-chunk cluster), "
                      f"{cores} threads, {dt:.1f} s; single-thread latency {single * 1e3:.0f} ms/query",
            "single_thread_ms": single * 1e3}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    k, w = args.steps, args.warmup
    per_step = max(5.0, min(60.0, 150.0 / max(1, k + w)))
    vals = []
    res = None
    for i in range(w + k):
        res = oracle_sample_qps(args.workload, per_step)
        if i >= w:
            vals.append(res["value"])
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus, "steps": k, "warmup": w,
            "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": dict(_oracle_prepare(args.workload)["config"], note="CPU oracle on a bounded sample per step"),
            "cpu_baseline": {"value": v, "unit": "queries/s", "kind": "oracle", "cores": res["cores"],
                             "sample": res["sample"]},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def autotune(wl, Wl):
    """Pick the launch shapes (wave size, lanes, MAC and transform CTAs per
    SM) with the library's autotuner (staged search) on a sample of the
    batch, before any timing.  N = 16384 uses a smaller grid and sample (a
    wave workspace of 130 MB a query)."""
    import torch
    t0 = time.perf_counter()
    if wl.ctx.info.log_n >= 14:
        cands = [dict(max_wave=w, lanes=l, mac_ctas_per_sm=3, ntt_ctas_per_sm=0) for w in (64, 128, 256) for l in (1, 2)]
        sample = 512
    else:
        cands, sample = None, 16384  # four waves a lane of the largest wave size
    b = wl.device_batch(0, min(wl.n, sample))
    out = wl.alloc_out(b[3])
    best, table = Wl.wally_autotune(wl.ctx.ptr, b[0].numel(), b[0], wl.pool.cts, wl.pool.keys, b[1], b[2], out,
                                    candidates=cands, reps=2)
    del out
    torch.cuda.empty_cache()
    ranked = sorted((t for t in table if t[1] > 0), key=lambda t: t[1])
    res = {"chosen": table[best][0], "sample_queries": int(b[0].numel()), "candidates": len(table),
           "skipped_out_of_memory": sum(1 for t in table if t[1] < 0), "seconds": time.perf_counter() - t0,
           "fastest": [{"shape": sh, "us_per_query": ms * 1e3} for sh, ms in ranked[:5]],
           "slowest": {"shape": ranked[-1][0], "us_per_query": ranked[-1][1] * 1e3} if ranked else None}
    log("autotune", res)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="full_scale")
    ap.add_argument("--pool", type=int, default=2048)
    ap.add_argument("--max-wave", type=int, default=0, help="fixed wave size (no autotuning)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--shape", default=None, help="fixed launch shape max_wave,lanes,mac_ctas,ntt_ctas (no autotuning)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--real-queries", type=int, default=None, help="override the batch size (testing)")
    ap.add_argument("--serving", action="store_true", help="measure the serving loop instead of the batch")
    ap.add_argument("--serving-seconds", type=float, default=10.0)
    ap.add_argument("--pir", action="store_true", help="measure the metadata fetch (keyword PIR) instead")
    ap.add_argument("--pir-clients", type=int, default=64)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.pir:
        return run_pir(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2406_06761_gb300 import harness as H
    from paper_2406_06761_gb300 import multigpu as M
    from paper_2406_06761_gb300 import wally as Wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    Wl.load()
    peaks = Wl.wally_measure_int_peaks(local)
    log("integer peaks", {k: f"{v:.3e}" for k, v in peaks.items()})

    t_setup = time.perf_counter()
    wl = H.DeviceWorkload(args.workload, device=local, pool=args.pool, max_wave=args.max_wave,
                          real_queries=args.real_queries, keep_embeddings=False, verbose=(rank == 0))
    tuning = None
    if args.shape:
        w_, l_, m_, k_ = (int(v) for v in args.shape.split(","))
        Wl.wally_set_tuning(wl.ctx.ptr, w_, l_, m_, k_)
        tuning = {"chosen": Wl.wally_get_tuning(wl.ctx.ptr).as_dict(), "fixed": True}
    elif not args.max_wave and not args.no_autotune:
        tuning = autotune(wl, Wl)
    wl.ctx.refresh()
    info = wl.ctx.info
    n = wl.n
    n_real = int(wl.is_real.sum())
    # allocate both lanes' workspaces (a call of two waves), then size the output buffer
    b0 = wl.device_batch(0, min(n, int(info.max_wave) + 1))
    tmp = wl.alloc_out(b0[3])
    wl.eval(b0, tmp)
    Wl.wally_sync(wl.ctx.ptr)
    del tmp
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(dev)
    total_chunks = int(wl.chunks[wl.ids].sum())
    out_bytes_all = total_chunks * wl.ctw * 8
    budget = int(free * 0.85) - (2 << 30)
    subs = wl.sub_batches(None if out_bytes_all <= budget else budget)
    batches = [wl.device_batch(lo, hi) for lo, hi in subs]
    max_chunks = max(b[3] for b in batches)
    out = wl.alloc_out(max_chunks)
    setup_s = time.perf_counter() - t_setup
    log(f"setup {setup_s:.1f}s: {n} queries ({n_real} real), {len(wl.sizes)} clusters, "
        f"{info.total_chunks} chunks ({info.cluster_bytes / 1e9:.1f} GB), {len(subs)} sub-batch(es), "
        f"output buffer {max_chunks * wl.ctw * 8 / 1e9:.1f} GB")

    stream = torch.cuda.current_stream(dev)

    def step(record=None):
        for b in batches:
            wl.eval(b, out[:b[3]], stream)
            if record is not None:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                record.append((ev, b[0].numel()))

    for i in range(args.warmup):
        t0 = time.perf_counter()
        step()
        Wl.wally_sync(wl.ctx.ptr)
        log(f"warm-up {i}: {time.perf_counter() - t0:.2f}s")

    clocks = ClockSampler(local)
    clocks.start()
    Wl.wally_profile_enable(wl.ctx.ptr, True)
    M.barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    marks = []
    start.record(stream)
    for _ in range(args.steps):
        step(marks)
    end.record(stream)
    torch.cuda.synchronize(dev)
    M.barrier()
    Wl.wally_sync(wl.ctx.ptr)
    ms_total = start.elapsed_time(end)
    prof = Wl.wally_profile_read(wl.ctx.ptr)
    Wl.wally_profile_enable(wl.ctx.ptr, False)
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    ms_step = M.max_over_ranks(ms_step, device=dev)
    value = world * n / (ms_step / 1e3)

    # latency: completion time of each query's sub-batch within its step
    lat = []
    for ev, cnt in marks[:len(batches)]:
        lat += [start.elapsed_time(ev)] * cnt
    lat = np.array(lat)
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))

    # roofline of the dominant kernel
    g, h, L, N = info.g, info.h, info.num_q, info.n
    pairs = int(wl.chunks[wl.ids].sum())
    ks_count = args.steps * (n * (g - 1) + pairs * (h - 1))
    work = modmuls_per_kind(L, N, info.log_n, ks_count, args.steps * pairs, g, h)
    kern = {}
    for kind, (launches, tms) in prof.items():
        kern[kind] = {"launches": launches, "total_ms": tms, "share": tms / max(1e-9, sum(v[1] for v in prof.values()))}
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    roof = None
    if dom in work:
        # waves overlap on two streams, so a kernel's event time includes time
        # shared with the other stream's kernels: attribute the step time to
        # kernels by their share of the summed event time
        achieved = work[dom] / (kern[dom]["share"] * ms_step * args.steps / 1e3)
        peak = peaks["mac128_per_s"] if dom == "mac" else peaks["butterfly_per_s"]
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": peak / 1e9,
                "unit": "Gmodmul/s", "frac": achieved / peak, "traffic": recorded_traffic(dom, ks_count / max(1, kern[dom]["launches"]) if dom.startswith("ks_") else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 1,024-item launch "
                                  "(profiles/), scaled to this run's mean items per launch",
                "peak_source": "measured: wally_measure_int_peaks (" +
                               ("128-bit multiply-accumulate" if dom == "mac" else "NTT butterfly") +
                               " throughput, all SMs, this GPU)",
                "avg_launch_ms": kern[dom]["total_ms"] / kern[dom]["launches"]}
    alg_bytes_q = 8 * (wl.ctw + wl.keysw + wl.ctw * float(wl.chunks[wl.ids].mean()))
    hbm_ctx = {"algorithmic_bytes_per_query": alg_bytes_q,
               "achieved_GBps": value / world * alg_bytes_q / 1e9,
               "peak_GBps": 6790.0, "frac_of_measured_hbm": value / world * alg_bytes_q / 1e9 / 6790.0}

    # the plain one-query-at-a-time GPU path: each query its own call, waited for
    single = None
    if rank == 0:
        one = []
        for qi in range(0, min(n, 200)):
            b = wl.device_batch(qi, qi + 1)
            o1 = wl.alloc_out(b[3]) if qi == 0 or b[3] > o1.shape[0] else o1
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            wl.eval(b, o1[:b[3]], stream)
            torch.cuda.synchronize(dev)
            one.append(time.perf_counter() - t0)
        one = np.array(one[5:])
        single = {"value": 1.0 / float(one.mean()), "unit": "queries/s", "latency_ms_p50": float(np.median(one) * 1e3),
                  "latency_ms_p99": float(np.percentile(one, 99) * 1e3), "queries": int(len(one)),
                  "note": "one query per wally_eval_batch call, synchronised"}
        log("one query at a time", single)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        del out, batches
        torch.cuda.empty_cache()
        e2e = run_e2e(wl, subs, args, dev)
        if world > 1:
            # whole job: every rank's batch over the slowest rank's time
            dt = M.max_over_ranks(e2e["seconds"], device=dev)
            e2e.update(value=world * n / dt, seconds=dt, h2d_bytes_per_step=world * e2e["h2d_bytes_per_step"],
                       d2h_bytes_per_step=world * e2e["d2h_bytes_per_step"])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = oracle_sample_qps(args.workload, args.cpu_seconds)
        except Exception as ex:  # the oracle is optional on the GPU machine
            cpu = {"value": None, "error": str(ex)[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "queries": n, "real_queries": n_real, "clusters": int(len(wl.sizes)),
                   "embeddings": int(wl.sizes.sum()), "N": N, "L": L, "d": info.dim, "g": g, "h": h,
                   "client_pool": wl.pool_size, "sub_batches": len(subs), "max_wave": int(info.max_wave),
                   "store": "compact" if info.store == Wl.STORE_COMPACT else "ntt",
                   "l2": f"inputs larger than L2 ({info.cluster_bytes / 1e9:.1f} GB cluster store, "
                         f"{wl.pool_size * (wl.ctw + wl.keysw) * 8 / 1e9:.1f} GB client pool); no flush"},
        "real_qps": world * n_real / (ms_step / 1e3),
        "latency_ms": {"p50": p50, "p99": p99, "note": "completion time of the query's sub-batch within a step"},
        "gpu_launches": int(sum(v[0] for v in prof.values()) / args.steps),
        "roofline": roof,
        "kernels": kern,
        "hbm_context": hbm_ctx,
        "int_peaks": peaks,
        "clocks": clk,
        "e2e": e2e,
        "one_query_path": single,
        "tuning": tuning,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """The serving workload: the full-scale database, Poisson arrivals of real
    queries and every client's negative-binomial fakes, a 10 ms per-cluster
    grouping window, waves on two lanes.  Reports served QPS and p50/p99
    latency at 0.5x and 0.9x of the measured batch capacity and at the
    workload's nominal 50,000 queries/s."""
    import numpy as np
    import torch
    from paper_2406_06761_gb300 import harness as H
    from paper_2406_06761_gb300 import serving as S
    from paper_2406_06761_gb300 import wally as Wl
    from paper_2406_06761_gb300 import workload as W
    dev = torch.device("cuda", 0)
    w = W.WORKLOADS["serving"]
    wl = H.DeviceWorkload("full_scale", pool=args.pool, max_wave=args.max_wave, real_queries=20000,
                          keep_embeddings=False, verbose=True)
    # capacity: one 20k-query batch on lane 0
    b = wl.device_batch(0, wl.n)
    out = wl.alloc_out(b[3])
    wl.eval(b, out)
    Wl.wally_sync(wl.ctx.ptr)
    t0 = time.perf_counter()
    wl.eval(b, out)
    Wl.wally_sync(wl.ctx.ptr)
    capacity = wl.n / (time.perf_counter() - t0)
    del out
    torch.cuda.empty_cache()
    fake_fraction = float((~wl.is_real).mean())
    max_wave = int(wl.ctx.info.max_wave)
    srv = S.Server(wl.ctx.ptr, wl.chunks, wl.pool.cts, wl.pool.keys, lanes=2, window_ms=w.window_ms,
                   max_wave=max_wave)
    # allocate both lanes' workspaces before timing
    srv.run(S.poisson_stream(5 * max_wave / 0.05, 0.05, wl.sizes, wl.pool_size, fake_fraction, seed=99))
    results = {}
    for label, rate, secs in (("0.5x_capacity", 0.5 * capacity, args.serving_seconds),
                              ("0.9x_capacity", 0.9 * capacity, args.serving_seconds),
                              ("nominal_50k", w.arrival_qps, min(2.0, args.serving_seconds))):
        st = S.poisson_stream(rate, secs, wl.sizes, wl.pool_size, fake_fraction, seed=1)
        Wl.wally_profile_enable(wl.ctx.ptr, True)
        r = srv.run(st)
        prof = Wl.wally_profile_read(wl.ctx.ptr)
        Wl.wally_profile_enable(wl.ctx.ptr, False)
        tot = max(1e-9, sum(v[1] for v in prof.values()))
        r["kernel_share"] = {k: round(v[1] / tot, 3) for k, v in prof.items()}
        r["offered_rate_qps"] = rate
        results[label] = r
        log(label, {k: (round(v, 2) if isinstance(v, float) else v) for k, v in r.items()})
    line = {"metric": "serving: served QPS and p50/p99 latency, 3.2M x 192 database, 10 ms window",
            "value": results["0.9x_capacity"]["served_qps"], "unit": "queries/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "serving", "window_ms": w.window_ms, "lanes": 2, "max_wave": max_wave,
                       "batch_capacity_qps": capacity},
            "serving": results}
    print(json.dumps(line), flush=True)
    return 0


def run_pir(args):
    """The metadata fetch of Sec. 4.2: keyword PIR over one cluster's
    metadata (the full-scale database's mean cluster: 1,778 entries of 1 KB),
    split cuckoo tables, MulPIR with both dimensions at N = 8192, three
    50-bit limbs.  A lookup is two index PIR answers (one per table);
    reports lookups/s for a batch of clients with device-resident queries
    and keys, and checks the first lookups by decryption."""
    import numpy as np
    import torch
    from paper_2406_06761_gb300 import pir
    from paper_2406_06761_gb300 import wally as Wl
    from paper_2406_06761_gb300 import workload as W
    dev = torch.device("cuda", 0)
    w = W.WORKLOADS["batched"]
    rng = np.random.default_rng(11)
    entries = {}
    while len(entries) < 1778:
        entries[int(rng.integers(1, 2**63))] = bytes(rng.integers(0, 256, 1024, dtype=np.uint8))
    tab = pir.build(entries)
    (d1, d2) = tab.dims[0]
    servers = []
    for t in (0, 1):
        ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
        Wl.wally_pir_load(ctx.ptr, tab.plaintexts(t, ctx.N))
        servers.append(ctx)
    ctx0 = servers[0]
    N, L, q, P, tval = ctx0.N, ctx0.L, ctx0.q, ctx0.P, int(ctx0.info.t)
    n = args.pir_clients
    lv = (d1 + d2 - 1).bit_length()
    keys_list = list(entries)
    wanted = [keys_list[int(i)] for i in rng.integers(0, len(keys_list), n)]
    cr = W.pir_client_randomness(n, lv, N, q, P, seed=12)
    rc = W.client_randomness(n, N, q, P, seed=13)
    sec = torch.from_numpy(cr.secret).to(dev)
    keys = torch.empty((n, lv, L, 2, L + 1, N), dtype=torch.int64, device=dev)
    Wl.wally_keygen_galois(ctx0.ptr, n, pir.galois_elements(N, lv), sec,
                           Wl.u64_tensor(cr.key_a, dev), torch.from_numpy(cr.key_e).to(dev), keys)
    rlk = torch.empty((n, L, 2, L + 1, N), dtype=torch.int64, device=dev)
    Wl.wally_keygen_relin(ctx0.ptr, n, sec, Wl.u64_tensor(np.ascontiguousarray(rc.key_a[:, 0]), dev),
                          torch.from_numpy(np.ascontiguousarray(rc.key_e[:, 0])).to(dev), rlk)
    cts, outs = [], []
    for t in (0, 1):
        m = np.stack([pir.query_plaintext(N, tval, lv, *tab.position(k, t), d1=d1) for k in wanted])
        ct = torch.empty((n, 2, L, N), dtype=torch.int64, device=dev)
        Wl.wally_encrypt_poly(ctx0.ptr, n, sec, Wl.u64_tensor(m, dev), Wl.u64_tensor(cr.enc_a, dev),
                              torch.from_numpy(cr.enc_e).to(dev), ct)
        cts.append(ct)
        outs.append(torch.empty((n, 2, L, N), dtype=torch.int64, device=dev))

    def step():
        for t in (0, 1):
            Wl.wally_pir_answer2(servers[t].ptr, n, cts[t], keys, rlk, outs[t])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(args.steps):
        step()
    s1.record()
    torch.cuda.synchronize(dev)
    ms = s0.elapsed_time(s1) / args.steps
    ok = 0
    for t in (0, 1):
        coeffs = torch.empty((n, N), dtype=torch.int64, device=dev)
        Wl.wally_decrypt_poly(ctx0.ptr, n, sec, None, outs[t], coeffs)
        for i, row in enumerate(coeffs.cpu().numpy()):
            e = pir.unpack(row)
            if e is not None and e[0] == wanted[i] and e[1] == entries[wanted[i]]:
                ok += 1
    line = {"metric": "metadata fetch: keyword PIR lookups/s (split cuckoo tables, MulPIR, both dimensions)",
            "value": n / (ms / 1e3), "unit": "lookups/s", "n_gpus": 1, "higher_is_better": True,
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "metadata of one cluster", "entries": len(entries), "value_bytes": 1024,
                       "table_slots": tab.sizes[0], "d1": d1, "d2": d2, "expansion_levels": lv, "clients": n,
                       "N": N, "L": L},
            "checked_lookups": {"found": ok, "of": n}}
    print(json.dumps(line), flush=True)
    for ctx in servers:
        ctx.close()
    return 0


def run_e2e(wl, subs, args, dev):
    """Same metric through wally_eval_batch_host: the host holds the client
    pool (pinned) and receives every output; each query's ciphertext and keys
    are copied to the device and its score ciphertexts back, inside the timed
    region.  Outputs land in a reused pinned host buffer of one call."""
    import numpy as np
    import torch
    from paper_2406_06761_gb300 import wally as Wl
    cts_h = wl.pool.cts.cpu().pin_memory()
    keys_h = wl.pool.keys.cpu().pin_memory()
    # calls of at most ~16 GB of outputs each
    cap_q = max(1, int(16e9 // (8 * wl.ctw * max(1, int(wl.chunks.max())))))
    calls = []
    for lo, hi in subs:
        for a in range(lo, hi, cap_q):
            calls.append((a, min(hi, a + cap_q)))
    prepared = []
    max_chunks = 0
    for lo, hi in calls:
        ids = wl.ids[lo:hi]
        m = wl.chunks[ids]
        offs = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
        max_chunks = max(max_chunks, int(m.sum()))
        prepared.append((torch.from_numpy(ids.astype(np.int32)).pin_memory(),
                         torch.from_numpy(wl.input_index[lo:hi].astype(np.int32)).pin_memory(),
                         torch.from_numpy(offs).pin_memory(), int(m.sum())))
    out_h = torch.empty((max_chunks, 2, wl.L, wl.N), dtype=torch.int64).pin_memory()
    h2d = d2h = 0
    for ids, idx, offs, ch in prepared:
        h2d += ids.numel() * 8 * (wl.ctw + wl.keysw) + ids.numel() * 16
        d2h += ch * wl.ctw * 8

    def one():
        for ids, idx, offs, ch in prepared:
            Wl.wally_eval_batch_host(wl.ctx.ptr, ids.numel(), ids, cts_h, keys_h, idx, offs, out_h[:ch])
    from paper_2406_06761_gb300 import multigpu as M
    one()  # warm-up (pins, staging buffers)
    torch.cuda.synchronize(dev)
    M.barrier()
    t0 = time.perf_counter()
    one()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    M.barrier()
    return {"value": wl.n / dt, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "calls": len(prepared), "seconds": dt}


if __name__ == "__main__":
    sys.exit(main())
