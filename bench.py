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

Under torchrun the clusters are sharded over the ranks (each rank holds the
clusters it owns and evaluates the queries that name them, out of one batch
per rank: weak scaling); --placement replica gives every rank its own copy of
the database and of the batch instead.  The only collectives are the timing
barrier, the max-over-ranks of the step time and the sum of the queries.
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
                  "paper_2406_06761_gb300/csrc/kernels.hpp", "paper_2406_06761_gb300/csrc/ntt_regs.cuh"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, items_per_launch: float | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary in
    profiles/ (`ncu_<kernel>_<items>_items.md`, a launch of that many items
    of a small case), scaled to `items_per_launch` items (the key-switch
    kernels' traffic grows in proportion to the items), or None when no
    capture exists or it was taken on other kernel sources."""
    import glob
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", f"ncu_{kernel}_*_items.md")))
    for path in paths:
        fields = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_source_sha256") != kernel_source_hash():
            continue
        try:
            b = float(fields["dram_bytes_per_launch"])
            items = float(fields["items_per_launch"])
        except (KeyError, ValueError):
            continue
        return b if items_per_launch is None else b / items * items_per_launch
    return None


# ---------------------------------------------------------------- algorithmic work

def work_per_kind(L: int, N: int, log_n: int, queries: int, pairs: int, g: int, h: int) -> dict:
    """Modular operations the method performs in each kernel kind, split by
    class -- NTT butterflies (bfly), Shoup products by a constant (mm) and
    exact multiply-accumulates into 128-bit sums (mac) -- for `queries` queries with
    `pairs` (query, chunk) products in all.  A transform of N points is
    N/2 log2 N butterflies; an inverse adds N scalings by N^-1.  Key switch
    (ks_b): L^2 forward transforms of the digits into the other moduli, the
    2L(L+1)N key products, two inverse transforms of the P residue; ModDown
    (ks_c): 2L forward transforms and 2LN products by P^-1, then, except at the
    end of a chain, the next rotation's L digit inverse transforms (ks_a does
    those at the start of each chain).  Chains: g-1 baby-step rotations per
    query, h-1 giant-step rotations per (query, chunk)."""
    B = N // 2 * log_n
    ks = queries * (g - 1) + pairs * (h - 1)
    starts = queries * (1 if g > 1 else 0) + pairs * (1 if h > 1 else 0)
    nexts = ks - starts
    polys_in = 2 * L + 4 * L * (L + 1)
    return {
        "ks_a": {"bfly": starts * L * B, "mm": starts * L * N, "mac": 0},
        "ks_b": {"bfly": ks * (L * L + 2) * B, "mm": ks * 2 * N, "mac": ks * 2 * L * (L + 1) * N},
        "ks_c": {"bfly": ks * 2 * L * B + nexts * L * B, "mm": ks * 2 * L * N + nexts * L * N, "mac": 0},
        "mac": {"bfly": 0, "mm": 0, "mac": pairs * g * h * 2 * L * N},
        "to_ntt": {"bfly": queries * polys_in * B, "mm": queries * 4 * L * (L + 1) * N, "mac": 0},
        "output": {"bfly": pairs * 2 * L * B, "mm": pairs * 2 * L * N, "mac": 0},
    }


def butterfly_equivalents(work: dict, peaks: dict) -> float:
    """Work of one kind in butterflies: each class weighted by the ratio of
    the butterfly peak to its own measured peak."""
    pb = peaks["butterfly_per_s"]
    return work["bfly"] + work["mm"] * pb / peaks["modmul_per_s"] + work["mac"] * pb / peaks["mac128_per_s"]


# ---------------------------------------------------------------- batch latency

def batch_latency(marks, wave_call, wave_q, wave_ms) -> dict:
    """Per-query latency inside the timed steps: every query of a step is
    submitted at the step's start and is done when its wave's outputs are
    written.  marks: ("step", event) at each step's start and ("call", event)
    just before each evaluation call, in order (the library's call start is
    recorded on the same stream at the call's entry); wave_*: the library's
    per-wave records (call index, queries, milliseconds from the call's
    start)."""
    import numpy as np
    call_off, step_ev = [], None
    for kind, ev in marks:
        if kind == "step":
            step_ev = ev
        else:
            call_off.append(step_ev.elapsed_time(ev))
    if not len(wave_q) or len(call_off) <= int(wave_call.max()):
        return {"p50": None, "p99": None, "note": "no wave records"}
    lat = np.array([call_off[int(c)] for c in wave_call]) + wave_ms.astype(np.float64)
    per_query = np.repeat(lat, wave_q.astype(np.int64))
    return {"p50": float(np.percentile(per_query, 50)), "p99": float(np.percentile(per_query, 99)),
            "max": float(per_query.max()), "waves": int(len(wave_q)),
            "note": "per query: from the step's start (all queries submitted) to its wave's outputs written"}


# ---------------------------------------------------------------- the oracle arm

_ORACLE_PREP = {}


def stratified_sample(ids, chunks, n_sample: int, n_clusters: int, seed: int = 0):
    """A sample of the batch's queries for timing the oracle: n_clusters
    clusters picked evenly over the load quantiles (queries per cluster) plus
    every cluster of two or more chunks; the sample holds as many queries of
    each chunk count as the batch does in proportion (at least one), spread
    over the picked clusters of that chunk count in proportion to their load.
    A query's cost depends only on its cluster's chunk count, so the sample's
    queries/s extrapolate linearly to the batch.  Returns the cluster id of
    every sampled query."""
    import numpy as np
    K = len(chunks)
    load = np.bincount(ids, minlength=K)
    live = np.flatnonzero(load > 0)
    order = live[np.argsort(load[live], kind="stable")]
    pick = set(int(c) for c in order[np.linspace(0, len(order) - 1, min(n_clusters, len(order))).round().astype(int)])
    pick |= set(int(c) for c in live[chunks[live] >= 2])
    pick = np.array(sorted(pick))
    rng = np.random.default_rng([seed, 0xc0])
    out = []
    for m in np.unique(chunks[pick]):
        cl = pick[chunks[pick] == m]
        share = load[chunks == m].sum() / len(ids)
        k = max(1, int(round(n_sample * share)))
        w = load[cl] / load[cl].sum()
        cnt = np.floor(w * k).astype(int)
        rest = k - cnt.sum()
        if rest > 0:
            cnt[np.argsort(-(w * k - cnt), kind="stable")[:rest]] += 1
        out.append(np.repeat(cl, cnt))
    sample = np.concatenate(out)
    return sample[rng.permutation(len(sample))]


def _oracle_prepare(workload: str, seed: int = 0, n_sample: int = 1024, n_clusters: int = 64) -> dict:
    """The oracle's inputs for a stratified sample of the workload's batch
    (built once): the sampled clusters, encoded (in parallel, one cluster a
    thread), one client submission per host core (queries cycle over them),
    and the single-thread latency of one query."""
    key = (workload, seed, n_sample, n_clusters)
    if key in _ORACLE_PREP:
        return _ORACLE_PREP[key]
    import concurrent.futures as cf
    import numpy as np
    import oracle as O
    from paper_2406_06761_gb300 import workload as W
    w = W.WORKLOADS[workload]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    cores = os.cpu_count() or 1
    sizes = W.cluster_sizes(w, seed)
    ids, is_real = W.query_mix(w, sizes, seed)
    chunks = np.maximum(1, -(-sizes // prm.N))
    sample = stratified_sample(ids, chunks, n_sample, n_clusters, seed)
    picked = np.unique(sample)
    rows = np.cumsum(sizes) - sizes
    emb = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound, seed)

    def encode(c):
        m, pt = O.encode_cluster(prm, emb[rows[c]:rows[c] + sizes[c]])
        return m, O.ptxt_to_ntt(prm, m, pt)

    with cf.ThreadPoolExecutor(cores) as ex:
        enc = list(ex.map(encode, [int(c) for c in picked]))
    local = {int(c): i for i, c in enumerate(picked)}
    cr = W.client_randomness(cores, prm.N, prm.q, prm.P, seed, index=999)
    qv = W.query_vectors(cores, w.dim, w.entry_bound, seed, index=999)
    with cf.ThreadPoolExecutor(cores) as ex:
        keys = np.stack(list(ex.map(lambda i: O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]),
                                    range(cores))))
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qv[i], cr.enc_a[i], cr.enc_e[i]) for i in range(cores)])
    t0 = time.perf_counter()
    O.eval_batch(prm, enc, np.zeros(1, np.uint32), cts[:1], keys[:1], nthreads=1)
    single = time.perf_counter() - t0
    prep = dict(prm=prm, cores=cores, enc=enc, local=np.array([local[int(c)] for c in sample], np.uint32),
                cts=cts, keys=keys, single=single, n_clusters=len(picked),
                multi=int((chunks[sample] >= 2).sum()),
                config=workload_config(workload, seed))
    _ORACLE_PREP[key] = prep
    return prep


def workload_config(workload: str, seed: int = 0, pool: int = 2048) -> dict:
    """The workload's shape (both arms report the same keys): batch, database,
    parameters, client pool, and the statement about L2."""
    import numpy as np
    from paper_2406_06761_gb300 import workload as W
    w = W.WORKLOADS[workload]
    sizes = W.cluster_sizes(w, seed)
    ids, is_real = W.query_mix(w, sizes, seed)
    N, L = 1 << w.log_n, w.num_q
    d_pad = 1 << (w.dim - 1).bit_length()
    g = 1 << ((d_pad.bit_length() - 1 + 1) // 2)
    chunks = int(np.maximum(1, -(-sizes // N)).sum())
    ctw, keysw = 2 * L * N, 2 * L * 2 * (L + 1) * N
    pool = min(pool, len(ids))
    return {"workload": workload, "queries": int(len(ids)), "real_queries": int(is_real.sum()),
            "clusters": int(len(sizes)), "embeddings": int(sizes.sum()), "N": N, "L": L, "d": w.dim, "g": g,
            "h": d_pad // g, "client_pool": pool,
            "l2": f"inputs larger than L2 ({chunks * d_pad * L * N * 8 / 1e9:.1f} GB cluster store, "
                  f"{pool * (ctw + keysw) * 8 / 1e9:.1f} GB client pool); no flush"}


def oracle_sample_qps(workload: str, n_queries: int | None = None, seed: int = 0, offset: int = 0) -> dict:
    """Time the CPU oracle on every host core over n_queries of the
    stratified sample (all of it by default), starting at `offset` (the
    sample wraps around).  Returns {value, unit, cores, sample, kind,
    extrapolated}."""
    import numpy as np
    import oracle as O
    p = _oracle_prepare(workload, seed)
    prm, cores, single = p["prm"], p["cores"], p["single"]
    total = len(p["local"])
    n = total if n_queries is None else max(1, n_queries)
    idx = (offset + np.arange(n)) % total
    sel = np.arange(n) % cores
    t0 = time.perf_counter()
    O.eval_batch(prm, p["enc"], p["local"][idx], p["cts"][sel], p["keys"][sel], nthreads=cores)
    dt = time.perf_counter() - t0
    ncl = len(np.unique(p["local"][idx]))
    return {"value": n / dt, "unit": "queries/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"{n} queries of the {workload} batch over {ncl} clusters (stratified by load, "
                      f"queries of two-chunk clusters in the batch's proportion), N={prm.N}, L={prm.L}, "
                      f"{cores} threads, {dt:.1f} s; queries/s extrapolates linearly to the batch; "
                      f"single-thread latency {single * 1e3:.0f} ms/query",
            "single_thread_ms": single * 1e3, "queries": int(n), "clusters": int(ncl)}


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, each step a
    bounded slice of the stratified sample of the same batch (successive
    steps take successive slices, so the run covers the whole sample)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    k, w = args.steps, args.warmup
    p = _oracle_prepare(args.workload)
    per_step = max(5.0, min(60.0, 150.0 / max(1, k + w)))
    n_step = max(p["cores"], int(per_step / (p["single"] * 1.15)) * p["cores"])
    vals, qs, cls = [], 0, set()
    res = None
    for i in range(w + k):
        res = oracle_sample_qps(args.workload, n_step, offset=i * n_step)
        if i >= w:
            vals.append(res["value"])
            qs += res["queries"]
    v = statistics.mean(vals)
    covered = min(len(p["local"]), (w + k) * n_step)
    line = {"metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus, "steps": k, "warmup": w,
            "ms_per_step": n_step / v * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args.workload, pool=args.pool),
            "cpu_baseline": {"value": v, "unit": "queries/s", "kind": "oracle", "cores": res["cores"],
                             "extrapolated": True,
                             "sample": f"{k} timed steps of {n_step} queries each ({qs} queries) from a stratified "
                                       f"sample of {len(p['local'])} queries over {p['n_clusters']} clusters of the "
                                       f"{args.workload} batch ({covered} sample queries covered, warm-up included)"},
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
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape max_wave,lanes,mac_ctas,ntt_ctas[,ks_core] (no autotuning)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time plain calls instead of CUDA-graph replays")
    ap.add_argument("--placement", choices=["shard", "replica"], default="shard",
                    help="under torchrun: cluster shards (each rank holds its clusters and takes the queries that "
                         "name them out of one batch per rank) or replicas (each rank its own copy of the batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--real-queries", type=int, default=None, help="override the batch size (testing)")
    ap.add_argument("--clusters", type=int, default=None,
                    help="override the number of clusters (small cases for profiling)")
    ap.add_argument("--serving", action="store_true", help="measure the serving loop instead of the batch")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving loads of the default line")
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
    pipes = Wl.wally_measure_pipe_rates(local)
    log("integer peaks", {k: f"{v:.3e}" for k, v in peaks.items()})
    log("pipe rates", {k: f"{v:.3e}" for k, v in pipes.items()})

    t_setup = time.perf_counter()
    shard = (world, rank) if world > 1 and args.placement == "shard" else None
    wl = H.DeviceWorkload(args.workload, device=local, pool=args.pool, max_wave=args.max_wave,
                          real_queries=args.real_queries, num_clusters=args.clusters, keep_embeddings=False,
                          verbose=(rank == 0), shard=shard)
    tuning = None
    if args.shape:
        Wl.wally_set_tuning(wl.ctx.ptr, *(int(v) for v in args.shape.split(",")))
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
        if record is not None:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            record.append(("step", ev))
        for b in batches:
            if record is not None:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                record.append(("call", ev))
            wl.eval(b, out[:b[3]], stream)

    for i in range(args.warmup):
        t0 = time.perf_counter()
        step()
        Wl.wally_sync(wl.ctx.ptr)
        log(f"warm-up {i}: {time.perf_counter() - t0:.2f}s")

    # the timed steps replay each sub-batch's whole evaluation (grouping,
    # every wave, every kernel) captured once in a CUDA graph; launches
    # captured with profiling on are timed at every replay (the last replay's
    # times are read back)
    use_graph = not args.no_graph and info.store != Wl.STORE_COMPACT
    Wl.wally_profile_enable(wl.ctx.ptr, True)
    graphs = []
    if use_graph:
        for b in batches:
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, capture_error_mode="relaxed"):
                wl.eval(b, out[:b[3]])
            graphs.append(gr)
        torch.cuda.synchronize(dev)

        def step(record=None):  # noqa: F811 -- the graph form of the step
            if record is not None:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                record.append(("step", ev))
            for gr in graphs:
                if record is not None:
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(stream)
                    record.append(("call", ev))
                gr.replay()

    clocks = ClockSampler(local)
    clocks.start()
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
    wave_call, wave_q, wave_ms = Wl.wally_profile_waves(wl.ctx.ptr)
    prof = Wl.wally_profile_read(wl.ctx.ptr)
    Wl.wally_profile_enable(wl.ctx.ptr, False)
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    ms_step = M.max_over_ranks(ms_step, device=dev)
    # whole job: every rank's queries over the slowest rank's step time
    n_job = int(round(M.sum_over_ranks(n, device=dev)))
    n_real_job = int(round(M.sum_over_ranks(n_real, device=dev)))
    value = n_job / (ms_step / 1e3)

    # latency: a query's result is ready when its wave's outputs are written;
    # every query of a step is submitted at the step's start
    latency = batch_latency(marks[-(1 + len(batches)):] if use_graph else marks, wave_call, wave_q, wave_ms)
    if use_graph:
        latency["note"] += " (the last timed step: captured events hold the latest replay)"
    launches_per_step = int(sum(v[0] for v in prof.values()) / (1 if use_graph else args.steps))
    del graphs

    # roofline of the dominant kernel
    g, h, L, N = info.g, info.h, info.num_q, info.n
    pairs = int(wl.chunks[wl.ids].sum())
    ks_count = args.steps * (n * (g - 1) + pairs * (h - 1))
    work = work_per_kind(L, N, info.log_n, args.steps * n, args.steps * pairs, g, h)
    kern = {}
    for kind, (launches, tms) in prof.items():
        kern[kind] = {"launches": launches, "total_ms": tms, "share": tms / max(1e-9, sum(v[1] for v in prof.values()))}
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    roof = None
    if dom in work:
        # waves overlap on two streams, so a kernel's event time includes time
        # shared with the other stream's kernels: attribute the step time to
        # kernels by their share of the summed event time
        t_dom = kern[dom]["share"] * ms_step * args.steps / 1e3
        eq = butterfly_equivalents(work[dom], peaks)
        achieved = eq / t_dom
        pb, ceil = peaks["butterfly_per_s"], pipes["bfly_ceiling_per_s"]
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": pb / 1e9,
                "unit": "Gbutterfly/s", "frac": achieved / pb, "frac_vs_probe": achieved / pb,
                "frac_vs_issue": achieved / ceil, "issue_ceiling": ceil / 1e9,
                "work": {k: float(v) for k, v in work[dom].items()},
                "traffic": recorded_traffic(dom, ks_count / max(1, kern[dom]["launches"] * (args.steps if use_graph else 1))
                                           if dom.startswith("ks_") else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of a small case "
                                  "(profiles/), scaled to this run's mean items per launch",
                "peak_source": "measured: wally_measure_int_peaks (the transforms' forward butterfly in registers, "
                               "all SMs, this GPU); Shoup products and exact multiply-accumulates counted as "
                               "butterflies by the ratio of their own measured peaks",
                "issue_source": "measured: wally_measure_pipe_rates (2 mul.hi + 3 mad.wide + 4 mad.lo a butterfly "
                                "on the integer multiplier)",
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
            e2e.update(value=n_job / dt, seconds=dt,
                       h2d_bytes_per_step=M.sum_over_ranks(e2e["h2d_bytes_per_step"], device=dev),
                       d2h_bytes_per_step=M.sum_over_ranks(e2e["d2h_bytes_per_step"], device=dev))

    if args.real_queries is None and args.clusters is None:
        config = dict(workload_config(args.workload, pool=wl.pool_size))
        if info.store == Wl.STORE_COMPACT:
            config["l2"] = (f"inputs larger than L2 ({info.cluster_bytes / 1e9:.1f} GB of resident embeddings, "
                            f"{wl.pool_size * (wl.ctw + wl.keysw) * 8 / 1e9:.1f} GB client pool); no flush")
    else:
        config = {"workload": args.workload, "queries": n, "real_queries": n_real, "clusters": int(len(wl.sizes)),
                  "embeddings": int(wl.sizes.sum()), "N": N, "L": L, "d": info.dim, "g": g, "h": h,
                  "client_pool": wl.pool_size,
                  "l2": f"inputs larger than L2 ({info.cluster_bytes / 1e9:.1f} GB cluster store, "
                        f"{wl.pool_size * (wl.ctw + wl.keysw) * 8 / 1e9:.1f} GB client pool); no flush"}
    if shard is None:
        assert config["queries"] == n and config["N"] == N and config["g"] == g, "workload shape mismatch"
    else:
        config["batches"] = world  # one batch per rank, routed to the owners of the clusters
    # the serving loop over the same database and client pool, at 0.5x and
    # 0.9x of the batch capacity just measured
    served = None
    if rank == 0 and not args.no_serving and args.workload == "full_scale":
        try:
            del out, batches
        except NameError:
            pass
        torch.cuda.empty_cache()
        cap = value / world
        served = serving_loads(wl, cap, [("0.5x_capacity", 0.5 * cap), ("0.9x_capacity", 0.9 * cap)],
                               args.serving_seconds)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = oracle_sample_qps(args.workload)
        except Exception as ex:  # the oracle is optional on the GPU machine
            cpu = {"value": None, "error": str(ex)[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config,
        "launch": {"sub_batches": len(subs), "max_wave": int(info.max_wave), "graph": use_graph,
                   "placement": ("cluster shards" if shard else "replicas") if world > 1 else "one GPU",
                   "store": "compact" if info.store == Wl.STORE_COMPACT else "ntt"},
        "real_qps": n_real_job / (ms_step / 1e3),
        "latency_ms": latency,
        "gpu_launches": launches_per_step,
        "roofline": roof,
        "kernels": kern,
        "hbm_context": hbm_ctx,
        "int_peaks": peaks,
        "pipe_rates": pipes,
        "clocks": clk,
        "e2e": e2e,
        "serving": served,
        "one_query_path": single,
        "tuning": tuning,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def serving_loads(wl, capacity: float, loads, seconds: float, max_wave: int = 1024, lanes: int = 2) -> dict:
    """Serve the anonymised request stream of the serving workload (Poisson
    arrivals, one real query and NB(0.5, 0.9) fakes per client, 10 ms
    per-cluster grouping window) over wl's database and client pool at each
    offered rate of `loads` ((label, rate, seconds) or (label, fraction of
    `capacity`)); returns served QPS, p50/p99 latency and per-kernel shares
    for each."""
    from paper_2406_06761_gb300 import serving as S
    from paper_2406_06761_gb300 import wally as Wl
    from paper_2406_06761_gb300 import workload as W
    w = W.WORKLOADS["serving"]
    srv = S.Server(wl.ctx.ptr, wl.chunks, wl.pool.cts, wl.pool.keys, lanes=lanes, window_ms=w.window_ms,
                   max_wave=max_wave)
    # allocate the lanes' workspaces before timing
    srv.run(S.poisson_stream(5 * max_wave / 0.05, 0.05, wl.sizes, wl.pool_size, w.nb_r, w.nb_p, seed=99))
    results = {}
    for item in loads:
        label, rate = item[0], item[1]
        secs = item[2] if len(item) > 2 else seconds
        st = S.poisson_stream(rate, secs, wl.sizes, wl.pool_size, w.nb_r, w.nb_p, seed=1)
        Wl.wally_profile_enable(wl.ctx.ptr, True)
        r = srv.run(st)
        prof = Wl.wally_profile_read(wl.ctx.ptr)
        Wl.wally_profile_enable(wl.ctx.ptr, False)
        tot = max(1e-9, sum(v[1] for v in prof.values()))
        r["kernel_share"] = {k: round(v[1] / tot, 3) for k, v in prof.items()}
        r["offered_rate_qps"] = rate
        r["seconds"] = secs
        results[label] = r
        log(label, {k: (round(v, 2) if isinstance(v, float) else v) for k, v in r.items()})
    del srv
    return {"window_ms": w.window_ms, "lanes": lanes, "max_wave": max_wave, "batch_capacity_qps": capacity,
            "loads": results}


def run_serving(args):
    """The serving workload: the full-scale database, Poisson arrivals of real
    queries and every client's negative-binomial fakes, a 10 ms per-cluster
    grouping window, waves on two lanes.  Reports served QPS and p50/p99
    latency at 0.5x and 0.9x of the measured batch capacity and at the
    workload's nominal 50,000 queries/s."""
    import torch
    from paper_2406_06761_gb300 import harness as H
    from paper_2406_06761_gb300 import wally as Wl
    from paper_2406_06761_gb300 import workload as W
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
    max_wave = int(wl.ctx.info.max_wave)
    res = serving_loads(wl, capacity, [("0.5x_capacity", 0.5 * capacity), ("0.9x_capacity", 0.9 * capacity),
                                       ("nominal_50k", w.arrival_qps, min(2.0, args.serving_seconds))],
                        args.serving_seconds, max_wave=max_wave)
    line = {"metric": "serving: served QPS and p50/p99 latency, 3.2M x 192 database, 10 ms window",
            "value": res["loads"]["0.9x_capacity"]["served_qps"], "unit": "queries/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "serving", "window_ms": w.window_ms, "lanes": 2, "max_wave": max_wave,
                       "batch_capacity_qps": capacity},
            "serving": res["loads"]}
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
