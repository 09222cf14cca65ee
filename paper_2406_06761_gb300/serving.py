"""Serving loop: continuous batching of a stream of cluster queries.

Requests (cluster id, client submission) arrive over time, as from the
anonymisation network of Sec. 3 (each client's real and fake queries at
independent times).  The encoded clusters and the client submissions stay
resident on the device; requests are evaluated in waves on the independent
lanes (workspaces) of one context:

- a request waits in the pending queue at most one grouping window
  (10 ms by default) before it is admitted;
- a wave is admitted when a lane is free and either the oldest pending
  request has waited a full window or a full wave is pending (the wave size
  is what one lane's device memory holds: admission by device memory);
- waves on different lanes overlap on the device, one CUDA stream per lane,
  so requests that arrive while others are running are admitted as soon as a
  lane frees up;
- a CUDA event per wave marks its completion; a request's latency is its
  wave's completion time minus its arrival time.

Every kernel runs in libwally; this module only schedules host-side calls.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import wally as Wl


@dataclasses.dataclass
class Stream:
    """A request stream: arrival time (s), cluster id, submission index, and
    (optionally) the client each request came from."""
    arrival: np.ndarray
    cluster: np.ndarray
    entry: np.ndarray
    is_real: np.ndarray
    client: np.ndarray | None = None


def poisson_stream(rate_qps: float, seconds: float, sizes, n_entries: int, nb_r: float = 0.5, nb_p: float = 0.9,
                   seed: int = 0) -> Stream:
    """The anonymised request stream over `seconds` at an offered rate of
    `rate_qps` real and fake queries together.  Clients follow Alg. "Client
    Query Generation": each sends one real query, on a cluster drawn in
    proportion to cluster size, and NB(nb_r, nb_p) fake queries (numpy's
    convention, the per-client count of the workload generator) on uniform
    clusters; every query is sent at its own uniform time (Alg. "Schedule"
    gives each query an independent random slot), so the arrivals form a
    Poisson process.  The number of clients is Poisson with mean
    rate * seconds / (1 + E[fakes]).  Submissions cycle over the pool: real
    queries over its first entries, fakes over the last ones (in proportion
    to the expected fake share, at least one)."""
    from . import workload as W
    rng = np.random.default_rng([seed, 0x5e4])
    mean_fakes = nb_r * (1.0 - nb_p) / nb_p if nb_r > 0 else 0.0
    n_clients = max(1, int(rng.poisson(rate_qps * seconds / (1.0 + mean_fakes))))
    fakes = W.fake_counts(n_clients, nb_r, nb_p, seed=seed + 0x5e4)
    client = np.concatenate([np.arange(n_clients), np.repeat(np.arange(n_clients), fakes)])
    is_real = np.concatenate([np.ones(n_clients, bool), np.zeros(int(fakes.sum()), bool)])
    n = len(client)
    p = np.asarray(sizes, dtype=np.float64)
    cluster = np.where(is_real, rng.choice(len(p), size=n, p=p / p.sum()), rng.integers(0, len(p), size=n))
    arrival = rng.uniform(0.0, seconds, size=n)
    order = np.argsort(arrival, kind="stable")
    arrival, client, is_real, cluster = arrival[order], client[order], is_real[order], cluster[order]
    share = mean_fakes / (1.0 + mean_fakes)
    n_fake_entries = max(1, int(round(n_entries * share))) if share > 0 else 0
    n_fake_entries = min(n_fake_entries, max(0, n_entries - 1))
    n_real_entries = n_entries - n_fake_entries
    k = np.arange(n)
    entry = np.where(is_real, k % max(1, n_real_entries), n_real_entries + k % max(1, n_fake_entries))
    return Stream(arrival, cluster.astype(np.uint32), entry.astype(np.uint32), is_real, client.astype(np.int64))


class _Lane:
    def __init__(self, idx, dev, max_wave, max_chunks, L, N):
        self.idx = idx
        self.stream = torch.cuda.Stream(device=dev)
        self.event = torch.cuda.Event()
        self.ids_h = torch.empty(max_wave, dtype=torch.int32).pin_memory()
        self.idx_h = torch.empty(max_wave, dtype=torch.int32).pin_memory()
        self.off_h = torch.empty(max_wave, dtype=torch.int64).pin_memory()
        self.ids_d = torch.empty(max_wave, dtype=torch.int32, device=dev)
        self.idx_d = torch.empty(max_wave, dtype=torch.int32, device=dev)
        self.off_d = torch.empty(max_wave, dtype=torch.int64, device=dev)
        self.out = torch.empty((max_chunks, 2, L, N), dtype=torch.int64, device=dev)
        self.requests = None
        self.offsets = None


class Server:
    """Continuous-batching server over one context's lanes."""

    def __init__(self, ctx_ptr: int, chunks: np.ndarray, cts: torch.Tensor, keys: torch.Tensor, lanes: int = 2,
                 window_ms: float = 10.0, max_wave: int = 1024, keep_outputs: bool = False):
        if lanes < 1 or lanes > 4:
            raise ValueError("1 to 4 lanes")
        self.ctx = ctx_ptr
        self.chunks = np.asarray(chunks, dtype=np.int64)
        self.cts, self.keys = cts, keys
        self.window = window_ms / 1e3
        self.max_wave = max_wave
        self.keep_outputs = keep_outputs
        dev = cts.device
        L, N = cts.shape[2], cts.shape[3]
        max_chunks = max_wave * int(self.chunks.max())
        self.lanes = [_Lane(i, dev, max_wave, max_chunks, L, N) for i in range(lanes)]
        self.outputs: dict[int, np.ndarray] = {}

    def _launch(self, lane: _Lane, reqs: list[int], s: Stream):
        n = len(reqs)
        ids = s.cluster[reqs]
        m = self.chunks[ids]
        offs = np.zeros(n, np.int64)
        offs[1:] = np.cumsum(m)[:-1]
        lane.ids_h[:n] = torch.from_numpy(ids.astype(np.int32))
        lane.idx_h[:n] = torch.from_numpy(s.entry[reqs].astype(np.int32))
        lane.off_h[:n] = torch.from_numpy(offs)
        with torch.cuda.stream(lane.stream):
            lane.ids_d[:n].copy_(lane.ids_h[:n], non_blocking=True)
            lane.idx_d[:n].copy_(lane.idx_h[:n], non_blocking=True)
            lane.off_d[:n].copy_(lane.off_h[:n], non_blocking=True)
            Wl.wally_eval_batch_lane(self.ctx, lane.idx, n, lane.ids_d[:n], self.cts, self.keys, lane.idx_d[:n],
                                     lane.off_d[:n], lane.out, lane.stream)
            lane.event.record(lane.stream)
        lane.requests = reqs
        lane.offsets = (offs, m)

    def run(self, s: Stream, poll_sleep_s: float = 50e-6) -> dict:
        """Serve the whole stream; returns latency and throughput figures."""
        n = len(s.arrival)
        done_at = np.full(n, np.nan)
        pending = collections.deque()
        nxt = 0
        waves = 0
        wave_sizes = []
        t0 = time.perf_counter()
        finished = 0
        while finished < n:
            now = time.perf_counter() - t0
            while nxt < n and s.arrival[nxt] <= now:
                pending.append(nxt)
                nxt += 1
            progressed = False
            for lane in self.lanes:
                if lane.requests is not None and lane.event.query():
                    t_done = time.perf_counter() - t0
                    done_at[lane.requests] = t_done
                    finished += len(lane.requests)
                    if self.keep_outputs:
                        out = Wl.to_u64_numpy(lane.out)
                        offs, m = lane.offsets
                        for r, o, k in zip(lane.requests, offs, m):
                            self.outputs[int(r)] = out[int(o):int(o + k)].copy()
                    lane.requests = None
                    progressed = True
            for lane in self.lanes:
                if lane.requests is None and pending:
                    oldest = s.arrival[pending[0]]
                    if len(pending) >= self.max_wave or now - oldest >= self.window or nxt == n:
                        take = [pending.popleft() for _ in range(min(self.max_wave, len(pending)))]
                        self._launch(lane, take, s)
                        waves += 1
                        wave_sizes.append(len(take))
                        progressed = True
            if not progressed:
                if nxt < n and not pending:
                    wait = s.arrival[nxt] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(poll_sleep_s)
        Wl.wally_sync(self.ctx)
        lat = (done_at - s.arrival) * 1e3
        span = float(np.nanmax(done_at))
        return {
            "requests": n, "real_requests": int(s.is_real.sum()), "waves": waves,
            "mean_wave": float(np.mean(wave_sizes)) if wave_sizes else 0.0,
            "offered_qps": n / float(s.arrival[-1] - s.arrival[0] + 1e-9) if n > 1 else 0.0,
            "served_qps": n / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(np.max(lat)),
        }
