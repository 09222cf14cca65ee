"""Device-resident workloads for the benchmark and the GPU tests.

Builds one of the workload shapes of ``workload.WORKLOADS`` on the GPU through
the library's own C ABI: parameters, the encoded cluster store, a pool of
client submissions (fresh Galois keys and an encrypted query per client,
generated on the device from host-drawn randomness), and the batch of
(cluster id, submission) pairs with real and negative-binomial fake queries.

A batch whose outputs do not fit in device memory next to the database is
evaluated as several consecutive calls ("sub-batches") into one reused output
buffer; every query of the batch is still evaluated and written out.
"""
from __future__ import annotations

import dataclasses
import sys

import numpy as np
import torch

from . import wally as Wl
from . import workload as W


@dataclasses.dataclass
class Pool:
    """Client submissions resident on the device."""
    cts: torch.Tensor        # int64 [P][2][L][N]
    keys: torch.Tensor       # int64 [P][2][L][2][L+1][N]
    chunk: int               # clients per randomness chunk
    is_fake: np.ndarray      # bool [P]


class DeviceWorkload:
    """shard = (world, rank): load only the clusters this rank owns (cluster
    shards balanced by chunks x expected queries, multigpu.shard_clusters) and
    take, out of `world` batches of the workload (seeds seed .. seed+world-1),
    the queries that name them, with local cluster ids; every rank then
    evaluates about one batch (weak scaling) and no query is evaluated
    twice."""

    def __init__(self, name: str, seed: int = 0, device: int = 0, pool: int | None = None, max_wave: int = 0,
                 real_queries: int | None = None, num_clusters: int | None = None, sizes=None,
                 keep_embeddings: bool = True, verbose: bool = False, shard: tuple[int, int] | None = None,
                 **ctx_kw):
        from . import multigpu as M
        w = W.WORKLOADS[name]
        if real_queries is not None or num_clusters is not None:
            w = dataclasses.replace(w, real_queries=real_queries if real_queries is not None else w.real_queries,
                                    num_clusters=num_clusters if num_clusters is not None else w.num_clusters)
        self.w, self.seed, self.verbose = w, seed, verbose
        self.dev = torch.device("cuda", device)
        self.ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, device=device, max_wave=max_wave, **ctx_kw)
        info = self.ctx.info
        self.N, self.L, self.q, self.P = info.n, info.num_q, self.ctx.q, self.ctx.P
        self.ctw, self.keysw = int(info.ct_words), int(info.keys_words)
        sizes_all = np.asarray(sizes if sizes is not None else W.cluster_sizes(w, seed), dtype=np.int64)
        emb_all = W.embeddings(int(sizes_all.sum()), w.dim, w.entry_bound, seed)
        self.shard = shard
        if shard is None:
            self.sizes, emb = sizes_all, emb_all
            self.ids, self.is_real = W.query_mix(w, self.sizes, seed)
            self.global_clusters = np.arange(len(sizes_all))
        else:
            world, rank = shard
            mixes = [W.query_mix(w, sizes_all, seed + b) for b in range(world)]
            ids_all = np.concatenate([m[0] for m in mixes])
            real_all = np.concatenate([m[1] for m in mixes])
            chunks_all = np.maximum(1, -(-sizes_all // self.N))
            owner = M.shard_clusters(chunks_all, np.bincount(ids_all, minlength=len(sizes_all)), world)
            self.global_clusters = M.local_clusters(owner, rank)
            mine, local_ids = M.route(ids_all, owner, rank)
            self.ids, self.is_real = local_ids, real_all[mine]
            self.sizes = sizes_all[self.global_clusters]
            row0_all = np.concatenate([[0], np.cumsum(sizes_all)[:-1]])
            emb = np.concatenate([emb_all[row0_all[c]:row0_all[c] + sizes_all[c]] for c in self.global_clusters])
        total = int(self.sizes.sum())
        self._log(f"load {len(self.sizes)} clusters, {total} embeddings")
        Wl.wally_load_clusters(self.ctx.ptr, self.sizes.astype(np.uint32), emb)
        self.ctx.refresh()
        self.embeddings = emb if keep_embeddings else None
        self.row0 = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.chunks = np.array([Wl.wally_cluster_chunks(self.ctx.ptr, c) for c in range(len(self.sizes))], np.int64)
        self.n = len(self.ids)
        self.pool_size = int(pool) if pool else self.n
        self._build_pool()
        self._assign()

    def _log(self, msg):
        if self.verbose:
            print(f"[workload] {msg}", file=sys.stderr, flush=True)

    # -------------------------------------------------------------- pool
    def entry_randomness(self, e: int) -> W.ClientRandomness:
        """The randomness client e drew (regenerated from its chunk)."""
        c = self.pool.chunk
        k, r = divmod(e, c)
        n = min(c, self.pool_size - k * c)
        cr = W.client_randomness(n, self.N, self.q, self.P, self.seed, index=k)
        return W.ClientRandomness(cr.secret[r], cr.key_a[r], cr.key_e[r], cr.enc_a[r], cr.enc_e[r])

    def secrets(self) -> np.ndarray:
        """Secret keys of every client of the pool, int8 [P][N]."""
        c = self.pool.chunk
        parts = []
        for k in range(0, self.pool_size, c):
            n = min(c, self.pool_size - k)
            parts.append(W.ternary(n, self.N, self.seed, f"clients{k // c}/s"))
        return np.concatenate(parts)

    def entry_query(self, e: int) -> np.ndarray | None:
        """Query vector of entry e (None for a fake)."""
        if self.pool.is_fake[e]:
            return None
        return W.query_vectors(1, self.w.dim, self.w.entry_bound, self.seed, index=1 + e)[0]

    def _build_pool(self):
        P = self.pool_size
        if P == self.n:
            is_fake = ~self.is_real
        else:
            # fakes get their own entries, in proportion, at least one if any
            n_fake_q = int((~self.is_real).sum())
            n_fake = 0 if n_fake_q == 0 else max(1, round(P * n_fake_q / self.n))
            if n_fake >= P and P > 1:
                n_fake = P - 1
            is_fake = np.zeros(P, bool)
            is_fake[P - n_fake:] = True
        chunk = 256
        cts = torch.empty((P, 2, self.L, self.N), dtype=torch.int64, device=self.dev)
        keys = torch.empty((P, 2, self.L, 2, self.L + 1, self.N), dtype=torch.int64, device=self.dev)
        self.pool = Pool(cts, keys, chunk, is_fake)
        for k0 in range(0, P, chunk):
            n = min(chunk, P - k0)
            cr = W.client_randomness(n, self.N, self.q, self.P, self.seed, index=k0 // chunk)
            qv = np.zeros((n, self.w.dim), np.int8)
            for r in range(n):
                v = self.entry_query(k0 + r)
                if v is not None:
                    qv[r] = v
            d = self.dev
            sec = torch.from_numpy(cr.secret).to(d)
            Wl.wally_keygen(self.ctx.ptr, n, sec, Wl.u64_tensor(cr.key_a, d), torch.from_numpy(cr.key_e).to(d),
                            keys[k0:k0 + n])
            Wl.wally_encrypt_query(self.ctx.ptr, n, sec, torch.from_numpy(qv).to(d), Wl.u64_tensor(cr.enc_a, d),
                                   torch.from_numpy(cr.enc_e).to(d), cts[k0:k0 + n])
            self._log(f"pool {k0 + n}/{P}")
        torch.cuda.synchronize(self.dev)

    def _assign(self):
        """Query i uses entry input_index[i]: real queries cycle over the real
        entries, fakes over the fake entries (identity when the pool holds one
        entry per query)."""
        P = self.pool_size
        if P == self.n:
            idx = np.arange(self.n, dtype=np.int64)
        else:
            real_entries = np.flatnonzero(~self.pool.is_fake)
            fake_entries = np.flatnonzero(self.pool.is_fake)
            idx = np.empty(self.n, np.int64)
            r = np.flatnonzero(self.is_real)
            f = np.flatnonzero(~self.is_real)
            idx[r] = real_entries[np.arange(len(r)) % len(real_entries)]
            if len(f):
                idx[f] = fake_entries[np.arange(len(f)) % len(fake_entries)]
        self.input_index = idx.astype(np.uint32)

    # -------------------------------------------------------------- batches
    def sub_batches(self, max_out_bytes: int | None = None) -> list[tuple[int, int]]:
        """Split the batch so that one sub-batch's outputs fit in max_out_bytes."""
        m = self.chunks[self.ids]
        if max_out_bytes is None:
            return [(0, self.n)]
        cap = max(1, max_out_bytes // (8 * self.ctw))
        out, start, acc = [], 0, 0
        for i, mi in enumerate(m):
            if acc + mi > cap and i > start:
                out.append((start, i))
                start, acc = i, 0
            acc += int(mi)
        out.append((start, self.n))
        return out

    def device_batch(self, lo: int, hi: int):
        """Device arrays of queries [lo, hi): ids, input_index, out_offsets, chunk total."""
        ids = self.ids[lo:hi]
        m = self.chunks[ids]
        offs = np.zeros(hi - lo, np.int64)
        if hi > lo:
            offs[1:] = np.cumsum(m)[:-1]
        return (torch.from_numpy(ids.astype(np.int32)).to(self.dev),
                torch.from_numpy(self.input_index[lo:hi].astype(np.int32)).to(self.dev),
                torch.from_numpy(offs).to(self.dev), int(m.sum()), offs)

    def alloc_out(self, chunks: int) -> torch.Tensor:
        return torch.empty((chunks, 2, self.L, self.N), dtype=torch.int64, device=self.dev)

    def eval(self, batch, out, stream=None):
        ids, idx, offs, _, _ = batch
        Wl.wally_eval_batch(self.ctx.ptr, ids.numel(), ids, self.pool.cts, self.pool.keys, idx, offs, out, stream)

    def expected_scores(self, cluster: int, qv: np.ndarray | None) -> np.ndarray:
        """Plain integer dot products of a query with every embedding of a cluster."""
        E = self.embeddings[self.row0[cluster]:self.row0[cluster] + self.sizes[cluster]].astype(np.int64)
        if qv is None:
            return np.zeros(len(E), np.int64)
        return E @ qv.astype(np.int64)

    def close(self):
        self.ctx.close()
