"""World-size-2 runs of the multi-GPU placement on CPU (gloo): cluster
shards and replicas partition the queries, each rank evaluates its share (here
with the CPU oracle standing in for its GPU), and the union of the ranks'
results equals the single-process evaluation; the step-time reduction takes
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_06761_gb300 import multigpu as M


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    """Three small clusters and seven queries at the tiny ring size."""
    import oracle as O
    from paper_2406_06761_gb300 import workload as W
    prm = O.params(12, 2, 36, 17, 192)
    sizes = np.array([300, 40, 700])
    E = W.embeddings(int(sizes.sum()), prm.d, 15, seed=31)
    ids = np.array([2, 0, 1, 2, 0, 2, 1], np.uint32)
    cr = W.client_randomness(len(ids), prm.N, prm.q, prm.P, seed=31)
    qs = W.query_vectors(len(ids), prm.d, 15, seed=31)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(len(ids))])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i], cr.enc_a[i], cr.enc_e[i]) for i in range(len(ids))])
    row0 = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    clusters = []
    for c in range(len(sizes)):
        m, pt = O.encode_cluster(prm, E[int(row0[c]):int(row0[c] + sizes[c])])
        clusters.append((m, O.ptxt_to_ntt(prm, m, pt)))
    return prm, sizes, ids, cts, keys, clusters


def _worker(rank, world, port, mode, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    prm, sizes, ids, cts, keys, clusters = _case()
    if mode == "shard":
        expected = np.bincount(ids, minlength=len(sizes))
        owner = M.shard_clusters([c[0] for c in clusters], expected, world)
        mine, local_ids = M.route(ids, owner, rank)
        local = [clusters[c] for c in M.local_clusters(owner, rank)]
    else:
        lo, hi = M.split_stream(len(ids), world, rank)
        mine = np.arange(lo, hi)
        local_ids = ids[mine]
        local = clusters
    res = {}
    if len(mine):
        out, offs = O.eval_batch(prm, local, local_ids, cts[mine], keys[mine], nthreads=1)
        for j, q in enumerate(mine):
            m = clusters[ids[q]][0]
            res[int(q)] = out[int(offs[j]):int(offs[j]) + m].tolist()
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    tmax = M.max_over_ranks(float(rank + 1))
    tsum = M.sum_over_ranks(float(rank + 1))
    if rank == 0:
        merged = {}
        for g in gathered:
            assert not (set(g) & set(merged)), "a query was evaluated twice"
            merged.update(g)
        full, offs = O.eval_batch(prm, clusters, ids, cts, keys, nthreads=2)
        ok = sorted(merged) == list(range(len(ids)))
        for q in range(len(ids)):
            m = clusters[ids[q]][0]
            ok = ok and merged[q] == full[int(offs[q]):int(offs[q]) + m].tolist()
        out_q.put((ok, tmax, tsum))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["shard", "replica"])
def test_two_ranks_partition_and_agree(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok, tmax, tsum = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ok
    assert tmax == 2.0 and tsum == 3.0


def test_shard_balance_and_split():
    owner = M.shard_clusters([1] * 10, [100, 1, 1, 1, 1, 1, 1, 1, 1, 1], 2)
    assert set(owner) == {0, 1}
    assert owner[0] != owner[1] or np.sum(owner == owner[0]) == 1
    spans = [M.split_stream(10, 3, r) for r in range(3)]
    assert spans == [(0, 4), (4, 7), (7, 10)]
    mine, local = M.route(np.array([3, 0, 3, 1]), np.array([0, 1, 1, 0]), 1)
    assert list(mine) == [3] and list(local) == [0]   # query 3 names cluster 1, owned by rank 1
    assert M.max_over_ranks(3.5) == 3.5 and M.sum_over_ranks(2.5) == 2.5
