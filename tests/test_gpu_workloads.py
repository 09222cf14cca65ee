"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark uses (device-resident client submissions, waves of max_wave
queries, device-side grouping by cluster): sampled outputs bit for bit
against the oracle, and every output checked by decryption against the
plain integer dot products (a property that holds at any size)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import harness as H
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _oracle_check(wl, prm, qi, got):
    """Recompute query qi with the oracle from the randomness its client drew."""
    e = int(wl.input_index[qi])
    c = int(wl.ids[qi])
    cr = wl.entry_randomness(e)
    keys = O.keygen_pair(prm, cr.secret, cr.key_a, cr.key_e)
    ct = O.encrypt_query(prm, cr.secret, wl.entry_query(e), cr.enc_a, cr.enc_e)
    E = wl.embeddings[wl.row0[c]:wl.row0[c] + wl.sizes[c]]
    m, pt = O.encode_cluster(prm, E)
    ref = O.eval_query(prm, m, pt, ct, keys)
    assert np.array_equal(got, ref), qi


def _decrypt_all(wl, out, offs):
    """GPU-decrypt every output and compare with E q (fakes: zeros)."""
    N = wl.N
    m_of = wl.chunks[wl.ids]
    sec_idx = []
    ct_rows = []
    for qi in range(wl.n):
        for k in range(m_of[qi]):
            sec_idx.append(int(wl.input_index[qi]))
            ct_rows.append(int(offs[qi]) + k)
    # client secrets, regenerated per randomness chunk
    secrets = wl.secrets()
    bad = 0
    step = 512
    for a in range(0, len(ct_rows), step):
        rows = ct_rows[a:a + step]
        scores = torch.empty((len(rows), N), dtype=torch.int64, device=wl.dev)
        Wl.wally_decrypt_scores(wl.ctx.ptr, len(rows), torch.from_numpy(secrets).to(wl.dev),
                                torch.tensor(sec_idx[a:a + step], dtype=torch.int32, device=wl.dev),
                                out[torch.tensor(rows, device=wl.dev)].contiguous(), scores)
        sc = scores.cpu().numpy()
        for j, r in enumerate(rows):
            qi = int(np.searchsorted(offs, r, side="right") - 1)
            k = r - int(offs[qi])
            c = int(wl.ids[qi])
            expect = wl.expected_scores(c, wl.entry_query(int(wl.input_index[qi])))
            seg = expect[k * N:(k + 1) * N]
            if not (np.array_equal(sc[j, :len(seg)], seg) and np.all(sc[j, len(seg):] == 0)):
                bad += 1
    return bad


def test_batched_workload_full_size():
    """64 clusters (log-normal sizes), 1,000 real queries + NB(0.5, 0.9)
    fakes per client, N = 8192, three 50-bit limbs: one call."""
    wl = H.DeviceWorkload("batched", max_wave=512)
    prm = O.params(wl.w.log_n, wl.w.num_q, wl.w.q_bits, wl.w.t_bits, wl.w.dim)
    ids, idx, offs_d, chunks, offs = wl.device_batch(0, wl.n)
    out = wl.alloc_out(chunks)
    wl.eval((ids, idx, offs_d, chunks, offs), out)
    Wl.wally_sync(wl.ctx.ptr)
    assert _decrypt_all(wl, out, offs) == 0
    got = Wl.to_u64_numpy(out)
    # sampled bit-exact checks: a fake, the largest cluster, the first and last
    big = int(np.argmax(wl.sizes))
    picks = {0, wl.n - 1, int(np.flatnonzero(wl.ids == big)[0])}
    if (~wl.is_real).any():
        picks.add(int(np.flatnonzero(~wl.is_real)[0]))
    for qi in sorted(picks):
        m = int(wl.chunks[wl.ids[qi]])
        _oracle_check(wl, prm, qi, got[offs[qi]:offs[qi] + m])
    wl.close()


def test_wide_workload_sampled():
    """Wide embeddings: N = 16384, six 50-bit limbs, d = 768 (g = h = 32),
    entries in [-7, 7]; two clusters, a real and a fake query, bit for bit."""
    w = W.WORKLOADS["wide"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=2)
    sizes = np.array([1000, 37], np.uint32)
    E = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound, seed=51)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=51)
    q = W.query_vectors(1, w.dim, w.entry_bound, seed=51)[0]
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(2)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0]),
                    O.encrypt_query(prm, cr.secret[1], None, cr.enc_a[1], cr.enc_e[1])])
    dev = torch.device("cuda", 0)
    out = torch.empty((2, 2, prm.L, prm.N), dtype=torch.int64, device=dev)
    Wl.wally_eval_batch(ctx.ptr, 2, torch.tensor([0, 1], dtype=torch.int32, device=dev), Wl.u64_tensor(cts, dev),
                        Wl.u64_tensor(keys, dev), None, torch.tensor([0, 1], dtype=torch.int64, device=dev), out)
    Wl.wally_sync(ctx.ptr)
    got = Wl.to_u64_numpy(out)
    m, pt = O.encode_cluster(prm, E[:1000])
    assert np.array_equal(got[0], O.eval_query(prm, m, pt, cts[0], keys[0])[0])
    scores = torch.empty((2, prm.N), dtype=torch.int64, device=dev)
    Wl.wally_decrypt_scores(ctx.ptr, 2, torch.from_numpy(cr.secret).to(dev), None, out, scores)
    sc = scores.cpu().numpy()
    assert np.array_equal(sc[0, :1000], E[:1000].astype(np.int64) @ q.astype(np.int64))
    assert np.all(sc[0, 1000:] == 0) and np.all(sc[1] == 0)
    ctx.close()


def _whole_batch_sampled(wl, prm, n_exact, n_decrypt, seed, ends=True):
    """Evaluate every query of the workload's batch (split into calls whose
    outputs share one buffer); keep sampled outputs, check them by GPU
    decryption against the plain dot products and a few bit for bit against
    the oracle (with ends: also the first and last query and the first fake)."""
    free, _ = torch.cuda.mem_get_info(wl.dev)
    subs = wl.sub_batches(int(free * 0.5))
    rng = np.random.default_rng(seed)
    exact = set(rng.choice(wl.n, size=n_exact, replace=False).tolist())
    if ends:
        exact |= {0, wl.n - 1, int(np.flatnonzero(~wl.is_real)[0])}
    decrypt = set(rng.choice(wl.n, size=n_decrypt, replace=False).tolist())
    keep = {}
    out = None
    for lo, hi in subs:
        b = wl.device_batch(lo, hi)
        if out is None or out.shape[0] < b[3]:
            out = wl.alloc_out(max(b[3], 1))
        wl.eval(b, out[:b[3]])
        Wl.wally_sync(wl.ctx.ptr)
        offs = b[4]
        for qi in (exact | decrypt):
            if lo <= qi < hi:
                m = int(wl.chunks[wl.ids[qi]])
                keep[qi] = out[int(offs[qi - lo]):int(offs[qi - lo]) + m].clone()
    assert len(subs) >= 1 and len(keep) == len(exact | decrypt)
    del out
    secrets = wl.secrets()
    for qi in sorted(decrypt | exact):
        ct = keep[qi]
        e = int(wl.input_index[qi])
        scores = torch.empty((ct.shape[0], wl.N), dtype=torch.int64, device=wl.dev)
        Wl.wally_decrypt_scores(wl.ctx.ptr, ct.shape[0], torch.from_numpy(secrets[e:e + 1]).to(wl.dev),
                                torch.zeros(ct.shape[0], dtype=torch.int32, device=wl.dev), ct.contiguous(), scores)
        sc = scores.cpu().numpy().reshape(-1)
        expect = wl.expected_scores(int(wl.ids[qi]), wl.entry_query(e))
        assert np.array_equal(sc[:len(expect)], expect) and np.all(sc[len(expect):] == 0), qi
    for qi in sorted(exact):
        _oracle_check(wl, prm, qi, Wl.to_u64_numpy(keep[qi]))


def test_full_scale_batch_sampled():
    """The full-scale batch as bench.py runs it: 3.2M x 192 in 1,800 clusters,
    500,000 real queries + fakes, a 2,048-client pool, waves of 1,024, the
    batch split into calls whose outputs share one buffer.  Sampled outputs
    are checked bit for bit against the oracle, and a larger sample by GPU
    decryption against the plain dot products."""
    wl = H.DeviceWorkload("full_scale", pool=2048, max_wave=1024)
    prm = O.params(wl.w.log_n, wl.w.num_q, wl.w.q_bits, wl.w.t_bits, wl.w.dim)
    _whole_batch_sampled(wl, prm, 4, 256, seed=7)
    wl.close()


def test_wide_full_size_sampled():
    """The wide workload at its full size: 1M x 768 (entries in [-7, 7]) in
    1,000 log-normal clusters, N = 16384, six 50-bit limbs, 100,000 real
    queries + fakes.  Its encoded clusters (805 MB a chunk) do not fit in
    device memory, so the store is the compact one (chosen automatically):
    every wave encodes its chunks on the fly.  Pool of 256 clients, waves of
    128 as bench.py --workload wide runs it."""
    wl = H.DeviceWorkload("wide", pool=256, max_wave=128)
    assert wl.ctx.info.store == Wl.STORE_COMPACT
    assert int(wl.sizes.sum()) == 1_000_000 and len(wl.sizes) == 1000
    prm = O.params(wl.w.log_n, wl.w.num_q, wl.w.q_bits, wl.w.t_bits, wl.w.dim)
    _whole_batch_sampled(wl, prm, 1, 64, seed=8, ends=False)
    wl.close()


def test_eval_batch_captured_in_a_cuda_graph():
    """The whole batched evaluation (grouping, waves, every kernel) captured
    once in a CUDA graph and replayed gives the same outputs."""
    wl = H.DeviceWorkload("batched", max_wave=512)
    ids, idx, offs_d, chunks, offs = wl.device_batch(0, wl.n)
    ref = wl.alloc_out(chunks)
    wl.eval((ids, idx, offs_d, chunks, offs), ref)
    Wl.wally_sync(wl.ctx.ptr)
    out = wl.alloc_out(chunks)
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        wl.eval((ids, idx, offs_d, chunks, offs), out)
    torch.cuda.synchronize()
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    Wl.wally_sync(wl.ctx.ptr)
    wl.close()


def test_wave_records_and_profiling_under_graph_replay():
    """wally_profile_waves: one record per wave, queries summing to the batch,
    times increasing within a lane's stream order; launches captured in a CUDA
    graph with profiling on are timed by each replay (same launch count as the
    plain call, positive times)."""
    wl = H.DeviceWorkload("batched", max_wave=256)
    b = wl.device_batch(0, wl.n)
    out = wl.alloc_out(b[3])
    wl.eval(b, out)
    Wl.wally_sync(wl.ctx.ptr)
    Wl.wally_profile_enable(wl.ctx.ptr, True)
    wl.eval(b, out)
    call, q, ms = Wl.wally_profile_waves(wl.ctx.ptr)
    plain = Wl.wally_profile_read(wl.ctx.ptr)
    Wl.wally_profile_enable(wl.ctx.ptr, False)
    assert len(q) == -(-wl.n // 256) and int(q.sum()) == wl.n and set(call.tolist()) == {0}
    assert np.all(ms > 0)
    assert np.all(np.diff(ms[0::2]) > 0) and np.all(np.diff(ms[1::2]) > 0)  # each lane's waves in order
    Wl.wally_profile_enable(wl.ctx.ptr, True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        wl.eval(b, out)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    call2, q2, ms2 = Wl.wally_profile_waves(wl.ctx.ptr)
    graphed = Wl.wally_profile_read(wl.ctx.ptr)
    Wl.wally_profile_enable(wl.ctx.ptr, False)
    del g
    assert {k: v[0] for k, v in graphed.items()} == {k: v[0] for k, v in plain.items()}
    assert all(v[1] > 0 for v in graphed.values())
    assert int(q2.sum()) == wl.n and np.all(ms2 > 0)
    wl.close()


def test_two_cluster_shards_match_a_context_with_every_cluster():
    """Cluster sharding on one GPU as two logical shards: each shard's context
    holds only the clusters it owns and evaluates the queries routed to it
    (local cluster ids) out of two batches of the workload.  The shards
    together take every query exactly once, and each query's outputs equal
    those of a context holding every cluster (global ids, same submission)."""
    from paper_2406_06761_gb300 import multigpu as M
    world = 2
    kw = dict(num_clusters=12, real_queries=150, pool=24, max_wave=64, keep_embeddings=False)
    shards = [H.DeviceWorkload("batched", shard=(world, r), **kw) for r in range(world)]
    full = H.DeviceWorkload("batched", **kw)
    # routing: disjoint owned clusters, every query of both batches once
    owned = np.concatenate([s.global_clusters for s in shards])
    assert sorted(owned.tolist()) == list(range(len(full.sizes)))
    mixes = [W.query_mix(full.w, full.sizes, b) for b in range(world)]
    assert sum(s.n for s in shards) == sum(len(m[0]) for m in mixes)
    for s in shards:
        b = s.device_batch(0, s.n)
        out = s.alloc_out(b[3])
        s.eval(b, out)
        Wl.wally_sync(s.ctx.ptr)
        gids = torch.from_numpy(s.global_clusters[s.ids].astype(np.int32)).to(out.device)
        ref = full.alloc_out(b[3])
        Wl.wally_eval_batch(full.ctx.ptr, s.n, gids, s.pool.cts, s.pool.keys, b[1], b[2], ref)
        Wl.wally_sync(full.ctx.ptr)
        assert torch.equal(out, ref)
        assert np.array_equal(full.chunks[s.global_clusters], s.chunks)
    for s in shards:
        s.close()
    full.close()
