"""Serving loop (continuous batching over lanes): every request's result is
identical, bit for bit, whether it runs alone or mixed into a loaded stream
whose waves overlap on two lanes, and equals the oracle's evaluation."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import serving as S
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def setup():
    prm = O.params(12, 2, 36, 17, 192)
    ctx = Wl.Context(12, 2, 36, 17, 192, max_wave=8)
    sizes = np.array([500, prm.N + 100, 64], np.uint32)
    E = W.embeddings(int(sizes.sum()), prm.d, 15, seed=41)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    chunks = np.array([Wl.wally_cluster_chunks(ctx.ptr, c) for c in range(3)])
    pool = 6
    cr = W.client_randomness(pool, prm.N, prm.q, prm.P, seed=41)
    qs = W.query_vectors(pool, prm.d, 15, seed=41)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(pool)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i] if i < pool - 1 else None, cr.enc_a[i],
                                    cr.enc_e[i]) for i in range(pool)])
    row0 = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))[:-1]])
    encoded = {}
    for c in range(3):
        m, pt = O.encode_cluster(prm, E[int(row0[c]):int(row0[c] + sizes[c])])
        encoded[c] = (m, pt)
    yield prm, ctx, chunks, Wl.u64_tensor(cts, DEV), Wl.u64_tensor(keys, DEV), cts, keys, encoded
    ctx.close()


def _stream(arrival, cluster, entry):
    n = len(arrival)
    return S.Stream(np.asarray(arrival, float), np.asarray(cluster, np.uint32), np.asarray(entry, np.uint32),
                    np.ones(n, bool))


def test_same_alone_and_in_the_mix(setup):
    prm, ctx, chunks, cts_d, keys_d, cts, keys, encoded = setup
    alone = S.Server(ctx.ptr, chunks, cts_d, keys_d, lanes=1, window_ms=1.0, max_wave=8, keep_outputs=True)
    alone.run(_stream([0.0], [1], [2]))
    ref_alone = alone.outputs[0]
    # a loaded stream: 48 requests within 2 ms, waves of 8 on two lanes
    rng = np.random.default_rng(5)
    n = 48
    cl = rng.integers(0, 3, size=n)
    en = rng.integers(0, 6, size=n)
    cl[[3, 20, 41]] = 1
    en[[3, 20, 41]] = 2
    mixed = S.Server(ctx.ptr, chunks, cts_d, keys_d, lanes=2, window_ms=0.5, max_wave=8, keep_outputs=True)
    res = mixed.run(_stream(np.linspace(0, 0.002, n), cl, en))
    assert res["requests"] == n and res["waves"] >= 6
    for r in (3, 20, 41):
        assert np.array_equal(mixed.outputs[r], ref_alone), r
    # and every mixed result equals the oracle for its (cluster, submission)
    cache = {}
    for r in range(n):
        key = (int(cl[r]), int(en[r]))
        if key not in cache:
            m, pt = encoded[key[0]]
            cache[key] = O.eval_query(prm, m, pt, cts[key[1]], keys[key[1]])
        assert np.array_equal(mixed.outputs[r], cache[key]), r


@pytest.fixture(scope="module")
def setup_batched():
    """The batched workload's parameters (N = 8192, three 50-bit limbs,
    t of 20 bits): eight clusters, one of two chunks, eight submissions of
    which the last is a fake."""
    prm = O.params(13, 3, 50, 20, 192)
    ctx = Wl.Context(13, 3, 50, 20, 192, max_wave=32)
    sizes = np.array([prm.N + 300, 900, 3000, 64, 5000, 1, 7000, 2500], np.uint32)
    E = W.embeddings(int(sizes.sum()), prm.d, 15, seed=43)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    chunks = np.array([Wl.wally_cluster_chunks(ctx.ptr, c) for c in range(len(sizes))])
    pool = 8
    cr = W.client_randomness(pool, prm.N, prm.q, prm.P, seed=43)
    qs = W.query_vectors(pool, prm.d, 15, seed=43)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(pool)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i] if i < pool - 1 else None, cr.enc_a[i],
                                    cr.enc_e[i]) for i in range(pool)])
    row0 = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))[:-1]])
    yield prm, ctx, chunks, Wl.u64_tensor(cts, DEV), Wl.u64_tensor(keys, DEV), cts, keys, E, sizes, row0
    ctx.close()


def test_mixed_stream_at_batched_parameters(setup_batched):
    """200 requests over eight clusters within 5 ms, waves of up to 32 on
    two lanes: requests also run alone are bit-identical in the mix, every
    repeat of a (cluster, submission) pair gives the same bits, and a sample
    of pairs (the two-chunk cluster and the fake among them) equals the
    oracle's evaluation."""
    prm, ctx, chunks, cts_d, keys_d, cts, keys, E, sizes, row0 = setup_batched
    assert chunks[0] == 2
    alone_pairs = [(0, 2), (5, 7), (3, 4)]
    alone = {}
    for c, e in alone_pairs:
        srv = S.Server(ctx.ptr, chunks, cts_d, keys_d, lanes=1, window_ms=1.0, max_wave=32, keep_outputs=True)
        srv.run(_stream([0.0], [c], [e]))
        alone[(c, e)] = srv.outputs[0]
    rng = np.random.default_rng(11)
    n = 200
    cl = rng.integers(0, len(sizes), size=n)
    en = rng.integers(0, 8, size=n)
    planted = {5: (0, 2), 77: (5, 7), 150: (3, 4), 151: (0, 2)}
    for r, (c, e) in planted.items():
        cl[r], en[r] = c, e
    mixed = S.Server(ctx.ptr, chunks, cts_d, keys_d, lanes=2, window_ms=1.0, max_wave=32, keep_outputs=True)
    res = mixed.run(_stream(np.linspace(0, 0.005, n), cl, en))
    assert res["requests"] == n and res["waves"] >= 7
    for r, pair in planted.items():
        assert np.array_equal(mixed.outputs[r], alone[pair]), r
    first = {}
    for r in range(n):
        key = (int(cl[r]), int(en[r]))
        if key in first:
            assert np.array_equal(mixed.outputs[r], mixed.outputs[first[key]]), (r, key)
        else:
            first[key] = r
    sample = [(0, 2), (5, 7), (3, 4)] + [k for k in first if k[0] not in (0, 3, 5)][:3]
    for c, e in sample:
        m, pt = O.encode_cluster(prm, E[int(row0[c]):int(row0[c] + sizes[c])])
        want = O.eval_query(prm, m, pt, cts[e], keys[e])
        assert np.array_equal(mixed.outputs[first[(c, e)]], want), (c, e)
