"""The compact cluster store: the embeddings stay resident and every wave
encodes the chunks its queries name right before the multiply-accumulate.
Results must be bit-identical to the resident NTT-form store (and to the
oracle) whatever the wave and cache limits cut: clusters split across waves,
several chunks per cluster, both lanes, one lane, and the host-buffer path."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

# chunks at N = 4096: 2, 1, 3, 1, 1, 2, 1
SIZES = np.array([5000, 300, 9000, 1, 4096, 4097, 77], np.uint32)


def _setup(store, cache_chunks=0, max_wave=8):
    w = W.WORKLOADS["tiny"]
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=max_wave, store=store,
                     cache_chunks=cache_chunks)
    E = W.embeddings(int(SIZES.sum()), w.dim, w.entry_bound, seed=81)
    Wl.wally_load_clusters(ctx.ptr, SIZES, E)
    ctx.refresh()
    return w, ctx, E


@pytest.fixture(scope="module")
def inputs():
    """40 queries over every cluster (ids grouped unevenly), each with its own
    client: keys and ciphertexts made on the device from seeded randomness."""
    w, ctx, E = _setup(Wl.STORE_NTT)
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    n = 40
    rng = np.random.default_rng(82)
    ids = np.concatenate([np.arange(len(SIZES)), rng.integers(0, len(SIZES), n - len(SIZES))]).astype(np.int32)
    rng.shuffle(ids)
    cr = W.client_randomness(n, prm.N, prm.q, prm.P, seed=82)
    qv = W.query_vectors(n, w.dim, w.entry_bound, seed=82)
    keys = torch.empty((n, 2, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    cts = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    sec = torch.from_numpy(cr.secret).to(DEV)
    Wl.wally_keygen(ctx.ptr, n, sec, Wl.u64_tensor(cr.key_a, DEV), torch.from_numpy(cr.key_e).to(DEV), keys)
    Wl.wally_encrypt_query(ctx.ptr, n, sec, torch.from_numpy(qv).to(DEV), Wl.u64_tensor(cr.enc_a, DEV),
                           torch.from_numpy(cr.enc_e).to(DEV), cts)
    m = np.array([Wl.wally_cluster_chunks(ctx.ptr, int(c)) for c in ids], np.int64)
    offs = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
    out = torch.empty((int(m.sum()), 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    args = (torch.from_numpy(ids).to(DEV), cts, keys, torch.from_numpy(offs).to(DEV))
    Wl.wally_eval_batch(ctx.ptr, n, args[0], cts, keys, None, args[3], out)
    Wl.wally_sync(ctx.ptr)
    ref = Wl.to_u64_numpy(out)
    ctx.close()
    return dict(w=w, prm=prm, E=E, ids=ids, m=m, offs=offs, args=args, ref=ref, n=n)


def _eval(ctx, inp, lane=None):
    ids, cts, keys, offs = inp["args"]
    out = torch.zeros((int(inp["m"].sum()), 2, inp["prm"].L, inp["prm"].N), dtype=torch.int64, device=DEV)
    if lane is None:
        Wl.wally_eval_batch(ctx.ptr, inp["n"], ids, cts, keys, None, offs, out)
    else:
        Wl.wally_eval_batch_lane(ctx.ptr, lane, inp["n"], ids, cts, keys, None, offs, out)
    Wl.wally_sync(ctx.ptr)
    return Wl.to_u64_numpy(out)


@pytest.mark.parametrize("cache_chunks,max_wave", [(3, 8), (4, 5), (16, 1024)])
def test_compact_store_equals_ntt_store(inputs, cache_chunks, max_wave):
    _, ctx, _ = _setup(Wl.STORE_COMPACT, cache_chunks=cache_chunks, max_wave=max_wave)
    assert ctx.info.store == Wl.STORE_COMPACT and ctx.info.cache_chunks == cache_chunks
    assert ctx.info.cluster_bytes == int(SIZES.sum()) * inputs["w"].dim
    assert np.array_equal(_eval(ctx, inputs), inputs["ref"])
    assert np.array_equal(_eval(ctx, inputs, lane=2), inputs["ref"])
    ctx.close()


def test_compact_store_host_path(inputs):
    _, ctx, _ = _setup(Wl.STORE_COMPACT, cache_chunks=3, max_wave=8)
    ids, cts, keys, offs = inputs["args"]
    out = torch.zeros((int(inputs["m"].sum()), 2, inputs["prm"].L, inputs["prm"].N), dtype=torch.int64).pin_memory()
    Wl.wally_eval_batch_host(ctx.ptr, inputs["n"], ids.cpu().to(torch.int32), cts.cpu().pin_memory(),
                             keys.cpu().pin_memory(), None, offs.cpu(), out)
    assert np.array_equal(out.numpy().view(np.uint64), inputs["ref"])
    ctx.close()


def test_compact_store_against_oracle(inputs):
    """Two outputs (a three-chunk cluster and a one-chunk cluster) of the
    compact store, bit for bit against the oracle's evaluation."""
    _, ctx, _ = _setup(Wl.STORE_COMPACT, cache_chunks=3, max_wave=8)
    got = _eval(ctx, inputs)
    prm, E, ids = inputs["prm"], inputs["E"], inputs["ids"]
    row0 = np.concatenate([[0], np.cumsum(SIZES.astype(np.int64))[:-1]])
    keys = Wl.to_u64_numpy(inputs["args"][2])
    cts = Wl.to_u64_numpy(inputs["args"][1])
    for c in (2, 1):
        q = int(np.flatnonzero(ids == c)[0])
        r0, r1 = int(row0[c]), int(row0[c]) + int(SIZES[c])
        m, pt = O.encode_cluster(prm, E[r0:r1])
        want = O.eval_query(prm, m, pt, cts[q], keys[q])
        o = int(inputs["offs"][q])
        assert np.array_equal(got[o:o + m], np.asarray(want)), (c, q)
    ctx.close()


def test_compact_export_equals_ntt_export():
    _, a, _ = _setup(Wl.STORE_NTT)
    _, b, _ = _setup(Wl.STORE_COMPACT, cache_chunks=3)
    for c in (2, 6):
        m = Wl.wally_cluster_chunks(a.ptr, c)
        shape = (m, a.info.h, a.info.g, a.info.num_q, a.info.n)
        x = torch.empty(shape, dtype=torch.int64, device=DEV)
        y = torch.zeros(shape, dtype=torch.int64, device=DEV)
        Wl.wally_export_cluster(a.ptr, c, x)
        Wl.wally_export_cluster(b.ptr, c, y)
        torch.cuda.synchronize()
        assert torch.equal(x, y), c
    a.close()
    b.close()


def test_compact_cache_smaller_than_a_cluster_is_rejected():
    w = W.WORKLOADS["tiny"]
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, store=Wl.STORE_COMPACT, cache_chunks=2)
    E = W.embeddings(int(SIZES.sum()), w.dim, w.entry_bound, seed=81)
    with pytest.raises(Wl.WallyError) as e:
        Wl.wally_load_clusters(ctx.ptr, SIZES, E)
    assert e.value.code == Wl.WALLY_EINVAL
    ctx.close()
