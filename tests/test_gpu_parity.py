"""GPU parity: every step of the CUDA path against the CPU oracle, bit for bit
(all arithmetic is integer; the tolerance is zero), through the C ABI.

Inputs are drawn by paper_2406_06761_gb300.workload and fed to both sides;
expected values come only from the oracle or from plain integer dot products.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _ctx(name, max_wave=0):
    w = W.WORKLOADS[name]
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=max_wave)
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    return w, ctx, prm


def _u64(a):
    return Wl.u64_tensor(a, DEV)


def _np(t):
    return Wl.to_u64_numpy(t)


@pytest.fixture(scope="module")
def tiny():
    w, ctx, prm = _ctx("tiny")
    yield w, ctx, prm
    ctx.close()


@pytest.fixture(scope="module")
def batched_ctx():
    w, ctx, prm = _ctx("batched")
    yield w, ctx, prm
    ctx.close()


@pytest.mark.parametrize("name", ["tiny", "batched", "wide"])
def test_parameters_match_oracle(name):
    w, ctx, prm = _ctx(name)
    info = ctx.info
    assert ctx.q == prm.q and ctx.P == prm.P and int(info.t) == prm.t
    assert int(info.zeta_t) == prm.zeta_t
    assert (info.d_pad, info.g, info.h) == (prm.d_pad, prm.g, prm.h)
    assert (int(info.k1), int(info.kg)) == (prm.k1, prm.kg)
    ctx.close()


def _keygen_gpu(ctx, prm, cr, n):
    keys = torch.empty((n, 2, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_keygen(ctx.ptr, n, torch.from_numpy(cr.secret).to(DEV), _u64(cr.key_a),
                    torch.from_numpy(cr.key_e).to(DEV), keys)
    torch.cuda.synchronize()
    return _np(keys)


@pytest.mark.parametrize("which", ["tiny", "batched_ctx"])
def test_keygen_parity(which, request):
    w, ctx, prm = request.getfixturevalue(which)
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=11)
    got = _keygen_gpu(ctx, prm, cr, 2)
    for i in range(2):
        assert np.array_equal(got[i], O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]))


@pytest.mark.parametrize("which", ["tiny", "batched_ctx"])
def test_encrypt_parity_real_and_fake(which, request):
    w, ctx, prm = request.getfixturevalue(which)
    cr = W.client_randomness(3, prm.N, prm.q, prm.P, seed=12)
    qs = W.query_vectors(3, prm.d, 15, seed=12)
    qs[2] = 0  # a fake query encrypts the zero vector
    cts = torch.empty((3, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_encrypt_query(ctx.ptr, 3, torch.from_numpy(cr.secret).to(DEV), torch.from_numpy(qs).to(DEV),
                           _u64(cr.enc_a), torch.from_numpy(cr.enc_e).to(DEV), cts)
    got = _np(cts)
    for i in range(3):
        ref = O.encrypt_query(prm, cr.secret[i], qs[i] if i < 2 else None, cr.enc_a[i], cr.enc_e[i])
        assert np.array_equal(got[i], ref)


def test_decrypt_parity(tiny):
    w, ctx, prm = tiny
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=13)
    v = np.random.default_rng(13).integers(0, prm.t, size=(2, prm.N), dtype=np.uint64)
    cts = np.stack([O.encrypt_slots(prm, cr.secret[i], v[i], cr.enc_a[i], cr.enc_e[i]) for i in range(2)])
    scores = torch.empty((2, prm.N), dtype=torch.int64, device=DEV)
    idx = torch.tensor([1, 0], dtype=torch.int32, device=DEV)
    sec = torch.from_numpy(cr.secret[::-1].copy()).to(DEV)   # ciphertext i uses secret row idx[i]
    Wl.wally_decrypt_scores(ctx.ptr, 2, sec, idx, _u64(cts), scores)
    got = scores.cpu().numpy()
    for i in range(2):
        assert np.array_equal(got[i], O.decrypt_slots(prm, cr.secret[i], cts[i]))


@pytest.mark.parametrize("which", ["tiny", "batched_ctx"])
def test_rotate_parity(which, request):
    """Rot_k = automorphism + hybrid key switch (Sec. 2 CtRotate, Sec. 7)."""
    w, ctx, prm = request.getfixturevalue(which)
    n = 3
    cr = W.client_randomness(n, prm.N, prm.q, prm.P, seed=14)
    v = np.random.default_rng(14).integers(0, prm.t, size=(n, prm.N), dtype=np.uint64)
    cts = np.stack([O.encrypt_slots(prm, cr.secret[i], v[i], cr.enc_a[i], cr.enc_e[i]) for i in range(n)])
    for which_key, k in ((0, prm.k1), (1, prm.kg)):
        keys = np.stack([O.keygen(prm, cr.secret[i], k, cr.key_a[i, which_key], cr.key_e[i, which_key])
                         for i in range(n)])
        out = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
        Wl.wally_rotate(ctx.ptr, n, k, _u64(cts), _u64(keys), out)
        torch.cuda.synchronize()
        got = _np(out)
        for i in range(n):
            assert np.array_equal(got[i], O.rotate(prm, k, keys[i], cts[i])), (which_key, i)


def test_encode_parity_chunks_and_degenerate(tiny):
    """Alg. "Server Initialization": one full cluster, a two-chunk cluster,
    a cluster of a single embedding."""
    w, ctx, prm = tiny
    sizes = np.array([1024, prm.N + 700, 1], np.uint32)
    E = W.embeddings(int(sizes.sum()), prm.d, 15, seed=15)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    row = 0
    for c, s in enumerate(sizes.astype(np.int64)):
        s = int(s)
        m = Wl.wally_cluster_chunks(ctx.ptr, c)
        mo, ref = O.encode_cluster(prm, E[row:row + s])
        assert m == mo
        out = torch.empty((m, prm.h, prm.g, prm.L, prm.N), dtype=torch.int64, device=DEV)
        Wl.wally_export_cluster(ctx.ptr, c, out)
        torch.cuda.synchronize()
        assert np.array_equal(_np(out), ref), c
        row += s


def _clusters_ntt(prm, E, sizes):
    res, row = [], 0
    for s in (int(x) for x in sizes):
        m, pt = O.encode_cluster(prm, E[row:row + s])
        res.append((m, O.ptxt_to_ntt(prm, m, pt)))
        row += s
    return res


def test_eval_tiny_bit_exact_and_decrypts(tiny):
    """The tiny workload: one cluster of 1024, one query, N = 4096."""
    w, ctx, prm = tiny
    sizes = W.cluster_sizes(w)
    E = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound)
    Wl.wally_load_clusters(ctx.ptr, sizes.astype(np.uint32), E)
    q = W.query_vectors(1, w.dim, w.entry_bound)
    cr = W.client_randomness(1, prm.N, prm.q, prm.P)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q[0], cr.enc_a[0], cr.enc_e[0])
    m, pt = O.encode_cluster(prm, E)
    ref = O.eval_query(prm, m, pt, ct, keys)
    out = torch.empty((m, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, 1, torch.zeros(1, dtype=torch.int32, device=DEV), _u64(ct[None]),
                        _u64(keys[None]), None, torch.zeros(1, dtype=torch.int64, device=DEV), out)
    Wl.wally_sync(ctx.ptr)
    got = _np(out)
    assert np.array_equal(got, ref)
    scores = torch.empty((1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_decrypt_scores(ctx.ptr, 1, torch.from_numpy(cr.secret).to(DEV), None, out[0:1], scores)
    assert np.array_equal(scores.cpu().numpy()[0, :len(E)], E.astype(np.int64) @ q[0].astype(np.int64))


def _mixed_case(prm):
    """Three clusters (one embedding, two chunks, 1024 embeddings), seven
    queries over them, a pool of four client submissions."""
    sizes = np.array([1, prm.N + 300, 1024], np.uint32)
    E = W.embeddings(int(sizes.sum()), prm.d, 15, seed=16)
    ids = np.array([2, 1, 0, 1, 2, 2, 1], np.uint32)
    pool = 4
    cr = W.client_randomness(pool, prm.N, prm.q, prm.P, seed=16)
    qs = W.query_vectors(pool, prm.d, 15, seed=16)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(pool)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i] if i < 3 else None, cr.enc_a[i], cr.enc_e[i])
                    for i in range(pool)])
    input_index = np.array([0, 1, 2, 3, 1, 0, 2], np.uint32)
    return sizes, E, ids, cts, keys, input_index, qs, cr


@pytest.mark.parametrize("max_wave", [3, 0])
def test_eval_mixed_clusters_ragged_waves(tiny, max_wave):
    """Uneven clusters, a two-chunk cluster, a pool mapping, and waves of 3
    queries over 7 (ragged last wave), against the oracle's batch driver."""
    w, _, prm = tiny
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=max_wave)
    sizes, E, ids, cts, keys, input_index, qs, cr = _mixed_case(prm)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    chunks = np.array([Wl.wally_cluster_chunks(ctx.ptr, c) for c in range(3)])
    assert list(chunks) == [1, 2, 1]
    # output offsets in reverse query order, to check the scatter
    m = chunks[ids]
    offs = np.zeros(len(ids), np.int64)
    run = 0
    for q in reversed(range(len(ids))):
        offs[q] = run
        run += m[q]
    out = torch.full((run, 2, prm.L, prm.N), -1, dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, len(ids), torch.from_numpy(ids.astype(np.int32)).to(DEV), _u64(cts), _u64(keys),
                        torch.from_numpy(input_index.astype(np.int32)).to(DEV), torch.from_numpy(offs).to(DEV), out)
    Wl.wally_sync(ctx.ptr)
    got = _np(out)
    ref, ref_off = O.eval_batch(prm, _clusters_ntt(prm, E, sizes), ids, cts[input_index], keys[input_index])
    for q in range(len(ids)):
        a, b, k = int(offs[q]), int(ref_off[q]), int(m[q])
        assert np.array_equal(got[a:a + k], ref[b:b + k]), q
    # and the scores decrypt to E q (query 3 uses the fake submission: zeros)
    sz = sizes.astype(np.int64)
    row0 = np.concatenate([[0], np.cumsum(sz)[:-1]]).astype(np.int64)
    for q in range(len(ids)):
        e = int(input_index[q])
        c = int(ids[q])
        Ec = E[int(row0[c]):int(row0[c] + sz[c])].astype(np.int64)
        expect = Ec @ qs[e].astype(np.int64) if e < 3 else np.zeros(len(Ec), np.int64)
        sc = np.concatenate([O.decrypt_slots(prm, cr.secret[e], got[int(offs[q]) + k]) for k in range(int(m[q]))])
        assert np.array_equal(sc[:len(Ec)], expect), q
    ctx.close()


def test_eval_host_buffers_match_device(tiny):
    """wally_eval_batch_host (host in/out, copies inside) = wally_eval_batch."""
    w, _, prm = tiny
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=3)
    sizes, E, ids, cts, keys, input_index, qs, cr = _mixed_case(prm)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    chunks = np.array([Wl.wally_cluster_chunks(ctx.ptr, c) for c in range(3)])
    m = chunks[ids]
    offs = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
    total = int(m.sum())
    out_d = torch.empty((total, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, len(ids), torch.from_numpy(ids.astype(np.int32)).to(DEV), _u64(cts), _u64(keys),
                        torch.from_numpy(input_index.astype(np.int32)).to(DEV), torch.from_numpy(offs).to(DEV), out_d)
    Wl.wally_sync(ctx.ptr)
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    out_h = torch.empty((total, 2, prm.L, prm.N), dtype=torch.int64).pin_memory()
    Wl.wally_eval_batch_host(ctx.ptr, len(ids), h(ids.astype(np.int32)), h(cts.view(np.int64)),
                             h(keys.view(np.int64)), h(input_index.astype(np.int32)), h(offs), out_h)
    assert np.array_equal(out_h.numpy(), out_d.cpu().numpy())
    ctx.close()


def test_eval_bad_cluster_id_reported(tiny):
    w, _, prm = tiny
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    sizes, E, ids, cts, keys, input_index, qs, cr = _mixed_case(prm)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    bad = np.array([2, 7, 0], np.uint32)
    out = torch.zeros((3, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    offs = torch.tensor([0, 1, 2], dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, 3, torch.from_numpy(bad.astype(np.int32)).to(DEV), _u64(cts[:3]), _u64(keys[:3]),
                        None, offs, out)
    with pytest.raises(Wl.WallyError) as ei:
        Wl.wally_sync(ctx.ptr)
    assert ei.value.code == Wl.WALLY_EINVAL
    got = _np(out)
    assert np.all(got[1] == 0)   # the bad query wrote nothing
    ref = O.eval_batch(prm, _clusters_ntt(prm, E, sizes), np.array([2, 0], np.uint32), cts[[0, 2]],
                       keys[[0, 2]])[0]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[1])
    Wl.wally_sync(ctx.ptr)   # the error was cleared
    ctx.close()


def test_eval_empty_batch_and_errors(tiny):
    w, ctx, prm = tiny
    Wl.wally_eval_batch(ctx.ptr, 0, None, None, None, None, None, None)
    with pytest.raises(Wl.WallyError):
        Wl.wally_cluster_chunks(ctx.ptr, 10 ** 6)
    fresh = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    x = torch.zeros(8, dtype=torch.int64, device=DEV)
    with pytest.raises(Wl.WallyError) as ei:
        Wl.wally_eval_batch(fresh.ptr, 1, x, x, x, None, x, x)
    assert ei.value.code == Wl.WALLY_ESTATE
    fresh.close()
    with pytest.raises(Wl.WallyError):
        Wl.wally_setup_params(11, 2, 36, 17, 192)   # unsupported ring size


def test_eval_largest_cluster_and_limit(tiny):
    """The largest cluster BSGS allows (m = g - 1 = 15 chunks at N = 4096,
    ragged last chunk), bit for bit against the oracle and decrypted; a
    cluster of g chunks is rejected (Sec. 5: BSGS while m < sqrt(d))."""
    w, _, prm = tiny
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    size = (prm.g - 2) * prm.N + 1
    E = W.embeddings(size, prm.d, 15, seed=17)
    Wl.wally_load_clusters(ctx.ptr, np.array([size], np.uint32), E)
    assert Wl.wally_cluster_chunks(ctx.ptr, 0) == prm.g - 1
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=17)
    q = W.query_vectors(1, prm.d, 15, seed=17)[0]
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    m = prm.g - 1
    out = torch.empty((m, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, 1, torch.zeros(1, dtype=torch.int32, device=DEV), _u64(ct[None]), _u64(keys[None]),
                        None, torch.zeros(1, dtype=torch.int64, device=DEV), out)
    Wl.wally_sync(ctx.ptr)
    got = _np(out)
    mo, pt = O.encode_cluster(prm, E)
    assert mo == m
    assert np.array_equal(got, O.eval_query(prm, m, pt, ct, keys))
    sc = np.concatenate([O.decrypt_slots(prm, cr.secret[0], got[k]) for k in range(m)])
    assert np.array_equal(sc[:size], E.astype(np.int64) @ q.astype(np.int64)) and np.all(sc[size:] == 0)
    with pytest.raises(Wl.WallyError) as ei:
        Wl.wally_load_clusters(ctx.ptr, np.array([(prm.g - 1) * prm.N + 1], np.uint32),
                               W.embeddings((prm.g - 1) * prm.N + 1, prm.d, 15, seed=18))
    assert ei.value.code == Wl.WALLY_EINVAL
    ctx.close()


@pytest.mark.parametrize("store", [Wl.STORE_NTT, Wl.STORE_COMPACT])
def test_eval_plain_diagonal_split(tiny, store):
    """baby_steps = d_pad (g = 256, h = 1: the plain diagonal method Sec. 5
    uses for clusters of sqrt(d) chunks or more): a 16-chunk cluster, which
    BSGS rejects, and small clusters, bit for bit against the oracle with the
    same split; ragged waves of 3 queries."""
    w, _, _ = tiny
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, baby_steps=256)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, max_wave=3, baby_steps=256, store=store)
    assert (ctx.info.g, ctx.info.h, int(ctx.info.kg)) == (256, 1, prm.kg)
    sizes = np.array([16 * prm.N, 1000, prm.N + 1], np.uint32)
    E = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound, seed=21)
    Wl.wally_load_clusters(ctx.ptr, sizes, E)
    assert [Wl.wally_cluster_chunks(ctx.ptr, c) for c in range(3)] == [16, 1, 2]
    ids = np.array([0, 2, 1, 0], np.uint32)
    cr = W.client_randomness(4, prm.N, prm.q, prm.P, seed=21)
    qs = W.query_vectors(4, w.dim, w.entry_bound, seed=21)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(4)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i] if i < 3 else None, cr.enc_a[i], cr.enc_e[i])
                    for i in range(4)])
    m = np.array([16, 1, 2])[ids]
    offs = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
    out = torch.full((int(m.sum()), 2, prm.L, prm.N), -1, dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, 4, torch.from_numpy(ids.astype(np.int32)).to(DEV), _u64(cts), _u64(keys), None,
                        torch.from_numpy(offs).to(DEV), out)
    Wl.wally_sync(ctx.ptr)
    got = _np(out)
    row0 = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))[:-1]])
    enc = {c: O.encode_cluster(prm, E[int(row0[c]):int(row0[c] + sizes[c])]) for c in (1, 2)}
    for q in (1, 2):  # the small clusters, against the oracle's evaluation
        c = int(ids[q])
        mc, pt = enc[c]
        assert np.array_equal(got[offs[q]:offs[q] + mc], O.eval_query(prm, mc, pt, cts[q], keys[q])), q
    # the 16-chunk cluster: query 0 bit for bit, query 3 (a fake) decrypts to zeros
    m0, pt0 = O.encode_cluster(prm, E[:int(sizes[0])])
    assert np.array_equal(got[0:16], O.eval_query(prm, m0, pt0, cts[0], keys[0]))
    sc = np.concatenate([O.decrypt_slots(prm, cr.secret[3], got[offs[3] + k]) for k in range(16)])
    assert np.all(sc == 0)
    ctx.close()
