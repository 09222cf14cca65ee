"""Response compression (Sec. 7 "Reducing the response size") on the GPU:
the packed bytes equal the oracle's switched-and-dropped values packed by a
plain Python packer, and compressed responses decrypt to the scores."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _bits(q, l):
    return int(((q - 1 + ((1 << (l - 1)) if l else 0)) >> l).bit_length())


def _pack(vals, b):
    out = bytearray()
    for g in range(0, len(vals), 8):
        acc = 0
        for k in range(8):
            acc |= int(vals[g + k]) << (k * b)
        out += acc.to_bytes(b, "little")
    return bytes(out)


@pytest.mark.parametrize("name", ["tiny", "batched", "wide"])
def test_compress_matches_oracle(name):
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    info = ctx.info
    l0, l1 = O.drop_bits(prm.q[-1], prm.t, prm.N)
    assert (info.drop_c0, info.drop_c1) == (l0, l1)
    b0, b1 = _bits(prm.q[-1], l0), _bits(prm.q[-1], l1)
    assert info.compressed_bytes == prm.N // 8 * (b0 + b1)
    rng = np.random.default_rng(61)
    n = 2
    cts = np.stack([np.stack([np.stack([rng.integers(0, q, size=prm.N, dtype=np.uint64) for q in prm.q])
                              for _ in range(2)]) for _ in range(n)])
    out = torch.empty((n, info.compressed_bytes), dtype=torch.uint8, device=DEV)
    Wl.wally_compress_responses(ctx.ptr, n, Wl.u64_tensor(cts, DEV), out)
    got = out.cpu().numpy()
    for i in range(n):
        cc = O.compress(prm, cts[i], l0, l1)
        assert bytes(got[i]) == _pack(cc[0], b0) + _pack(cc[1], b1), i
    ctx.close()


def test_compressed_responses_decrypt_to_scores():
    w = W.WORKLOADS["tiny"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    E = W.embeddings(1024, w.dim, w.entry_bound, seed=62)
    Wl.wally_load_clusters(ctx.ptr, np.array([1024], np.uint32), E)
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=62)
    qs = W.query_vectors(2, w.dim, w.entry_bound, seed=62)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(2)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i], cr.enc_a[i], cr.enc_e[i]) for i in range(2)])
    res = torch.empty((2, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_eval_batch(ctx.ptr, 2, torch.zeros(2, dtype=torch.int32, device=DEV), Wl.u64_tensor(cts, DEV),
                        Wl.u64_tensor(keys, DEV), None, torch.tensor([0, 1], dtype=torch.int64, device=DEV), res)
    packed = torch.empty((2, ctx.info.compressed_bytes), dtype=torch.uint8, device=DEV)
    Wl.wally_compress_responses(ctx.ptr, 2, res, packed)
    scores = torch.empty((2, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_decrypt_compressed(ctx.ptr, 2, torch.from_numpy(cr.secret).to(DEV), None, packed, scores)
    Wl.wally_sync(ctx.ptr)
    sc = scores.cpu().numpy()
    for i in range(2):
        assert np.array_equal(sc[i, :1024], E.astype(np.int64) @ qs[i].astype(np.int64))
        assert np.all(sc[i, 1024:] == 0)
    # 393 KB -> compressed size
    assert ctx.info.compressed_bytes * 5 < 2 * prm.L * prm.N * 8
    ctx.close()
