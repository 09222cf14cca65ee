"""Keyword PIR (Sec. 4.2): split cuckoo tables, slot packing, and, on the
GPU, a full keyword lookup through two index PIR answers."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import pir
from paper_2406_06761_gb300 import workload as W


def _entries(n, seed):
    rng = np.random.default_rng(seed)
    kws = set()
    while len(kws) < n:
        kws.add(int(rng.integers(1, 2**63)))
    return {k: bytes(rng.integers(0, 256, int(rng.integers(0, 300)), dtype=np.uint8)) for k in sorted(kws)}


def test_cuckoo_places_every_keyword_at_one_of_its_two_slots():
    ent = _entries(500, 1)
    tab = pir.build(ent)
    assert tab.sizes[0] == tab.sizes[1] == 550  # (1 + u) N' / 2 with u = 1.2
    placed = 0
    for t in (0, 1):
        for s, e in enumerate(tab.slots[t]):
            if e is not None:
                assert pir.slot_of(e[0], t, tab.seed, tab.sizes[t]) == s
                placed += 1
    assert placed == len(ent)
    for k, v in ent.items():
        assert pir.lookup_plain(tab, k) == v
    assert pir.lookup_plain(tab, 12345) is None


def test_dims_follow_the_uneven_split():
    d1, d2 = pir.dims(10000)
    assert d2 == 41 and d1 * d2 >= 10000 and (d1 - 1) * d2 < 10000  # 0.41 sqrt(N')


def test_pack_unpack_roundtrip_and_empty():
    n = 4096
    for val in (b"", b"x", bytes(range(256)) * 3):
        p = pir.pack(77, val, n)
        assert p.max() < 2**16
        assert pir.unpack(p) == (77, val)
    assert pir.unpack(np.zeros(n, np.int64)) is None
    with pytest.raises(ValueError):
        pir.pack(1, b"a" * (2 * n), n)


def test_plaintext_matrix_positions():
    ent = _entries(60, 2)
    tab = pir.build(ent)
    for t in (0, 1):
        mat = tab.plaintexts(t, 64 * 8)
        for k, v in ent.items():
            r, c = tab.position(k, t)
            e = pir.unpack(mat[r, c])
            if e is not None and e[0] == k:
                assert e[1] == v


@pytest.mark.gpu
def test_keyword_lookup_on_the_gpu():
    """200 entries with values of up to 300 bytes in two tables of 220 slots
    (32 x 7 each, 5 expansion levels), N = 4096: five present keywords and
    one absent, each looked up by two index PIR queries answered by the
    GPU, decrypted and unpacked by the client."""
    from paper_2406_06761_gb300 import wally as Wl
    dev = torch.device("cuda", 0)
    w = W.WORKLOADS["tiny"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ent = _entries(200, 3)
    tab = pir.build(ent)
    servers = []
    for t in (0, 1):
        ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
        Wl.wally_pir_load(ctx.ptr, tab.plaintexts(t, prm.N))
        servers.append(ctx)
    lv = max(pir.levels(tab.dims[t][0]) for t in (0, 1))
    keys_list = list(ent)
    wanted = [keys_list[i] for i in (0, 17, 99, 150, 199)] + [424242]
    n = len(wanted)
    cr = W.pir_client_randomness(n, lv, prm.N, prm.q, prm.P, seed=4)
    sec = torch.from_numpy(cr.secret).to(dev)
    ctx0 = servers[0]
    keys = torch.empty((n, lv, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=dev)
    Wl.wally_keygen_galois(ctx0.ptr, n, [O.pir_galois(prm, a) for a in range(lv)], sec,
                           Wl.u64_tensor(cr.key_a, dev), torch.from_numpy(cr.key_e).to(dev), keys)
    found = [None] * n
    for t in (0, 1):
        d1, d2 = tab.dims[t]
        lt = pir.levels(d1)
        pos = [tab.position(k, t) for k in wanted]
        m = np.stack([O.pir_query_plaintext(prm, r, lt) for r, _ in pos])
        cts = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_encrypt_poly(ctx0.ptr, n, sec, Wl.u64_tensor(m, dev), Wl.u64_tensor(cr.enc_a, dev),
                              torch.from_numpy(cr.enc_e).to(dev), cts)
        out = torch.empty((n, d2, 2, prm.L, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_pir_answer(servers[t].ptr, n, cts, keys[:, :lt].contiguous(), out)
        Wl.wally_sync(servers[t].ptr)
        picked = torch.stack([out[i, c] for i, (_, c) in enumerate(pos)]).contiguous()
        coeffs = torch.empty((n, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_decrypt_poly(ctx0.ptr, n, sec, None, picked, coeffs)
        for i, row in enumerate(coeffs.cpu().numpy()):
            e = pir.unpack(row)
            if e is not None and e[0] == wanted[i]:
                found[i] = e[1]
    for i, k in enumerate(wanted):
        assert found[i] == ent.get(k), i
    for ctx in servers:
        ctx.close()


@pytest.mark.gpu
def test_keyword_lookup_two_dimensions_on_the_gpu():
    """The same lookup with MulPIR's two dimensions at N = 8192, three 50-bit
    limbs: 100 entries, tables of 110 slots (22 x 5, 5 expansion levels for
    rows + columns), one answer ciphertext per table and keyword."""
    from paper_2406_06761_gb300 import wally as Wl
    dev = torch.device("cuda", 0)
    w = W.WORKLOADS["batched"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ent = _entries(100, 5)
    tab = pir.build(ent)
    assert tab.dims[0] == (22, 5)
    servers = []
    for t in (0, 1):
        ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
        Wl.wally_pir_load(ctx.ptr, tab.plaintexts(t, prm.N))
        servers.append(ctx)
    d1, d2 = tab.dims[0]
    lv = (d1 + d2 - 1).bit_length()
    keys_list = list(ent)
    wanted = [keys_list[i] for i in (0, 42, 99)] + [777]
    n = len(wanted)
    cr = W.pir_client_randomness(n, lv, prm.N, prm.q, prm.P, seed=6)
    rc = W.client_randomness(n, prm.N, prm.q, prm.P, seed=7)
    sec = torch.from_numpy(cr.secret).to(dev)
    ctx0 = servers[0]
    keys = torch.empty((n, lv, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=dev)
    Wl.wally_keygen_galois(ctx0.ptr, n, [O.pir_galois(prm, a) for a in range(lv)], sec,
                           Wl.u64_tensor(cr.key_a, dev), torch.from_numpy(cr.key_e).to(dev), keys)
    rlk = torch.empty((n, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=dev)
    Wl.wally_keygen_relin(ctx0.ptr, n, sec, Wl.u64_tensor(np.ascontiguousarray(rc.key_a[:, 0]), dev),
                          torch.from_numpy(np.ascontiguousarray(rc.key_e[:, 0])).to(dev), rlk)
    found = [None] * n
    for t in (0, 1):
        m = np.stack([O.pir_query_plaintext2(prm, *tab.position(k, t), d1, lv) for k in wanted])
        cts = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_encrypt_poly(ctx0.ptr, n, sec, Wl.u64_tensor(m, dev), Wl.u64_tensor(cr.enc_a, dev),
                              torch.from_numpy(cr.enc_e).to(dev), cts)
        out = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_pir_answer2(servers[t].ptr, n, cts, keys, rlk, out)
        Wl.wally_sync(servers[t].ptr)
        coeffs = torch.empty((n, prm.N), dtype=torch.int64, device=dev)
        Wl.wally_decrypt_poly(ctx0.ptr, n, sec, None, out, coeffs)
        for i, row in enumerate(coeffs.cpu().numpy()):
            e = pir.unpack(row)
            if e is not None and e[0] == wanted[i]:
                found[i] = e[1]
    for i, k in enumerate(wanted):
        assert found[i] == ent.get(k), i
    for ctx in servers:
        ctx.close()


def test_client_query_helpers_match_the_oracle(tiny_params):
    prm = tiny_params
    assert pir.galois_elements(prm.N, 5) == [O.pir_galois(prm, a) for a in range(5)]
    assert np.array_equal(pir.query_plaintext(prm.N, prm.t, 4, 9), O.pir_query_plaintext(prm, 9, 4))
    assert np.array_equal(pir.query_plaintext(prm.N, prm.t, 5, 3, 2, d1=20), O.pir_query_plaintext2(prm, 3, 2, 20, 5))
