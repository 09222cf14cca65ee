"""Index PIR (the server side of Sec. 4.2's keyword PIR) on the GPU against
the oracle, bit for bit: Galois keys for the expansion elements,
relinearisation keys, encryption and decryption of coefficient plaintexts,
the one-dimensional answer (oblivious expansion + MulPIR's first dimension)
and the two-dimensional one (+ the second dimension by ciphertext
products)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _setup(name):
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    return prm, ctx


def _client(ctx, prm, n, levels, rows_wanted, seed):
    """Keys and queries made on the device from seeded randomness."""
    cr = W.pir_client_randomness(n, levels, prm.N, prm.q, prm.P, seed=seed)
    sec = torch.from_numpy(cr.secret).to(DEV)
    keys = torch.empty((n, levels, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    if levels:
        Wl.wally_keygen_galois(ctx.ptr, n, [O.pir_galois(prm, a) for a in range(levels)], sec,
                               Wl.u64_tensor(cr.key_a, DEV), torch.from_numpy(cr.key_e).to(DEV), keys)
    m = np.stack([O.pir_query_plaintext(prm, r, levels) for r in rows_wanted])
    cts = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_encrypt_poly(ctx.ptr, n, sec, Wl.u64_tensor(m, DEV), Wl.u64_tensor(cr.enc_a, DEV),
                          torch.from_numpy(cr.enc_e).to(DEV), cts)
    return cr, sec, keys, cts, m


def test_keygen_encrypt_decrypt_poly_parity():
    prm, ctx = _setup("tiny")
    levels = 3
    cr, sec, keys, cts, m = _client(ctx, prm, 2, levels, [5, 0], seed=51)
    kg = Wl.to_u64_numpy(keys)
    ct = Wl.to_u64_numpy(cts)
    for i in range(2):
        for a in range(levels):
            ref = O.keygen(prm, cr.secret[i], O.pir_galois(prm, a), cr.key_a[i, a], cr.key_e[i, a])
            assert np.array_equal(kg[i, a], ref), (i, a)
        assert np.array_equal(ct[i], O.encrypt(prm, cr.secret[i], m[i], cr.enc_a[i], cr.enc_e[i])), i
    coeffs = torch.empty((2, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_decrypt_poly(ctx.ptr, 2, sec, None, cts, coeffs)
    got = coeffs.cpu().numpy()
    for i in range(2):
        assert np.array_equal(got[i], np.asarray(O.decrypt_poly(prm, cr.secret[i], ct[i])[0], np.int64))
        assert np.array_equal(got[i], m[i].astype(np.int64))
    ctx.close()


@pytest.mark.parametrize("rows,cols,wanted", [(6, 3, [4, 0, 5]), (1, 2, [0]), (8, 1, [7, 3])])
def test_pir_answer_matches_oracle(rows, cols, wanted):
    """Tables of 6 x 3 (8 indicators for 6 rows), 1 x 2 (no expansion) and
    8 x 1, at N = 4096: every answer bit for bit, and decrypted to the row."""
    prm, ctx = _setup("tiny")
    levels = max(0, (rows - 1).bit_length())
    db = W.pir_plaintexts(rows, cols, prm.N, prm.t, seed=52)
    Wl.wally_pir_load(ctx.ptr, db)
    n = len(wanted)
    cr, sec, keys, cts, _ = _client(ctx, prm, n, levels, wanted, seed=53)
    out = torch.empty((n, cols, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_pir_answer(ctx.ptr, n, cts, keys, out)
    Wl.wally_sync(ctx.ptr)
    got = Wl.to_u64_numpy(out)
    kg = Wl.to_u64_numpy(keys)
    ct = Wl.to_u64_numpy(cts)
    for i in range(n):
        ind = O.pir_expand(prm, ct[i], [kg[i, a] for a in range(levels)], levels)
        ref = O.pir_first_dimension(prm, db, ind)
        assert np.array_equal(got[i], ref), i
    coeffs = torch.empty((n * cols, prm.N), dtype=torch.int64, device=DEV)
    idx = torch.tensor([i for i in range(n) for _ in range(cols)], dtype=torch.int32, device=DEV)
    Wl.wally_decrypt_poly(ctx.ptr, n * cols, sec, idx, out.reshape(n * cols, 2, prm.L, prm.N), coeffs)
    dec = coeffs.cpu().numpy().reshape(n, cols, prm.N)
    for i, r in enumerate(wanted):
        assert np.array_equal(dec[i], db[r].astype(np.int64)), i
    ctx.close()


def test_pir_answer_batched_parameters():
    """N = 8192, three 50-bit limbs: a 64 x 4 table (6 levels), 70 queries
    (two chunks of the answer loop, which takes 64 at a time); all decrypt
    to their rows, one of the second chunk bit for bit against the oracle."""
    prm, ctx = _setup("batched")
    rows, cols, levels = 64, 4, 6
    db = W.pir_plaintexts(rows, cols, prm.N, prm.t, seed=54)
    Wl.wally_pir_load(ctx.ptr, db)
    wanted = [int(x) for x in np.random.default_rng(55).integers(0, rows, 70)]
    cr, sec, keys, cts, _ = _client(ctx, prm, len(wanted), levels, wanted, seed=56)
    out = torch.empty((len(wanted), cols, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_pir_answer(ctx.ptr, len(wanted), cts, keys, out)
    Wl.wally_sync(ctx.ptr)
    n = len(wanted)
    coeffs = torch.empty((n * cols, prm.N), dtype=torch.int64, device=DEV)
    idx = torch.tensor([i for i in range(n) for _ in range(cols)], dtype=torch.int32, device=DEV)
    Wl.wally_decrypt_poly(ctx.ptr, n * cols, sec, idx, out.reshape(n * cols, 2, prm.L, prm.N), coeffs)
    dec = coeffs.cpu().numpy().reshape(n, cols, prm.N)
    for i, r in enumerate(wanted):
        assert np.array_equal(dec[i], db[r].astype(np.int64)), i
    i = 67
    kg = Wl.to_u64_numpy(keys[i])
    ind = O.pir_expand(prm, Wl.to_u64_numpy(cts[i]), [kg[a] for a in range(levels)], levels)
    assert np.array_equal(Wl.to_u64_numpy(out[i]), O.pir_first_dimension(prm, db, ind))
    ctx.close()


def test_pir_errors():
    prm, ctx = _setup("tiny")
    x = torch.zeros(8, dtype=torch.int64, device=DEV)
    with pytest.raises(Wl.WallyError) as e:
        Wl.wally_pir_answer(ctx.ptr, 1, x, x, x)
    assert e.value.code == Wl.WALLY_ESTATE
    bad = np.full((2, 1, prm.N), prm.t, np.uint64)
    with pytest.raises(Wl.WallyError) as e:
        Wl.wally_pir_load(ctx.ptr, bad)
    assert e.value.code == Wl.WALLY_EINVAL
    ctx.close()


def test_relin_key_parity():
    prm, ctx = _setup("tiny")
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=71)
    keys = torch.empty((2, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_keygen_relin(ctx.ptr, 2, torch.from_numpy(cr.secret).to(DEV), Wl.u64_tensor(cr.key_a[:, 0], DEV),
                          torch.from_numpy(np.ascontiguousarray(cr.key_e[:, 0])).to(DEV), keys)
    got = Wl.to_u64_numpy(keys)
    for i in range(2):
        assert np.array_equal(got[i], O.relin_keygen(prm, cr.secret[i], cr.key_a[i, 0], cr.key_e[i, 0])), i
    ctx.close()


@pytest.mark.parametrize("rows,cols,nq", [(4, 2, 3), (40, 9, 10)])
def test_pir_two_dimensions(rows, cols, nq):
    """MulPIR with both dimensions at N = 8192, three 50-bit limbs: one
    answer ciphertext a query, decrypting to table[row][col]; the first
    query bit for bit against the oracle (expansion, first dimension, exact
    tensor summed over the columns, one rescaling, one relinearisation)."""
    prm, ctx = _setup("batched")
    levels = (rows + cols - 1).bit_length()
    db = W.pir_plaintexts(rows, cols, prm.N, prm.t, seed=72)
    Wl.wally_pir_load(ctx.ptr, db)
    rng = np.random.default_rng(73)
    want = [(int(rng.integers(0, rows)), int(rng.integers(0, cols))) for _ in range(nq)]
    cr = W.pir_client_randomness(nq, levels, prm.N, prm.q, prm.P, seed=74)
    rc = W.client_randomness(nq, prm.N, prm.q, prm.P, seed=75)
    sec = torch.from_numpy(cr.secret).to(DEV)
    keys = torch.empty((nq, levels, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_keygen_galois(ctx.ptr, nq, [O.pir_galois(prm, a) for a in range(levels)], sec,
                           Wl.u64_tensor(cr.key_a, DEV), torch.from_numpy(cr.key_e).to(DEV), keys)
    rlk = torch.empty((nq, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_keygen_relin(ctx.ptr, nq, sec, Wl.u64_tensor(np.ascontiguousarray(rc.key_a[:, 0]), DEV),
                          torch.from_numpy(np.ascontiguousarray(rc.key_e[:, 0])).to(DEV), rlk)
    m = np.stack([O.pir_query_plaintext2(prm, r, c, rows, levels) for r, c in want])
    cts = torch.empty((nq, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_encrypt_poly(ctx.ptr, nq, sec, Wl.u64_tensor(m, DEV), Wl.u64_tensor(cr.enc_a, DEV),
                          torch.from_numpy(cr.enc_e).to(DEV), cts)
    out = torch.empty((nq, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_pir_answer2(ctx.ptr, nq, cts, keys, rlk, out)
    Wl.wally_sync(ctx.ptr)
    coeffs = torch.empty((nq, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_decrypt_poly(ctx.ptr, nq, sec, None, out, coeffs)
    dec = coeffs.cpu().numpy()
    for i, (r, c) in enumerate(want):
        assert np.array_equal(dec[i], db[r, c].astype(np.int64)), i
    kg = Wl.to_u64_numpy(keys[0])
    ind = O.pir_expand(prm, Wl.to_u64_numpy(cts[0]), [kg[a] for a in range(levels)], levels)
    first = O.pir_first_dimension(prm, db, ind[:rows])
    ref = O.pir_second_dimension(prm, first, ind[rows:rows + cols], Wl.to_u64_numpy(rlk[0]))
    assert np.array_equal(Wl.to_u64_numpy(out[0]), ref)
    ctx.close()


def test_pir_answer_with_derived_keys():
    """Key derivation (Sec. 4.2): at N = 4096 a 200-row table needs 8 levels;
    the client sends the keys of levels 5..7 only, the server substitutes
    2^(5-a) times with the level-5 key below; bit for bit against the
    oracle's derived expansion, and decrypted."""
    prm, ctx = _setup("tiny")
    rows, cols, levels = 200, 2, 8
    db = W.pir_plaintexts(rows, cols, prm.N, prm.t, seed=57)
    Wl.wally_pir_load(ctx.ptr, db)
    Wl.wally_pir_derive_keys(ctx.ptr, True)
    first, count = Wl.wally_pir_key_levels(ctx.ptr)
    assert (first, count) == (5, 3) and first == O.pir_key_base(prm, levels)
    wanted = [137, 4]
    n = len(wanted)
    cr = W.pir_client_randomness(n, levels, prm.N, prm.q, prm.P, seed=58)
    sec = torch.from_numpy(cr.secret).to(DEV)
    keys = torch.empty((n, count, prm.L, 2, prm.L + 1, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_keygen_galois(ctx.ptr, n, [O.pir_galois(prm, a) for a in range(first, levels)], sec,
                           Wl.u64_tensor(np.ascontiguousarray(cr.key_a[:, first:]), DEV),
                           torch.from_numpy(np.ascontiguousarray(cr.key_e[:, first:])).to(DEV), keys)
    m = np.stack([O.pir_query_plaintext(prm, r, levels) for r in wanted])
    cts = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_encrypt_poly(ctx.ptr, n, sec, Wl.u64_tensor(m, DEV), Wl.u64_tensor(cr.enc_a, DEV),
                          torch.from_numpy(cr.enc_e).to(DEV), cts)
    out = torch.empty((n, cols, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
    Wl.wally_pir_answer(ctx.ptr, n, cts, keys, out)
    Wl.wally_sync(ctx.ptr)
    got = Wl.to_u64_numpy(out)
    kg = Wl.to_u64_numpy(keys[0])
    ind = O.pir_expand(prm, Wl.to_u64_numpy(cts[0]), [kg[a] for a in range(count)], levels, derive=True)
    assert np.array_equal(got[0], O.pir_first_dimension(prm, db, ind))
    coeffs = torch.empty((n * cols, prm.N), dtype=torch.int64, device=DEV)
    idx = torch.tensor([i for i in range(n) for _ in range(cols)], dtype=torch.int32, device=DEV)
    Wl.wally_decrypt_poly(ctx.ptr, n * cols, sec, idx, out.reshape(n * cols, 2, prm.L, prm.N), coeffs)
    dec = coeffs.cpu().numpy().reshape(n, cols, prm.N)
    for i, r in enumerate(wanted):
        assert np.array_equal(dec[i], db[r].astype(np.int64)), i
    ctx.close()
