"""Pins of the CPU oracle against the mathematics and the paper (no GPU).

Each test checks the oracle against something other than itself: a library
routine (sympy primality, numpy convolution), a closed form, direct
evaluation, a big-integer restatement (tests/bigint_ref.py), a worked example
printed in the paper (tests/golden/), or decryption of the result.
"""
import os

import numpy as np
import pytest
import sympy

import oracle as O
from paper_2406_06761_gb300 import workload as W
from tests import bigint_ref as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(i=0):
    return np.random.default_rng(1234 + i)


def _rand_poly(p, N, i=0):
    return _rng(i).integers(0, p, size=N, dtype=np.uint64)


# ------------------------------------------------------------------ parameters

@pytest.mark.parametrize("name", ["tiny", "batched", "wide"])
def test_primes_are_the_largest_of_their_form(name):
    """Sec. 2 "Vectorized SHE" (t prime, t = 1 mod 2n) and the configs' rule for
    q_i: the largest primes = 1 mod 2N below 2^bits; P the next one below."""
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    two_n = 2 * prm.N
    bound = 1 << w.q_bits
    for x in prm.q + [prm.P]:
        assert sympy.isprime(x) and x % two_n == 1
    chain = [bound] + prm.q + [prm.P]
    for hi, lo in zip(chain, chain[1:]):
        # no prime of the form strictly between lo and hi
        c = lo + two_n
        while c < hi:
            assert not sympy.isprime(c)
            c += two_n
    t = prm.t
    assert sympy.isprime(t) and t % two_n == 1 and t < (1 << w.t_bits)
    c = t + two_n
    while c < (1 << w.t_bits):
        assert not sympy.isprime(c)
        c += two_n


@pytest.mark.parametrize("name", ["tiny", "batched", "wide"])
def test_delta_is_floor_q_over_t(name):
    """Sec. 2: ciphertexts carry floor(Q/t)*m; the oracle stores it per limb."""
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    delta = prm.Q // prm.t
    assert prm.delta == [delta % q for q in prm.q]


@pytest.mark.parametrize("name", ["tiny", "batched", "wide"])
def test_slot_root_is_smallest_primitive_2n_root(name):
    """Reading R7: zeta_t is the smallest x of multiplicative order 2N mod t."""
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    z = prm.zeta_t
    assert sympy.n_order(z, prm.t) == 2 * prm.N
    for x in range(2, z):
        assert sympy.n_order(x, prm.t) != 2 * prm.N


def test_bsgs_dimensions_match_paper():
    """Sec. 4.1 packing / BSGS counts (tests/golden/packing_sec41.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "packing_sec41.txt")) if l.strip() and l[0] != "#"]
    for n, nprime, d_pad, mults, resp, g, h in (map(int, r) for r in rows):
        log_n = n.bit_length() - 1
        prm = O.params(log_n, 1, 40 if log_n < 14 else 50, 22 if log_n == 14 else 20, d_pad)
        m = -(-nprime // n)
        assert prm.d_pad == d_pad and prm.g == g and prm.h == h
        assert m * prm.g * prm.h == mults and m == resp


# ------------------------------------------------------------------ NTT / ring

def test_ntt_is_evaluation_at_odd_powers(small_params):
    """A[i] = a(psi^(2i+1)): direct evaluation with Python integers."""
    prm = small_params
    for j in range(prm.L + 2):
        p, psi = prm.mods[j], prm.psi[j]
        assert pow(psi, prm.N, p) == p - 1
        a = _rand_poly(p, prm.N, j)
        A = O.ntt_fwd(prm, j, a)
        for i in range(prm.N):
            x = pow(psi, 2 * i + 1, p)
            assert int(A[i]) == sum(int(a[k]) * pow(x, k, p) for k in range(prm.N)) % p
        assert np.array_equal(O.ntt_inv(prm, j, A), a)


def test_polymul_matches_numpy_convolution(small_params):
    """Negacyclic product = linear convolution folded by X^N = -1."""
    prm = small_params
    for j in range(prm.L + 1):
        p = prm.mods[j]
        a, b = _rand_poly(p, prm.N, 10 + j), _rand_poly(p, prm.N, 20 + j)
        full = np.convolve(a.astype(object), b.astype(object))
        ref = [(int(full[k]) - (int(full[k + prm.N]) if k + prm.N < len(full) else 0)) % p for k in range(prm.N)]
        assert [int(v) for v in O.polymul(prm, j, a, b)] == ref
        assert [int(v) for v in O.polymul_schoolbook(prm, j, a, b)] == ref


def test_polymul_spot_check_n4096(tiny_params):
    """At N = 4096, sampled coefficients of the NTT product by direct sums."""
    prm = tiny_params
    p = prm.q[0]
    a, b = _rand_poly(p, prm.N, 3), _rand_poly(p, prm.N, 4)
    c = O.polymul(prm, 0, a, b)
    ai, bi = [int(v) for v in a], [int(v) for v in b]
    N = prm.N
    for k in (0, 1, 17, 2048, 4095):
        s = sum(ai[x] * bi[k - x] for x in range(k + 1)) - sum(ai[x] * bi[k + N - x] for x in range(k + 1, N))
        assert int(c[k]) == s % p


def test_galois_worked_example():
    """Sec. 4.2: g_a = n/2^a + 1, and 129^2 = 257 (mod 8192) (golden file)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "galois_sec42.txt")) if l.strip() and l[0] != "#"]
    prm = O.params(12, 1, 36, 17, 192)
    for r in rows:
        if r[0] == "square":
            n, base, res = int(r[1]), int(r[2]), int(r[3])
            assert n == prm.N
            a = _rand_poly(prm.q[0], prm.N, 7)
            twice = O.automorphism(prm, 0, base, O.automorphism(prm, 0, base, a))
            assert np.array_equal(twice, O.automorphism(prm, 0, res, a))
        else:
            n, a_idx, ga = map(int, r)
            assert n // 2 ** a_idx + 1 == ga


def test_automorphism_composition_and_evaluation(small_params):
    """sigma_a o sigma_b = sigma_(ab mod 2N); (sigma_k a)(x) = a(x^k) at the roots."""
    prm = small_params
    p, psi, N = prm.q[0], prm.psi[0], prm.N
    a = _rand_poly(p, N, 5)
    for ka, kb in [(3, 5), (3, 3), (7, 2 * N - 1), (prm.kg, prm.k1)]:
        lhs = O.automorphism(prm, 0, ka, O.automorphism(prm, 0, kb, a))
        assert np.array_equal(lhs, O.automorphism(prm, 0, (ka * kb) % (2 * N), a))
    for k in (3, prm.kg):
        sa = O.automorphism(prm, 0, k, a)
        for i in range(N):
            x = pow(psi, 2 * i + 1, p)
            lhs = sum(int(sa[n]) * pow(x, n, p) for n in range(N)) % p
            rhs = sum(int(a[n]) * pow(x, n * k, p) for n in range(N)) % p
            assert lhs == rhs


# ------------------------------------------------------------------ slots

def _rowrot(v, r, N):
    h = N // 2
    return np.concatenate([np.roll(v[:h], -r), np.roll(v[h:], -r)])


def test_slot_encoding_is_evaluation(small_params):
    """Reading R7: slot (rho, c) = m(zeta^(+-3^c)); encode is its inverse."""
    prm = small_params
    N, t, z = prm.N, prm.t, prm.zeta_t
    v = _rng(8).integers(0, t, size=N, dtype=np.uint64)
    m = O.slots_encode(prm, v)
    for s in range(N):
        rho, c = divmod(s, N // 2)
        e = pow(3, c, 2 * N)
        if rho:
            e = 2 * N - e
        x = pow(z, e, t)
        assert sum(int(m[k]) * pow(x, k, t) for k in range(N)) % t == int(v[s])
    assert np.array_equal(O.slots_decode(prm, m), v)


@pytest.mark.parametrize("which", ["small", "tiny"])
def test_rotation_is_left_row_shift(which, small_params, tiny_params):
    """Sec. 2 CtRotate: sigma_(3^r) shifts both rows left by r (reading R6)."""
    prm = small_params if which == "small" else tiny_params
    N, t = prm.N, prm.t
    v = _rng(9).integers(0, t, size=N, dtype=np.uint64)
    m = O.slots_encode(prm, v)
    jt = prm.L + 1
    for r in (1, 2, prm.g, N // 2 - 1):
        k = O.galois_element(prm, r)
        got = O.slots_decode(prm, O.automorphism(prm, jt, k, m))
        assert np.array_equal(got, _rowrot(v, r, N))


def test_replicate_query_layout(tiny_params):
    """Alg. "Client Query Generation": n/d_pad copies of q, zero padding."""
    prm = tiny_params
    q = _rng(11).integers(-15, 16, size=prm.d)
    v = O.replicate_query(prm, q).astype(np.int64)
    v = np.where(v > prm.t // 2, v - prm.t, v)
    blocks = v.reshape(-1, prm.d_pad)
    assert np.all(blocks[:, :prm.d] == q) and np.all(blocks[:, prm.d:] == 0)
    assert np.all(O.replicate_query(prm, None) == 0)


def _decode_plaintexts(prm, pt):
    """Decode every P' of a cluster back to slot values, centred."""
    t = prm.t
    out = np.empty(pt.shape[:3] + (prm.N,), dtype=np.int64)
    for idx in np.ndindex(*pt.shape[:3]):
        lim = pt[idx][0].astype(object)
        q0 = prm.q[0]
        cen = [int(x) - q0 if int(x) > q0 // 2 else int(x) for x in lim]
        mt = np.array([c % t for c in cen], dtype=np.uint64)
        v = O.slots_decode(prm, mt).astype(np.int64)
        out[idx] = np.where(v > t // 2, v - t, v)
    return out


def test_cluster_encoding_bsgs_identity(tiny_params):
    """Sec. 4.1 diagonal identity with BSGS (Alg. "Server Initialization",
    Alg. "Server Computation"): in the slot domain,
    sum_i rowrot(sum_b P'_{i,b} * rowrot(q, b), g*i) = E q for every slot."""
    prm = tiny_params
    N, g, h = prm.N, prm.g, prm.h
    E = W.embeddings(700, prm.d, 15, seed=5)
    q = W.query_vectors(1, prm.d, 15, seed=5)[0]
    m, pt = O.encode_cluster(prm, E)
    assert m == 1
    dec = _decode_plaintexts(prm, pt)
    qrep = O.replicate_query(prm, q).astype(np.int64)
    qrep = np.where(qrep > prm.t // 2, qrep - prm.t, qrep)
    total = np.zeros(N, dtype=np.int64)
    for i in range(h):
        Ti = sum(dec[0, i, b] * _rowrot(qrep, b, N) for b in range(g))
        total += _rowrot(Ti, g * i, N)
    expect = np.zeros(N, dtype=np.int64)
    expect[:700] = E.astype(np.int64) @ q.astype(np.int64)
    assert np.array_equal(total, expect)
    # same as the plain diagonal method of Sec. 4.1 (d rotations, no BSGS)
    plain = np.zeros(N, dtype=np.int64)
    for i in range(h):
        for b in range(g):
            pj = _rowrot(dec[0, i, b], g * i, N)   # undo the pre-rotation by -g*i
            plain += pj * _rowrot(qrep, g * i + b, N)
    assert np.array_equal(plain, expect)


def test_cluster_encoding_two_chunks_and_padding():
    """m = ceil(|C|/N) chunks; padding of d and of the last chunk is zero."""
    prm = O.params(12, 1, 36, 17, 100)   # d = 100 -> d_pad = 128, g = 16, h = 8
    assert (prm.d_pad, prm.g, prm.h) == (128, 16, 8)
    E = W.embeddings(prm.N + 5, prm.d, 15, seed=6)
    m, pt = O.encode_cluster(prm, E)
    assert m == 2
    dec = _decode_plaintexts(prm, pt)
    # chunk 1, diagonal j = 0 (i = 0, b = 0): slots s < 5 hold E[N+s][s mod 128]
    d0 = dec[1, 0, 0]
    for s in range(5):
        assert d0[s] == E[prm.N + s][s % prm.d_pad]
    assert np.all(d0[5:] == 0)
    # diagonal 1 at slot x = 127 reads column 0 of embedding 127 (wrap-around)
    assert dec[0, 0, 1][127] == E[127][0]
    # column x + j >= d is padding
    assert dec[0, 0, 1][99] == 0


def _expected_slots(prm, E, k, i, b):
    """Slot values of P'_{k,i,b} written out from the layout of Sec. 4.1
    (chunk k, slot s = beta*d_pad + x holds embedding k*N + s, diagonal j
    takes column (x + j) mod d_pad) and the BSGS pre-rotation of Alg.
    "Server Initialization" (row rotation right by g*i), as integers."""
    N, half, dp = prm.N, prm.N // 2, prm.d_pad
    j = prm.g * i + b
    p = np.zeros(N, dtype=np.int64)
    for s in range(N):
        u, col = k * N + s, (s % dp + j) % dp
        if u < len(E) and col < prm.d:
            p[s] = int(E[u][col])
    out = np.empty(N, dtype=np.int64)
    sh = (prm.g * i) % half
    for s in range(N):
        rho, c = divmod(s, half)
        out[s] = p[rho * half + (c - sh) % half]
    return out


@pytest.mark.parametrize("which", ["small", "tiny"])
def test_cluster_encoding_lift_is_centred(which, small_params, tiny_params):
    """Reading R9 (the plaintext lift, on which the paper is silent): each
    encoded plaintext, CRT-composed over its L limbs and read as an integer
    in (-Q/2, Q/2], lies in [-(t-1)/2, (t-1)/2] (the centred representative,
    not [0, t)), and decodes mod t to the pre-rotated diagonal it encodes.
    A lift into [0, t) or a dropped limb reduction fails the first check; a
    wrong diagonal, packing or pre-rotation fails the second."""
    prm = small_params if which == "small" else tiny_params
    t, Q = prm.t, 1
    for q in prm.q:
        Q *= int(q)
    E = W.embeddings(11 if which == "small" else 700, prm.d, 15, seed=9)
    m, pt = O.encode_cluster(prm, E)
    picks = [(k, i, b) for k in range(m) for i in range(prm.h) for b in range(prm.g)]
    if which == "tiny":
        picks = [(0, 0, 0), (0, 0, 5), (0, 3, 1), (0, prm.h - 1, prm.g - 1)]
    seen_negative = False
    for k, i, b in picks:
        x = B.poly_crt([pt[k, i, b, l] for l in range(prm.L)], [int(q) for q in prm.q])
        x = [v - Q if v > Q // 2 else v for v in x]
        assert all(-(t - 1) // 2 <= v <= (t - 1) // 2 for v in x), (k, i, b)
        seen_negative |= any(v < 0 for v in x)
        dec = O.slots_decode(prm, np.array([v % t for v in x], dtype=np.uint64)).astype(np.int64)
        dec = np.where(dec > t // 2, dec - t, dec)
        assert np.array_equal(dec, _expected_slots(prm, E, k, i, b)), (k, i, b)
    assert seen_negative  # the centred range is used, not only its upper half


# ------------------------------------------------------------------ client

def test_encrypt_decrypt_roundtrip(tiny_params):
    prm = tiny_params
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=3)
    v = _rng(12).integers(0, prm.t, size=prm.N, dtype=np.uint64)
    ct = O.encrypt_slots(prm, cr.secret[0], v, cr.enc_a[0], cr.enc_e[0])
    got = O.decrypt_slots(prm, cr.secret[0], ct)
    vc = v.astype(np.int64)
    assert np.array_equal(got, np.where(vc > prm.t // 2, vc - prm.t, vc))
    # fresh noise is exactly the drawn error: ||e|| <= 19
    assert O.noise_bits(prm, cr.secret[0], ct) <= np.log2(19) + 1e-9


def test_galois_key_relation(small_params):
    """Reading R2/R3: b_i + a_i*s = e_i + [i=j] P sigma_k(s) on every modulus."""
    prm = small_params
    N, L, P = prm.N, prm.L, prm.P
    cr = W.client_randomness(1, N, prm.q, P, seed=4)
    s = cr.secret[0].astype(np.int64)
    key = O.keygen(prm, cr.secret[0], prm.kg, cr.key_a[0, 1], cr.key_e[0, 1])
    sk = B.automorphism([int(x) for x in s], prm.kg, 1 << 200)
    sk = [x - (1 << 200) if x > (1 << 199) else x for x in sk]
    for i in range(L):
        e = cr.key_e[0, 1, i].astype(np.int64)
        for j, p in enumerate(prm.q + [P]):
            b, a = key[i, 0, j], key[i, 1, j]
            lhs = [(int(x) + y) % p for x, y in zip(b, B.negacyclic_mul(a, [int(v) % p for v in s], p))]
            rhs = [(int(e[n]) + (P * sk[n] if i == j else 0)) % p for n in range(N)]
            assert lhs == rhs


# ------------------------------------------------------------------ server

def test_rotation_bits_match_bigint_definition(small_params):
    """Hybrid key switching (Sec. 7), readings R3/R4: the RNS result equals
    round(sum_i d_i key_i / P) computed over Z_QP with big integers."""
    prm = small_params
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=5)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    v = _rng(13).integers(0, prm.t, size=prm.N, dtype=np.uint64)
    ct = O.encrypt_slots(prm, cr.secret[0], v, cr.enc_a[0], cr.enc_e[0])
    for which, k in ((0, prm.k1), (1, prm.kg)):
        got = O.rotate(prm, k, keys[which], ct)
        ref = B.rotate(prm, k, keys[which].tolist(), ct.tolist())
        assert got.tolist() == ref


@pytest.mark.parametrize("which", ["small", "tiny"])
def test_rotation_decrypts_to_shift(which, small_params, tiny_params):
    """Sec. 2 CtRotate semantics through encryption; noise stays small."""
    prm = small_params if which == "small" else tiny_params
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=6)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    v = _rng(14).integers(0, prm.t, size=prm.N, dtype=np.uint64)
    ct = O.encrypt_slots(prm, cr.secret[0], v, cr.enc_a[0], cr.enc_e[0])
    vc = v.astype(np.int64)
    vc = np.where(vc > prm.t // 2, vc - prm.t, vc)
    for which_key, r in ((0, 1), (1, prm.g)):
        k = O.galois_element(prm, r)
        out = O.rotate(prm, k, keys[which_key], ct)
        assert np.array_equal(O.decrypt_slots(prm, cr.secret[0], out), _rowrot(vc, r, prm.N))
        # key-switching noise: sum_i d_i e_i / P is about L * 19 * N in the worst case
        assert O.noise_bits(prm, cr.secret[0], out) < np.log2(prm.L * 19 * prm.N) + 2


def test_ptct_sum_matches_bigint(small_params):
    prm = small_params
    rng = _rng(15)
    pts = [[rng.integers(0, q, size=prm.N, dtype=np.uint64) for q in prm.q] for _ in range(3)]
    cts = [[[rng.integers(0, q, size=prm.N, dtype=np.uint64) for q in prm.q] for _ in range(2)] for _ in range(3)]
    got = O.ptct_sum(prm, np.array(pts), np.array(cts))
    ref = B.ptct_sum(prm, [[list(map(int, l)) for l in p] for p in pts],
                     [[[list(map(int, l)) for l in c] for c in ct] for ct in cts])
    assert got.tolist() == ref


def test_eval_bits_match_bigint_small(small_params):
    """Whole Alg. "Server Computation" at N = 16 (d = 4, g = h = 2), bit for bit."""
    prm = small_params
    assert (prm.g, prm.h) == (2, 2)
    E = W.embeddings(11, prm.d, 15, seed=7)
    q = W.query_vectors(1, prm.d, 15, seed=7)[0]
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=7)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    m, pt = O.encode_cluster(prm, E)
    got = O.eval_query(prm, m, pt, ct, keys)
    ref = B.eval_query(prm, pt.tolist(), ct.tolist(), [keys[0].tolist(), keys[1].tolist()])
    assert got.tolist() == ref
    sc = O.decrypt_slots(prm, cr.secret[0], got[0])
    assert np.array_equal(sc[:11], (E.astype(np.int64) @ q.astype(np.int64) + prm.t // 2) % prm.t - prm.t // 2)


def test_eval_tiny_decrypts_to_scores(tiny_params):
    """The tiny workload end to end: decrypt(eval(Enc(q))) = E q exactly
    (|E q| <= 192 * 15^2 < t/2, so no wrap, Sec. 7 fixed-point condition),
    padding slots decrypt to 0, and the noise budget stays positive."""
    prm = tiny_params
    w = W.WORKLOADS["tiny"]
    sizes = W.cluster_sizes(w)
    E = W.embeddings(int(sizes.sum()), w.dim, w.entry_bound)
    q = W.query_vectors(1, w.dim, w.entry_bound)[0]
    cr = W.client_randomness(1, prm.N, prm.q, prm.P)
    m, pt = O.encode_cluster(prm, E)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    out = O.eval_query(prm, m, pt, ct, keys)
    sc = O.decrypt_slots(prm, cr.secret[0], out[0])
    assert np.array_equal(sc[:len(E)], E.astype(np.int64) @ q.astype(np.int64))
    assert np.all(sc[len(E):] == 0)
    assert O.noise_budget_bits(prm, cr.secret[0], out[0]) > 5
    # a fake query (all-zero vector) scores zero everywhere
    ctf = O.encrypt_query(prm, cr.secret[0], None, cr.enc_a[0], cr.enc_e[0])
    assert np.all(O.decrypt_slots(prm, cr.secret[0], O.eval_query(prm, m, pt, ctf, keys)[0]) == 0)


def test_eval_rejects_too_many_chunks(tiny_params):
    """Sec. 5: BSGS is used only while the chunk count is below sqrt(d)."""
    prm = tiny_params
    with pytest.raises(ValueError):
        O.eval_query(prm, prm.g, np.zeros((prm.g, prm.h, prm.g, prm.L, prm.N), np.uint64),
                     np.zeros((2, prm.L, prm.N), np.uint64), np.zeros((2, prm.L, 2, prm.L + 1, prm.N), np.uint64))


def test_eval_batch_equals_single(tiny_params):
    """The threaded batch driver returns exactly the per-query results."""
    prm = tiny_params
    E1 = W.embeddings(300, prm.d, 15, seed=8)
    E2 = W.embeddings(900, prm.d, 15, seed=9)
    (m1, p1), (m2, p2) = O.encode_cluster(prm, E1), O.encode_cluster(prm, E2)
    cr = W.client_randomness(3, prm.N, prm.q, prm.P, seed=8)
    qs = W.query_vectors(3, prm.d, 15, seed=8)
    keys = np.stack([O.keygen_pair(prm, cr.secret[i], cr.key_a[i], cr.key_e[i]) for i in range(3)])
    cts = np.stack([O.encrypt_query(prm, cr.secret[i], qs[i], cr.enc_a[i], cr.enc_e[i]) for i in range(3)])
    ids = np.array([1, 0, 1], np.uint32)
    out, offs = O.eval_batch(prm, [(m1, O.ptxt_to_ntt(prm, m1, p1)), (m2, O.ptxt_to_ntt(prm, m2, p2))],
                             ids, cts, keys, nthreads=3)
    for i, c in enumerate(ids):
        m, pt = (m1, p1) if c == 0 else (m2, p2)
        assert np.array_equal(out[offs[i]:offs[i] + m], O.eval_query(prm, m, pt, cts[i], keys[i]))


# ------------------------------------------------------------------ response compression

def test_drop_bits_worked_example():
    """Sec. 7: n = 4096, 27-bit last limb, 16-bit t, z = 8 -> l0 = 9, l1 <= 1
    (the paper uses 0); 55 KB -> 23.5 KB (tests/golden/response_size_sec7.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "response_size_sec7.txt")) if l.strip() and l[0] != "#"]
    for n, qb, tb, z, l0_paper, l1_used, kb in rows:
        n, qb, tb, l0_paper, l1_used = int(n), int(qb), int(tb), int(l0_paper), int(l1_used)
        l0, l1_max = O.drop_bits(2 ** qb, 2 ** tb, n, float(z))
        assert l0 == l0_paper and 0 <= l1_used <= l1_max
        size_kb = n * ((qb - l0) + (qb - l1_used)) / 8 / 1000
        assert abs(size_kb - float(kb)) / float(kb) < 0.03


def test_compress_is_a_chain_of_rounded_divisions(small_params):
    """Reading R16 against big integers: c' = round(...round(c / q_0)... / q_{L-2})
    mod q_{L-1}, then floor((c' + 2^(l-1)) / 2^l)."""
    for prm in (small_params, O.params(4, 3, 30, 10, 4)):
        rng = _rng(40)
        ct = np.stack([np.stack([rng.integers(0, q, size=prm.N, dtype=np.uint64) for q in prm.q]) for _ in range(2)])
        l0, l1 = 7, 3
        got = O.compress(prm, ct, l0, l1)
        for c, l in ((0, l0), (1, l1)):
            comp = B.poly_crt(ct[c], prm.q)
            for n in range(prm.N):
                v, mod = comp[n], prm.Q
                for qi in prm.q[:-1]:
                    v = (2 * v + qi) // (2 * qi)   # nearest integer to v / q_i (q_i odd)
                    mod //= qi
                    v %= mod
                assert int(got[c][n]) == (v + (1 << (l - 1))) >> l


def test_compressed_tiny_response_decrypts(tiny_params):
    prm = tiny_params
    w = W.WORKLOADS["tiny"]
    E = W.embeddings(1024, w.dim, w.entry_bound)
    q = W.query_vectors(1, w.dim, w.entry_bound)[0]
    cr = W.client_randomness(1, prm.N, prm.q, prm.P)
    m, pt = O.encode_cluster(prm, E)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    out = O.eval_query(prm, m, pt, ct, keys)[0]
    l0, l1 = O.drop_bits(prm.q[-1], prm.t, prm.N)
    cc = O.compress(prm, out, l0, l1)
    sc = O.decrypt_compressed_slots(prm, cr.secret[0], cc, l0, l1)
    assert np.array_equal(sc[:1024], E.astype(np.int64) @ q.astype(np.int64)) and np.all(sc[1024:] == 0)


def test_plain_diagonal_split_bits_match_bigint_small():
    """The split g = d_pad, h = 1 (Sec. 5: no pre-rotation and no giant steps
    once a cluster has sqrt(d) chunks or more) at N = 16, d = 4, two chunks,
    bit for bit against the big-integer restatement, and decrypted."""
    prm = O.params(4, 2, 30, 10, 4, baby_steps=4)
    assert (prm.g, prm.h, prm.kg) == (4, 1, pow(3, 4, 32))
    E = W.embeddings(27, prm.d, 15, seed=19)
    q = W.query_vectors(1, prm.d, 15, seed=19)[0]
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=19)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    m, pt = O.encode_cluster(prm, E)
    assert m == 2
    got = O.eval_query(prm, m, pt, ct, keys)
    ref = B.eval_query(prm, pt.tolist(), ct.tolist(), [keys[0].tolist(), keys[1].tolist()])
    assert got.tolist() == ref
    sc = np.concatenate([O.decrypt_slots(prm, cr.secret[0], got[k]) for k in range(m)])
    assert np.array_equal(sc[:27], (E.astype(np.int64) @ q.astype(np.int64) + prm.t // 2) % prm.t - prm.t // 2)


def test_plain_diagonal_split_at_sqrt_d_chunks(tiny_params):
    """A cluster of exactly sqrt(d_pad) = 16 chunks, which BSGS may not take
    (m < g), evaluated with the plain split g = 256, h = 1: the scores
    decrypt exactly; the plaintexts of the plain split are the unrotated
    diagonals, i.e. those of BSGS's first giant step.  (BSGS itself rejects
    m >= g: test_eval_rejects_too_many_chunks.)"""
    w = W.WORKLOADS["tiny"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, baby_steps=256)
    assert (prm.g, prm.h) == (256, 1)
    n = 16 * prm.N
    E = W.embeddings(n, w.dim, w.entry_bound, seed=20)
    q = W.query_vectors(1, w.dim, w.entry_bound, seed=20)[0]
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=20)
    keys = O.keygen_pair(prm, cr.secret[0], cr.key_a[0], cr.key_e[0])
    ct = O.encrypt_query(prm, cr.secret[0], q, cr.enc_a[0], cr.enc_e[0])
    m, pt = O.encode_cluster(prm, E)
    assert m == 16
    got = O.eval_query(prm, m, pt, ct, keys)
    sc = np.concatenate([O.decrypt_slots(prm, cr.secret[0], got[k]) for k in range(m)])
    assert np.array_equal(sc, E.astype(np.int64) @ q.astype(np.int64))
    bsgs = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    m1, pt1 = O.encode_cluster(bsgs, E[:prm.N])
    assert m1 == 1 and np.array_equal(pt[0, 0, :bsgs.g], pt1[0, 0])


# ---------------------------------------------------------------- index PIR (Sec. 4.2)

def _pir_keys(prm, cr, levels):
    return [O.keygen(prm, cr.secret[0], O.pir_galois(prm, a), cr.key_a[0, a], cr.key_e[0, a]) for a in range(levels)]


def test_pir_expansion_bits_match_bigint_small(small_params):
    """Two expansion levels at N = 16, bit for bit against a big-integer
    restatement (substitution = big-integer Rot_k; add, subtract and the
    monomial X^-e over Z_Q)."""
    prm = small_params
    levels = 2
    cr = W.pir_client_randomness(1, levels, prm.N, prm.q, prm.P, seed=41)
    keys = _pir_keys(prm, cr, levels)
    ct = O.encrypt(prm, cr.secret[0], O.pir_query_plaintext(prm, 3, levels), cr.enc_a[0], cr.enc_e[0])
    got = O.pir_expand(prm, ct, keys, levels)

    def shift(c, e):
        out = []
        for comp in range(2):
            limbs = []
            for l, q in enumerate(prm.q):
                x = [int(v) for v in c[comp][l]]
                limbs.append([x[n + e] if n + e < prm.N else (-x[n + e - prm.N]) % q for n in range(prm.N)])
            out.append(limbs)
        return out

    def sub(a, b):
        return [[[(int(x) - int(y)) % prm.q[l] for x, y in zip(a[c][l], b[c][l])] for l in range(prm.L)]
                for c in range(2)]

    cur = [ct.tolist()]
    for a in range(levels):
        k = O.pir_galois(prm, a)
        nxt = [None] * (2 * len(cur))
        for i, C in enumerate(cur):
            S = B.rotate(prm, k, keys[a].tolist(), C)
            nxt[i] = B.add(prm, C, S)
            nxt[i + len(cur)] = shift(sub(C, S), 1 << a)
        cur = nxt
    assert got.tolist() == cur


def test_pir_expansion_decrypts_to_indicators(tiny_params):
    """Expanding (2^c)^-1 X^row over c = 3 levels gives 8 ciphertexts; number
    `row` decrypts to the constant 1 and every other one to 0."""
    prm = tiny_params
    levels, row = 3, 5
    cr = W.pir_client_randomness(1, levels, prm.N, prm.q, prm.P, seed=42)
    keys = _pir_keys(prm, cr, levels)
    ct = O.encrypt(prm, cr.secret[0], O.pir_query_plaintext(prm, row, levels), cr.enc_a[0], cr.enc_e[0])
    ind = O.pir_expand(prm, ct, keys, levels)
    assert ind.shape[0] == 8
    for k in range(8):
        m, _ = O.decrypt_poly(prm, cr.secret[0], ind[k])
        want = np.zeros(prm.N, np.int64)
        want[0] = 1 if k == row else 0
        assert np.array_equal(np.asarray(m, np.int64), want), k


def test_pir_first_dimension_returns_the_row(tiny_params):
    """The first dimension over a 6 x 3 table (rows padded to 8 indicators):
    column j decrypts to the plaintext at (row, j), coefficient for
    coefficient."""
    prm = tiny_params
    levels, row = 3, 4
    db = W.pir_plaintexts(6, 3, prm.N, prm.t, seed=43)
    cr = W.pir_client_randomness(1, levels, prm.N, prm.q, prm.P, seed=43)
    keys = _pir_keys(prm, cr, levels)
    ct = O.encrypt(prm, cr.secret[0], O.pir_query_plaintext(prm, row, levels), cr.enc_a[0], cr.enc_e[0])
    out = O.pir_first_dimension(prm, db, O.pir_expand(prm, ct, keys, levels))
    for j in range(3):
        m, _ = O.decrypt_poly(prm, cr.secret[0], out[j])
        assert np.array_equal(np.asarray(m, np.uint64), db[row, j]), j


def test_monomial_shift_is_negacyclic(small_params):
    """X^-e times a polynomial equals the negacyclic product with the
    coefficient vector of X^(N-e) times -1 (schoolbook)."""
    prm = small_params
    rng = np.random.default_rng(44)
    ct = np.stack([np.stack([rng.integers(0, q, prm.N, dtype=np.uint64) for q in prm.q]) for _ in range(2)])
    for e in (1, 3, 8):
        got = O.monomial_shift(prm, ct, e)
        for c in range(2):
            for l, q in enumerate(prm.q):
                mono = np.zeros(prm.N, np.uint64)
                mono[prm.N - e] = q - 1  # X^-e = -X^(N-e)
                assert np.array_equal(got[c, l], O.polymul_schoolbook(prm, l, ct[c, l], mono)), (e, c, l)


# ---------------------------------------------------------------- ciphertext products (MulPIR's second dimension)

def _schoolbook_z(a, b):
    """Exact negacyclic product over Z (no reduction)."""
    N = len(a)
    out = [0] * N
    for x in range(N):
        for y in range(N):
            k = x + y
            if k < N:
                out[k] += a[x] * b[y]
            else:
                out[k - N] -= a[x] * b[y]
    return out


def test_mul_relin_bits_match_bigint_small(small_params):
    """At N = 16: the tensor of the centred lifts by schoolbook products over
    Z, round(t T / Q) by integer division, and the relinearisation as the
    big-integer key switch of c2 (Rot with k = 1) plus c1 -- bit for bit."""
    prm = small_params
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=61)
    rng = np.random.default_rng(61)
    ma, mb = (rng.integers(0, prm.t, prm.N, dtype=np.uint64) for _ in range(2))
    a = O.encrypt(prm, cr.secret[0], ma, cr.enc_a[0], cr.enc_e[0])
    b = O.encrypt(prm, cr.secret[0], mb, cr.enc_a[1], cr.enc_e[1])
    rlk = O.relin_keygen(prm, cr.secret[0], cr.key_a[0, 0], cr.key_e[0, 0])
    got = O.mul_relin(prm, a, b, rlk)
    Q, t = prm.Q, prm.t

    def lift(ct, c):
        z = B.poly_crt(ct[c].tolist(), prm.q)
        return [v - Q if v > Q // 2 else v for v in z]

    A = [lift(a, c) for c in range(2)]
    Bb = [lift(b, c) for c in range(2)]
    T = [_schoolbook_z(A[0], Bb[0]),
         [x + y for x, y in zip(_schoolbook_z(A[0], Bb[1]), _schoolbook_z(A[1], Bb[0]))],
         _schoolbook_z(A[1], Bb[1])]
    c3 = [[[((2 * t * v + Q) // (2 * Q)) % q for v in T[k]] for q in prm.q] for k in range(3)]
    assert np.array_equal(np.stack([O.scale_round(prm, O.tensor(prm, [(a, b)])[k]) for k in range(3)]),
                          np.array(c3, np.uint64))
    r = B.rotate(prm, 1, rlk.tolist(), [c3[0], c3[2]])
    ref = B.add(prm, r, [[[0] * prm.N for _ in prm.q], c3[1]])
    assert got.tolist() == ref
    m, _ = O.decrypt_poly(prm, cr.secret[0], got)
    assert np.array_equal(np.asarray(m, np.uint64), O.polymul(prm, prm.L + 1, ma, mb))


def test_relin_key_relation(small_params):
    """b_i + a_i s = e_i + [i == j] P s^2 on every limb j of the key."""
    prm = small_params
    cr = W.client_randomness(1, prm.N, prm.q, prm.P, seed=62)
    s = cr.secret[0]
    key = O.relin_keygen(prm, s, cr.key_a[0, 0], cr.key_e[0, 0])
    mods = prm.q + [prm.P]
    for i in range(prm.L):
        for j, p in enumerate(mods):
            sj = np.array([int(v) % p for v in s], np.uint64)
            lhs = (key[i, 0, j].astype(object) + O.polymul_schoolbook(prm, j, key[i, 1, j], sj).astype(object)) % p
            e = np.array([int(v) % p for v in cr.key_e[0, 0, i]], dtype=object)
            s2 = O.polymul_schoolbook(prm, j, sj, sj).astype(object)
            want = (e + ((prm.P % p) * s2 if i == j else 0)) % p
            assert np.array_equal(lhs, want), (i, j)


def test_mul_relin_decrypts_to_product(tiny_params):
    """N = 4096, two 36-bit limbs: the relinearised product of two fresh
    ciphertexts decrypts to the negacyclic product of their plaintexts mod t."""
    prm = tiny_params
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=63)
    rng = np.random.default_rng(63)
    ma, mb = (rng.integers(0, prm.t, prm.N, dtype=np.uint64) for _ in range(2))
    a = O.encrypt(prm, cr.secret[0], ma, cr.enc_a[0], cr.enc_e[0])
    b = O.encrypt(prm, cr.secret[0], mb, cr.enc_a[1], cr.enc_e[1])
    rlk = O.relin_keygen(prm, cr.secret[0], cr.key_a[0, 0], cr.key_e[0, 0])
    m, _ = O.decrypt_poly(prm, cr.secret[0], O.mul_relin(prm, a, b, rlk))
    assert np.array_equal(np.asarray(m, np.uint64), O.polymul(prm, prm.L + 1, ma, mb))


def test_pir_two_dimensions_batched_params():
    """MulPIR end to end at N = 8192, three 50-bit limbs: a 4 x 2 table, one
    query ciphertext for (row 2, column 1), expanded over 3 levels into 8
    indicators (rows 0..3, then columns), first dimension, second dimension
    with one rescaling and one relinearisation: decrypts to table[2][1]."""
    w = W.WORKLOADS["batched"]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    d1, d2, levels, row, col = 4, 2, 3, 2, 1
    db = W.pir_plaintexts(d1, d2, prm.N, prm.t, seed=64)
    cr = W.pir_client_randomness(1, levels, prm.N, prm.q, prm.P, seed=64)
    keys = _pir_keys(prm, cr, levels)
    rc = W.client_randomness(1, prm.N, prm.q, prm.P, seed=65)
    rlk = O.relin_keygen(prm, cr.secret[0], rc.key_a[0, 0], rc.key_e[0, 0])
    ct = O.encrypt(prm, cr.secret[0], O.pir_query_plaintext2(prm, row, col, d1, levels), cr.enc_a[0], cr.enc_e[0])
    ind = O.pir_expand(prm, ct, keys, levels)
    first = O.pir_first_dimension(prm, db, ind[:d1])
    ans = O.pir_second_dimension(prm, first, ind[d1:d1 + d2], rlk)
    m, _ = O.decrypt_poly(prm, cr.secret[0], ans)
    assert np.array_equal(np.asarray(m, np.uint64), db[row, col])


def test_pir_key_derivation_by_squaring(tiny_params):
    """Sec. 4.2 "Reducing evaluation key size": the squaring relation of the
    substitution elements holds up to level floor((log2 N - 1)/2) and fails
    above (N = 4096: 129^2 = 257 mod 8192); an expansion over 8 levels with
    keys only for levels 5..7 decrypts to the same indicators."""
    prm = tiny_params
    b = O.pir_key_base(prm, 8)
    assert b == 5 and O.pir_galois(prm, 5) == 129 and pow(129, 2, 2 * prm.N) == 257
    for a in range(1, b + 1):
        assert pow(O.pir_galois(prm, a), 2, 2 * prm.N) == O.pir_galois(prm, a - 1)
    assert pow(O.pir_galois(prm, b + 1), 2, 2 * prm.N) != O.pir_galois(prm, b)
    levels, row = 8, 77
    cr = W.pir_client_randomness(1, levels, prm.N, prm.q, prm.P, seed=45)
    keys = [O.keygen(prm, cr.secret[0], O.pir_galois(prm, a), cr.key_a[0, a], cr.key_e[0, a]) for a in range(b, levels)]
    ct = O.encrypt(prm, cr.secret[0], O.pir_query_plaintext(prm, row, levels), cr.enc_a[0], cr.enc_e[0])
    ind = O.pir_expand(prm, ct, keys, levels, derive=True)
    for k in (0, row, 255):
        m, _ = O.decrypt_poly(prm, cr.secret[0], ind[k])
        want = np.zeros(prm.N, np.int64)
        want[0] = 1 if k == row else 0
        assert np.array_equal(np.asarray(m, np.int64), want), k


def test_noise_of_additions_and_plaintext_products(tiny_params):
    """Noise invariants of Sec. 2 (Table of operations: addition adds the
    noises, PtCtMult multiplies them by about N ||P||): with e the noise of
    c0 + c1 s - Delta m,
      ||e(a + b)|| <= ||e(a)|| + ||e(b)|| + t           (the carry of m_a + m_b past t costs [Q]_t < t)
      ||e(P a)||   <= N ||P||_inf ||e(a)|| + N t^2 / 4  (centred P; the carry of P m_a past t)."""
    prm = tiny_params
    cr = W.client_randomness(2, prm.N, prm.q, prm.P, seed=66)
    rng = np.random.default_rng(66)
    ma, mb, pv = (rng.integers(0, prm.t, prm.N, dtype=np.uint64) for _ in range(3))
    a = O.encrypt(prm, cr.secret[0], ma, cr.enc_a[0], cr.enc_e[0])
    b = O.encrypt(prm, cr.secret[0], mb, cr.enc_a[1], cr.enc_e[1])
    ea, eb = (2.0 ** O.noise_bits(prm, cr.secret[0], c) for c in (a, b))
    s = O._ct_add(prm, a, b, +1)
    m, _ = O.decrypt_poly(prm, cr.secret[0], s)
    assert np.array_equal(np.asarray(m, np.uint64), (ma + mb) % np.uint64(prm.t))
    assert 2.0 ** O.noise_bits(prm, cr.secret[0], s) <= ea + eb + prm.t
    P = O.lift_plaintext(prm, pv)
    pa = O.ptct_sum(prm, P[None], a[None])
    m, _ = O.decrypt_poly(prm, cr.secret[0], pa)
    assert np.array_equal(np.asarray(m, np.uint64), O.polymul(prm, prm.L + 1, pv, ma))
    pinf = prm.t // 2
    assert 2.0 ** O.noise_bits(prm, cr.secret[0], pa) <= prm.N * pinf * ea + prm.N * prm.t ** 2 / 4


@pytest.mark.parametrize("log_n", [3, 6])
def test_polymul_matches_convolution_other_sizes(log_n):
    """NTT products against the folded linear convolution at N = 8 and 64."""
    prm = O.params(log_n, 2, 30, 10, 4)
    for j in range(prm.L + 1):
        p = prm.mods[j]
        a, b = _rand_poly(p, prm.N, 30 + j), _rand_poly(p, prm.N, 40 + j)
        full = np.convolve(a.astype(object), b.astype(object))
        ref = [(int(full[k]) - (int(full[k + prm.N]) if k + prm.N < len(full) else 0)) % p for k in range(prm.N)]
        assert [int(v) for v in O.polymul(prm, j, a, b)] == ref


@pytest.mark.parametrize("name", ["tiny", "batched", "serving", "full_scale", "wide"])
def test_scores_cannot_wrap_around_t(name):
    """Sec. 7's no-wrap condition for the workloads: the largest possible
    dot product d * bound^2 stays below (t - 1)/2, so decrypted scores are
    the exact integers, not residues."""
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    assert w.dim * w.entry_bound ** 2 < (prm.t - 1) // 2


def test_fake_query_counts_follow_the_negative_binomial():
    """Alg. "Client Query Generation": NB(r = 0.5, p = 0.9) fake queries per
    client: sample mean and variance against r(1-p)/p and r(1-p)/p^2, and
    infinite divisibility (Sec. 8): the sum over U clients of NB(r/U, p) has
    the mean and variance of one NB(r, p)."""
    r, p, n = 0.5, 0.9, 400_000
    c = W.fake_counts(n, r, p, seed=3)
    mean, var = r * (1 - p) / p, r * (1 - p) / p ** 2
    assert abs(c.mean() - mean) < 5 * np.sqrt(var / n)
    assert abs(c.var() - var) / var < 0.05
    U = 8
    parts = sum(W.fake_counts(n, r / U, p, seed=10 + u) for u in range(U))
    assert abs(parts.mean() - mean) < 5 * np.sqrt(var / n)
    assert abs(parts.var() - var) / var < 0.05
