"""Plain CPU oracle of Wally's BFV server evaluation (arXiv 2406.06761).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` are the only users.  The product
library never imports this package, and this package never imports the
product library.  The arithmetic lives in ``wally_oracle.c`` (compiled with
gcc on first use); this wrapper adds the big-integer half of decryption
(CRT composition and the t/Q scaling, Sec. 2 decryption formula), which Python
integers state directly.

Every function cites the passage of the paper it follows; the readings taken
where the paper is silent are listed in the header of ``wally_oracle.c``.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wally_oracle.c")
_BUILD = os.path.join(_HERE, "_oracle_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_MAX_MODS = 18
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, position independent, pthreads)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("logN", ctypes.c_uint32), ("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("d", ctypes.c_uint32),
        ("d_pad", ctypes.c_uint32), ("g", ctypes.c_uint32), ("h", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
        ("mod", ctypes.c_uint64 * _MAX_MODS), ("psi", ctypes.c_uint64 * _MAX_MODS),
        ("delta", ctypes.c_uint64 * _MAX_MODS), ("k1", ctypes.c_uint64), ("kg", ctypes.c_uint64),
    ]


_u64p = ctypes.POINTER(ctypes.c_uint64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_pp = ctypes.POINTER(_Params)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "or_params_init": (ctypes.c_int, [ctypes.c_uint32] * 5 + [_u64p, ctypes.c_uint64, ctypes.c_uint64, _pp]),
                "or_params_set_split": (ctypes.c_int, [_pp, ctypes.c_uint32]),
                "or_relinkey": (None, [_pp, _i8p, _u64p, _i8p, _u64p]),
                "or_is_prime": (ctypes.c_int, [ctypes.c_uint64]),
                "or_prev_prime_1mod": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
                "or_smallest_root": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint32]),
                "or_ntt_fwd": (None, [_pp, ctypes.c_uint32, _u64p]),
                "or_ntt_inv": (None, [_pp, ctypes.c_uint32, _u64p]),
                "or_polymul": (None, [_pp, ctypes.c_uint32, _u64p, _u64p, _u64p]),
                "or_polymul_schoolbook": (None, [_pp, ctypes.c_uint32, _u64p, _u64p, _u64p]),
                "or_automorphism": (None, [_pp, ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p]),
                "or_slots_encode": (None, [_pp, _u64p, _u64p]),
                "or_slots_decode": (None, [_pp, _u64p, _u64p]),
                "or_replicate_query": (None, [_pp, _i32p, _u64p]),
                "or_encode_cluster": (ctypes.c_int, [_pp, ctypes.c_uint32, _i8p, _u64p]),
                "or_keygen": (None, [_pp, _i8p, ctypes.c_uint64, _u64p, _i8p, _u64p]),
                "or_encrypt": (None, [_pp, _i8p, _u64p, _u64p, _i8p, _u64p]),
                "or_decrypt_residues": (None, [_pp, _i8p, _u64p, _u64p]),
                "or_rotate": (None, [_pp, ctypes.c_uint64, _u64p, _u64p, _u64p]),
                "or_ptct_sum": (None, [_pp, ctypes.c_uint32, _u64p, _u64p, _u64p]),
                "or_ptxt_to_ntt": (None, [_pp, ctypes.c_uint32, _u64p, _u64p]),
                "or_eval": (ctypes.c_int, [_pp, ctypes.c_uint32, _u64p, _u64p, _u64p, _u64p]),
                "or_compress": (None, [_pp, _u64p, ctypes.c_uint32, ctypes.c_uint32, _u64p]),
                "or_decompress_residue": (None, [_pp, _i8p, _u64p, ctypes.c_uint32, ctypes.c_uint32, _u64p]),
                "or_eval_batch": (ctypes.c_int, [_pp, ctypes.c_uint32, _u32p, ctypes.POINTER(_u64p), ctypes.c_uint32,
                                                 _u32p, _u64p, _u64p, _u64p, _u64p, ctypes.c_uint32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray, ty):
    return a.ctypes.data_as(ty)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int8)


class Params:
    """BFV/RNS parameters (Sec. 2, Sec. 7 "Parameters Selection").

    ``mods[:L]`` are the ciphertext primes q_i, ``mods[L]`` the special prime P,
    ``mods[L+1]`` the plaintext modulus t; modulus index j selects one of them
    in the ring functions below.
    """

    def __init__(self, raw: _Params):
        self.raw = raw
        self.N = raw.N
        self.log_n = raw.logN
        self.L = raw.L
        self.q = [int(raw.mod[i]) for i in range(raw.L)]
        self.P = int(raw.mod[raw.L])
        self.t = int(raw.mod[raw.L + 1])
        self.mods = self.q + [self.P, self.t]
        self.psi = [int(raw.psi[i]) for i in range(raw.L + 2)]
        self.zeta_t = self.psi[raw.L + 1]
        self.delta = [int(raw.delta[i]) for i in range(raw.L)]
        self.d, self.d_pad, self.g, self.h = raw.d, raw.d_pad, raw.g, raw.h
        self.k1, self.kg = int(raw.k1), int(raw.kg)
        self.Q = 1
        for q in self.q:
            self.Q *= q

    @property
    def ptr(self):
        return ctypes.byref(self.raw)


@functools.lru_cache(maxsize=None)
def params(log_n: int, L: int, q_bits: int, t_bits: int, dim: int,
           q: tuple | None = None, p: int = 0, t: int = 0, baby_steps: int = 0) -> Params:
    """Derive the parameter set (primes by trial division, roots by search).
    baby_steps: another split g x h of the diagonals (Sec. 5: g = d_pad,
    h = 1 is the plain diagonal method for clusters of sqrt(d) chunks or
    more); 0 keeps g = h = sqrt(d_pad)."""
    lib = _load()
    raw = _Params()
    qa = _u64(q) if q else None
    rc = lib.or_params_init(log_n, L, q_bits, t_bits, dim, _p(qa, _u64p) if qa is not None else None, p, t,
                            ctypes.byref(raw))
    if rc != 0:
        raise ValueError(f"or_params_init failed ({rc})")
    if baby_steps and lib.or_params_set_split(ctypes.byref(raw), baby_steps) != 0:
        raise ValueError(f"baby_steps = {baby_steps} does not split d_pad = {raw.d_pad}")
    return Params(raw)


def is_prime(n: int) -> bool:
    return bool(_load().or_is_prime(n))


def prev_prime_1mod(below: int, step: int) -> int:
    return int(_load().or_prev_prime_1mod(below, step))


def smallest_root(t: int, n: int) -> int:
    return int(_load().or_smallest_root(t, n))


# ------------------------------------------------------------------ ring

def ntt_fwd(prm: Params, j: int, a) -> np.ndarray:
    """Negacyclic NTT: A[i] = sum_k a[k] psi^((2i+1)k) mod mods[j] (Sec. 7)."""
    x = _u64(a).copy()
    _load().or_ntt_fwd(prm.ptr, j, _p(x, _u64p))
    return x


def ntt_inv(prm: Params, j: int, a) -> np.ndarray:
    x = _u64(a).copy()
    _load().or_ntt_inv(prm.ptr, j, _p(x, _u64p))
    return x


def polymul(prm: Params, j: int, a, b) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty(prm.N, np.uint64)
    _load().or_polymul(prm.ptr, j, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p))
    return out


def polymul_schoolbook(prm: Params, j: int, a, b) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty(prm.N, np.uint64)
    _load().or_polymul_schoolbook(prm.ptr, j, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p))
    return out


def automorphism(prm: Params, j: int, k: int, a) -> np.ndarray:
    """sigma_k : a(X) -> a(X^k) mod (X^N+1, mods[j]) (Sec. 2 CtRotate, Sec. 4.2)."""
    a = _u64(a)
    out = np.empty(prm.N, np.uint64)
    _load().or_automorphism(prm.ptr, j, k, _p(a, _u64p), _p(out, _u64p))
    return out


def galois_element(prm: Params, r: int) -> int:
    """Left row rotation by r is sigma_(3^r mod 2N) (Sec. 2 CtRotate)."""
    return pow(3, r, 2 * prm.N)


# ------------------------------------------------------------------ slots

def slots_encode(prm: Params, v) -> np.ndarray:
    """Slot vector (values mod t, linear index rho*N/2 + c) -> polynomial mod t."""
    v = _u64(v)
    out = np.empty(prm.N, np.uint64)
    _load().or_slots_encode(prm.ptr, _p(v, _u64p), _p(out, _u64p))
    return out


def slots_decode(prm: Params, m) -> np.ndarray:
    m = _u64(m)
    out = np.empty(prm.N, np.uint64)
    _load().or_slots_decode(prm.ptr, _p(m, _u64p), _p(out, _u64p))
    return out


def replicate_query(prm: Params, q) -> np.ndarray:
    """Alg. "Client Query Generation": the query repeated n/d_pad times (zeros for a fake)."""
    out = np.empty(prm.N, np.uint64)
    if q is None:
        _load().or_replicate_query(prm.ptr, None, _p(out, _u64p))
    else:
        qa = np.ascontiguousarray(q, dtype=np.int32)
        _load().or_replicate_query(prm.ptr, _p(qa, _i32p), _p(out, _u64p))
    return out


def encode_cluster(prm: Params, emb) -> tuple[int, np.ndarray]:
    """Alg. "Server Initialization": diagonals, packing, BSGS pre-rotation, encoding.

    Returns (m, plaintexts[m][h][g][L][N]) in coefficient form."""
    emb = _i8(emb).reshape(-1, prm.d) if len(emb) else np.zeros((0, prm.d), np.int8)
    size = emb.shape[0]
    m = max(1, -(-size // prm.N))
    out = np.empty((m, prm.h, prm.g, prm.L, prm.N), np.uint64)
    got = _load().or_encode_cluster(prm.ptr, size, _p(emb, _i8p) if size else None, _p(out, _u64p))
    assert got == m
    return m, out


# ------------------------------------------------------------------ client

def keygen(prm: Params, s, k: int, a_rand, e_rand) -> np.ndarray:
    """Galois key for element k, layout [L][2][L+1][N] (Sec. 5, Sec. 7 hybrid key switching)."""
    s, a_rand, e_rand = _i8(s), _u64(a_rand), _i8(e_rand)
    assert a_rand.size == prm.L * (prm.L + 1) * prm.N and e_rand.size == prm.L * prm.N
    out = np.empty((prm.L, 2, prm.L + 1, prm.N), np.uint64)
    _load().or_keygen(prm.ptr, _p(s, _i8p), k, _p(a_rand, _u64p), _p(e_rand, _i8p), _p(out, _u64p))
    return out


def keygen_pair(prm: Params, s, a_rand, e_rand) -> np.ndarray:
    """The two keys a query carries (Sec. 7 "Reducing the request size"): rotation by 1, by g."""
    a_rand = _u64(a_rand).reshape(2, -1)
    e_rand = _i8(e_rand).reshape(2, -1)
    return np.stack([keygen(prm, s, prm.k1, a_rand[0], e_rand[0]), keygen(prm, s, prm.kg, a_rand[1], e_rand[1])])


def encrypt(prm: Params, s, m_poly, a_rand, e) -> np.ndarray:
    """Symmetric BFV encryption of a plaintext polynomial m (coefficients in [0, t))."""
    s, m_poly, a_rand, e = _i8(s), _u64(m_poly), _u64(a_rand), _i8(e)
    out = np.empty((2, prm.L, prm.N), np.uint64)
    _load().or_encrypt(prm.ptr, _p(s, _i8p), _p(m_poly, _u64p), _p(a_rand, _u64p), _p(e, _i8p), _p(out, _u64p))
    return out


def encrypt_slots(prm: Params, s, v, a_rand, e) -> np.ndarray:
    return encrypt(prm, s, slots_encode(prm, v), a_rand, e)


def encrypt_query(prm: Params, s, q, a_rand, e) -> np.ndarray:
    """EncSemPt of the replicated query (Alg. "Client Query Generation"); q=None is a fake."""
    return encrypt_slots(prm, s, replicate_query(prm, q), a_rand, e)


def _crt(prm: Params, x: np.ndarray) -> list[int]:
    Q = prm.Q
    coef = []
    for qi in prm.q:
        Qi = Q // qi
        coef.append(Qi * pow(Qi % qi, -1, qi))
    rows = [[int(v) for v in x[i]] for i in range(prm.L)]
    return [sum(rows[i][n] * coef[i] for i in range(prm.L)) % Q for n in range(prm.N)]


def decrypt_poly(prm: Params, s, ct) -> tuple[np.ndarray, list[int]]:
    """Sec. 2 decryption: x = [c0 + c1*s]_Q, m = round(t*x/Q) mod t (ties up).

    Returns (m coefficients, x as Python integers)."""
    s, ct = _i8(s), _u64(ct)
    x = np.empty((prm.L, prm.N), np.uint64)
    _load().or_decrypt_residues(prm.ptr, _p(s, _i8p), _p(ct, _u64p), _p(x, _u64p))
    xs = _crt(prm, x)
    Q, t = prm.Q, prm.t
    m = np.array([((t * v + Q // 2) // Q) % t for v in xs], dtype=np.uint64)
    return m, xs


def decrypt_slots(prm: Params, s, ct) -> np.ndarray:
    """Decrypt and decode; slot values centred into (-t/2, t/2]."""
    m, _ = decrypt_poly(prm, s, ct)
    v = slots_decode(prm, m).astype(np.int64)
    t = prm.t
    return np.where(v > t // 2, v - t, v)


def noise_bits(prm: Params, s, ct) -> float:
    """log2 of the infinity norm of e = [c0 + c1*s - Delta*m]_Q (centred)."""
    m, xs = decrypt_poly(prm, s, ct)
    Q = prm.Q
    delta = Q // prm.t
    worst = 0
    for v, mv in zip(xs, m):
        e = (v - delta * int(mv)) % Q
        if e > Q // 2:
            e = Q - e
        worst = max(worst, e)
    return float(np.log2(worst)) if worst else 0.0


def noise_budget_bits(prm: Params, s, ct) -> float:
    """log2(Q/2t) - log2||e||: decryption is correct while this is positive (Sec. 2)."""
    return float(np.log2(prm.Q / (2 * prm.t))) - noise_bits(prm, s, ct)


# ------------------------------------------------------------------ server

def rotate(prm: Params, k: int, key, ct) -> np.ndarray:
    """Rot_k = automorphism + hybrid key switching, key [L][2][L+1][N] coefficient form."""
    key, ct = _u64(key), _u64(ct)
    out = np.empty((2, prm.L, prm.N), np.uint64)
    _load().or_rotate(prm.ptr, k, _p(key, _u64p), _p(ct, _u64p), _p(out, _u64p))
    return out


def ptct_sum(prm: Params, ptxt, cts) -> np.ndarray:
    """sum_b P_b * ct_b (PtCtMult + CtCtAdd, Sec. 2)."""
    ptxt, cts = _u64(ptxt), _u64(cts)
    count = ptxt.size // (prm.L * prm.N)
    out = np.empty((2, prm.L, prm.N), np.uint64)
    _load().or_ptct_sum(prm.ptr, count, _p(ptxt, _u64p), _p(cts, _u64p), _p(out, _u64p))
    return out


def ptxt_to_ntt(prm: Params, m: int, ptxt) -> np.ndarray:
    ptxt = _u64(ptxt)
    out = np.empty_like(ptxt)
    _load().or_ptxt_to_ntt(prm.ptr, m, _p(ptxt, _u64p), _p(out, _u64p))
    return out


def eval_query(prm: Params, m: int, ptxt, ct, keys) -> np.ndarray:
    """Alg. "Server Computation" for one query; returns [m][2][L][N] coefficient form."""
    ptxt, ct, keys = _u64(ptxt), _u64(ct), _u64(keys)
    out = np.empty((m, 2, prm.L, prm.N), np.uint64)
    rc = _load().or_eval(prm.ptr, m, _p(ptxt, _u64p), _p(ct, _u64p), _p(keys, _u64p), _p(out, _u64p))
    if rc != 0:
        raise ValueError("or_eval rejected the input (chunks must satisfy 0 < m < g)")
    return out


def eval_batch(prm: Params, clusters_ntt: list, ids, cts, keys, nthreads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Many queries; clusters_ntt[c] = (m_c, plaintexts of cluster c in NTT form).

    Returns (out [sum m][2][L][N], chunk offsets [nq])."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    cts, keys = _u64(cts), _u64(keys)
    chunks = np.array([c[0] for c in clusters_ntt], dtype=np.uint32)
    arrs = [_u64(c[1]) for c in clusters_ntt]
    ptrs = (_u64p * len(arrs))(*[_p(a, _u64p) for a in arrs])
    offs = np.zeros(len(ids), dtype=np.uint64)
    if len(ids):
        offs[1:] = np.cumsum(chunks[ids])[:-1]
    total = int(chunks[ids].sum()) if len(ids) else 0
    out = np.empty((total, 2, prm.L, prm.N), np.uint64)
    rc = _load().or_eval_batch(prm.ptr, len(arrs), _p(chunks, _u32p), ptrs, len(ids), _p(ids, _u32p),
                               _p(cts, _u64p), _p(keys, _u64p), _p(offs, _u64p), _p(out, _u64p),
                               nthreads or os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("or_eval_batch rejected the input")
    return out, offs.astype(np.int64)


# ------------------------------------------------------------------ response compression

def drop_bits(q_last: int, t: int, n: int, z: float = 8.0) -> tuple[int, int]:
    """Bits dropped from c0 and c1 (Sec. 7 "Reducing the response size"):
    l0 = floor(log2(q'/t) - 2), l1 = floor(log2(q'/t) - 2 - log2(z sqrt(2n/9)))."""
    import math
    r = math.log2(q_last / t)
    l0 = max(0, math.floor(r - 2))
    l1 = max(0, math.floor(r - 2 - math.log2(z * math.sqrt(2 * n / 9))))
    return l0, l1


def compress(prm: Params, ct, l0: int, l1: int) -> np.ndarray:
    """Switch a response to its last limb and drop l0 / l1 low bits: [2][N]."""
    ct = _u64(ct)
    out = np.empty((2, prm.N), np.uint64)
    _load().or_compress(prm.ptr, _p(ct, _u64p), l0, l1, _p(out, _u64p))
    return out


def decrypt_compressed_slots(prm: Params, s, cc, l0: int, l1: int) -> np.ndarray:
    """m = round(t x / q') mod t with x = c0'' 2^l0 + c1'' 2^l1 s (mod q'),
    decoded to slots and centred."""
    s, cc = _i8(s), _u64(cc)
    x = np.empty(prm.N, np.uint64)
    _load().or_decompress_residue(prm.ptr, _p(s, _i8p), _p(cc, _u64p), l0, l1, _p(x, _u64p))
    q, t = prm.q[-1], prm.t
    m = np.array([((t * int(v) + q // 2) // q) % t for v in x], dtype=np.uint64)
    v = slots_decode(prm, m).astype(np.int64)
    return np.where(v > t // 2, v - t, v)


# ------------------------------------------------------------------ index PIR (Sec. 4.2)
# The server side of the index PIR under the keyword PIR of Sec. 4.2
# ("Details of keyword PIR", MulPIR): oblivious expansion of the query
# ciphertext into indicator ciphertexts (substitutions, i.e. Galois
# automorphisms X -> X^(N/2^a + 1) followed by key switching, plus additions
# and a monomial shift), then the first dimension: d2 sums of d1
# plaintext-ciphertext products.  Coefficient form throughout.

def pir_galois(prm: Params, a: int) -> int:
    """Galois element of expansion level a: N/2^a + 1 (Sec. 4.2, "Reducing
    evaluation key size")."""
    return prm.N // (1 << a) + 1


def pir_query_plaintext(prm: Params, row: int, levels: int) -> np.ndarray:
    """The client's query plaintext: (2^levels)^-1 mod t times X^row, so that
    after `levels` expansion levels ciphertext `row` encrypts 1 and every
    other one 0."""
    m = np.zeros(prm.N, np.uint64)
    m[row] = pow(1 << levels, -1, prm.t)
    return m


def _ct_add(prm: Params, a, b, sign: int = 1) -> np.ndarray:
    out = np.empty((2, prm.L, prm.N), np.uint64)
    for c in range(2):
        for l, q in enumerate(prm.q):
            x = a[c, l].astype(object)
            y = b[c, l].astype(object)
            out[c, l] = ((x + y) % q if sign > 0 else (x - y) % q).astype(np.uint64)
    return out


def monomial_shift(prm: Params, ct, e: int) -> np.ndarray:
    """ct * X^(-e) in Z_q[X]/(X^N + 1): coefficient n moves to n - e; those
    that wrap below 0 move to n - e + N with their sign flipped (X^-N = -1)."""
    ct = _u64(ct)
    out = np.empty_like(ct)
    N = prm.N
    for c in range(2):
        for l, q in enumerate(prm.q):
            x = ct[c, l]
            out[c, l, :N - e] = x[e:]
            out[c, l, N - e:] = (np.uint64(q) - x[:e]) % np.uint64(q)
    return out


def pir_key_base(prm: Params, levels: int) -> int:
    """Sec. 4.2 "Reducing evaluation key size": (N/2^a + 1)^2 = N/2^(a-1) + 1
    (mod 2N) while a <= floor((log2 N - 1) / 2), so the client sends the key
    of level b = min(levels - 1, floor((log2 N - 1) / 2)) and those above it;
    the server reaches a level a < b by substituting 2^(b - a) times with the
    key of level b."""
    return max(0, min(levels - 1, (prm.log_n - 1) // 2))


def pir_expand(prm: Params, ct, keys, levels: int, derive: bool = False) -> np.ndarray:
    """Oblivious expansion (Angel et al., used by MulPIR): at level a every
    ciphertext C becomes C + sigma(C) (kept at index i) and
    (C - sigma(C)) X^(-2^a) (index i + 2^a), sigma = substitution by
    N/2^a + 1 with keys[a].  With derive, keys holds the keys of levels
    b .. levels - 1 only (pir_key_base) and sigma for a < b is the
    substitution by N/2^b + 1 applied 2^(b - a) times.  Returns
    [2^levels][2][L][N]."""
    b = pir_key_base(prm, levels) if derive else 0
    cur = [_u64(ct)]
    for a in range(levels):
        k = pir_galois(prm, a)
        half = len(cur)
        nxt = [None] * (2 * half)
        for i, C in enumerate(cur):
            if derive and a < b:
                S = C
                for _ in range(1 << (b - a)):
                    S = rotate(prm, pir_galois(prm, b), keys[0], S)
            else:
                S = rotate(prm, k, keys[a - b], C)
            nxt[i] = _ct_add(prm, C, S, +1)
            nxt[i + half] = monomial_shift(prm, _ct_add(prm, C, S, -1), 1 << a)
        cur = nxt
    return np.stack(cur)


def lift_plaintext(prm: Params, m) -> np.ndarray:
    """A plaintext polynomial (coefficients in [0, t)) lifted centred into
    every ciphertext modulus (reading R9): [L][N]."""
    m = _u64(m).astype(np.int64)
    t = prm.t
    v = np.where(m > (t - 1) // 2, m - t, m)
    return np.stack([(v % q).astype(np.uint64) for q in prm.q])


def pir_first_dimension(prm: Params, db, indicators) -> np.ndarray:
    """MulPIR's first dimension: out[j] = sum_i db[i][j] * indicators[i]
    (PtCtMult + CtCtAdd), db [d1][d2][N] coefficients in [0, t).
    Returns [d2][2][L][N]."""
    db = _u64(db)
    d1, d2 = db.shape[0], db.shape[1]
    ind = _u64(indicators)[:d1]
    out = np.empty((d2, 2, prm.L, prm.N), np.uint64)
    for j in range(d2):
        pts = np.stack([lift_plaintext(prm, db[i, j]) for i in range(d1)])
        out[j] = ptct_sum(prm, pts, ind)
    return out


# ------------------------------------------------------------------ ciphertext products (MulPIR's second dimension)
# BFV multiplication (Sec. 2 CtCtMult; used by MulPIR's second dimension,
# Sec. 4.2): the tensor of the centred lifts over Z[X]/(X^N + 1), scaled by
# t/Q and rounded, then relinearised with the key switching key from s^2 to s.
# The exact integer tensor is formed from negacyclic products modulo enough
# extra primes, composed by the Chinese remainder theorem with Python
# integers.

def relin_keygen(prm: Params, s, a_rand, e_rand) -> np.ndarray:
    """Key switching key from s^2 to s, layout [L][2][L+1][N]."""
    s, a_rand, e_rand = _i8(s), _u64(a_rand), _i8(e_rand)
    out = np.empty((prm.L, 2, prm.L + 1, prm.N), np.uint64)
    _load().or_relinkey(prm.ptr, _p(s, _i8p), _p(a_rand, _u64p), _p(e_rand, _i8p), _p(out, _u64p))
    return out


def _centred(prm: Params, limbs) -> list[int]:
    """Integers in (-Q/2, Q/2] from residues [L][N] (CRT)."""
    Q = prm.Q
    out = [0] * prm.N
    for l, q in enumerate(prm.q):
        Ml = Q // q
        c = Ml * pow(Ml % q, -1, q)
        x = limbs[l]
        for n in range(prm.N):
            out[n] += int(x[n]) * c
    half = Q // 2
    return [v % Q - Q if v % Q > half else v % Q for v in out]


def _ext_params(prm: Params, bound_bits: int) -> Params:
    """The ciphertext primes followed by further primes = 1 mod 2N below P,
    enough that their product exceeds 2^bound_bits."""
    qs, below, bits = list(prm.q), prm.P, 0
    for q in prm.q:
        bits += q.bit_length() - 1
    while bits <= bound_bits:
        below = prev_prime_1mod(below, 2 * prm.N)
        qs.append(below)
        bits += below.bit_length() - 1
    return params(prm.log_n, len(qs), 61, 10, prm.d, q=tuple(qs), t=prm.t)


def tensor(prm: Params, pairs) -> list[list[int]]:
    """sum over (a, b) in pairs of (A0 B0, A0 B1 + A1 B0, A1 B1), exact integer
    negacyclic products of the centred lifts A, B."""
    bound = (len(pairs) * prm.N).bit_length() + 2 * prm.Q.bit_length() + 2
    ext = _ext_params(prm, bound)
    R = ext.Q
    acc = [[np.zeros(prm.N, np.uint64) for _ in ext.q] for _ in range(3)]
    for a, b in pairs:
        A = [_centred(prm, _u64(a)[c]) for c in range(2)]
        Bv = [_centred(prm, _u64(b)[c]) for c in range(2)]
        for j, p in enumerate(ext.q):
            Ar = [np.array([v % p for v in A[c]], np.uint64) for c in range(2)]
            Br = [np.array([v % p for v in Bv[c]], np.uint64) for c in range(2)]
            prods = [polymul(ext, j, Ar[0], Br[0]),
                     (polymul(ext, j, Ar[0], Br[1]).astype(object) + polymul(ext, j, Ar[1], Br[0]).astype(object)) % p,
                     polymul(ext, j, Ar[1], Br[1])]
            for k in range(3):
                acc[k][j] = ((acc[k][j].astype(object) + np.asarray(prods[k]).astype(object)) % p).astype(np.uint64)
    out = []
    for k in range(3):
        vals = [0] * prm.N
        for j, p in enumerate(ext.q):
            Mj = R // p
            c = Mj * pow(Mj % p, -1, p)
            x = acc[k][j]
            for n in range(prm.N):
                vals[n] += int(x[n]) * c
        out.append([v % R - R if v % R > R // 2 else v % R for v in vals])
    return out


def scale_round(prm: Params, T: list[int]) -> np.ndarray:
    """round(t T / Q) mod q_l (halves rounded up): [L][N]."""
    Q, t = prm.Q, prm.t
    v = [(2 * t * x + Q) // (2 * Q) for x in T]
    return np.stack([np.array([x % q for x in v], np.uint64) for q in prm.q])


def relinearize(prm: Params, c3, rlk) -> np.ndarray:
    """(c0, c1, c2) -> (c0, c1) + key switch of c2 from s^2 to s: the hybrid
    key switch of Rot with the identity automorphism (k = 1)."""
    c3 = _u64(c3)
    r = rotate(prm, 1, rlk, np.stack([c3[0], c3[2]]))
    return _ct_add(prm, r, np.stack([np.zeros_like(c3[1]), c3[1]]), +1)


def mul_relin(prm: Params, a, b, rlk) -> np.ndarray:
    T = tensor(prm, [(a, b)])
    return relinearize(prm, np.stack([scale_round(prm, T[k]) for k in range(3)]), rlk)


def pir_second_dimension(prm: Params, first, col_ind, rlk) -> np.ndarray:
    """MulPIR's second dimension: sum_j first[j] x col_ind[j] with the
    tensors summed before the one rescaling and the one relinearisation."""
    T = tensor(prm, list(zip(_u64(first), _u64(col_ind))))
    return relinearize(prm, np.stack([scale_round(prm, T[k]) for k in range(3)]), rlk)


def pir_query_plaintext2(prm: Params, row: int, col: int, d1: int, levels: int) -> np.ndarray:
    """A two-dimensional query: (2^levels)^-1 (X^row + X^(d1 + col)); after
    expansion, ciphertext row and ciphertext d1 + col encrypt 1."""
    m = np.zeros(prm.N, np.uint64)
    inv = pow(1 << levels, -1, prm.t)
    m[row] = inv
    m[d1 + col] = (int(m[d1 + col]) + inv) % prm.t
    return m
