"""The library's host-side number theory (csrc/host_nt.cpp: Miller-Rabin,
prime search, roots of unity, NTT tables, Montgomery constant, multiword
helpers), built with g++ and checked without a GPU against sympy, Python
integers and the oracle's independent trial-division search."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2406_06761_gb300", "csrc")

WRAP = r"""
#include "host_nt.hpp"
using namespace wally;
extern "C" int h_is_prime(uint64_t n) { return is_prime_u64(n) ? 1 : 0; }
extern "C" uint64_t h_prime_below(uint64_t below, uint64_t step) { return prime_1mod_below(below, step); }
extern "C" uint64_t h_root_2n(uint64_t p, uint32_t n) { return root_2n(p, n); }
extern "C" uint64_t h_smallest_root(uint64_t t, uint32_t n) { return smallest_root_2n(t, n); }
extern "C" uint64_t h_mont_neg_inv(uint64_t p) { return mont_neg_inv(p); }
extern "C" void h_tables(uint64_t p, uint64_t psi, uint32_t log_n, uint64_t *fwd, uint64_t *fwd_s, uint64_t *inv)
{
    NttTables t = make_tables(p, psi, log_n);
    for (size_t i = 0; i < t.fwd.size(); i++) { fwd[i] = t.fwd[i]; fwd_s[i] = t.fwd_s[i]; inv[i] = t.inv[i]; }
}
extern "C" int h_big(const uint64_t *a, int na, uint64_t m, uint64_t *prod, uint64_t *quot, uint64_t *rem, uint64_t *mod)
{
    std::vector<uint64_t> v(a, a + na);
    std::vector<uint64_t> p = big_mul_small(v, m), q = big_div_small(v, m, rem);
    for (size_t i = 0; i < p.size(); i++) prod[i] = p[i];
    for (size_t i = 0; i < q.size(); i++) quot[i] = q[i];
    *mod = big_mod_small(v, m);
    return (int)p.size();
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("hnt")
    src = d / "wrap.cpp"
    src.write_text(WRAP)
    so = d / "libhnt.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src),
                           os.path.join(CSRC, "host_nt.cpp"), "-o", str(so)])
    L = ctypes.CDLL(str(so))
    u64 = ctypes.c_uint64
    L.h_is_prime.argtypes = [u64]
    L.h_prime_below.restype = u64
    L.h_prime_below.argtypes = [u64, u64]
    L.h_root_2n.restype = u64
    L.h_root_2n.argtypes = [u64, ctypes.c_uint32]
    L.h_smallest_root.restype = u64
    L.h_smallest_root.argtypes = [u64, ctypes.c_uint32]
    L.h_mont_neg_inv.restype = u64
    L.h_mont_neg_inv.argtypes = [u64]
    L.h_tables.argtypes = [u64, u64, ctypes.c_uint32] + [ctypes.c_void_p] * 3
    L.h_big.argtypes = [ctypes.c_void_p, ctypes.c_int, u64] + [ctypes.c_void_p] * 4
    return L


def test_miller_rabin_against_sympy(lib):
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(5)
    for n in list(rng.integers(2, 2**62, 300)) + [2, 3, 4, 561, 1105, 3215031751, 2**61 - 1, 2**62 - 57]:
        assert bool(lib.h_is_prime(int(n))) == sympy.isprime(int(n)), n


@pytest.mark.parametrize("bits,log_n", [(36, 12), (50, 13), (50, 14), (20, 13)])
def test_prime_search_matches_the_oracle(lib, bits, log_n):
    """The library's Miller-Rabin search and the oracle's trial division pick
    the same chain of primes = 1 mod 2N below 2^bits."""
    step = 2 << log_n
    below_l = below_o = 1 << bits
    for _ in range(4):
        below_l = lib.h_prime_below(below_l, step)
        below_o = O.prev_prime_1mod(below_o, step)
        assert below_l == below_o and below_l % step == 1


def test_roots_tables_and_montgomery(lib):
    p, log_n = 1125899906826241, 13
    n = 1 << log_n
    psi = lib.h_root_2n(p, n)
    assert pow(psi, n, p) == p - 1 and pow(psi, 2 * n, p) == 1
    t = 1032193
    z = lib.h_smallest_root(t, n)
    assert z == O.smallest_root(t, n) == 94
    fwd, fwd_s, inv = (np.zeros(n, np.uint64) for _ in range(3))
    lib.h_tables(p, psi, log_n, fwd.ctypes.data, fwd_s.ctypes.data, inv.ctypes.data)
    for k in (0, 1, 2, 3, 1000, n - 1):
        r = int(format(k, f"0{log_n}b")[::-1], 2)
        assert int(fwd[k]) == pow(psi, r, p) and int(inv[k]) == pow(psi, -r, p)
        assert int(fwd_s[k]) == (int(fwd[k]) << 64) // p
    ni = lib.h_mont_neg_inv(p)
    assert (p * ni + 1) % (1 << 64) == 0


def test_multiword_helpers(lib):
    rng = np.random.default_rng(6)
    for _ in range(50):
        na = int(rng.integers(1, 6))
        a = rng.integers(0, 2**63, na, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, na, dtype=np.uint64)
        m = int(rng.integers(2, 2**62))
        A = sum(int(v) << (64 * i) for i, v in enumerate(a))
        prod, quot = np.zeros(na + 1, np.uint64), np.zeros(na, np.uint64)
        rem, mod = ctypes.c_uint64(), ctypes.c_uint64()
        npw = lib.h_big(a.ctypes.data, na, m, prod.ctypes.data, quot.ctypes.data, ctypes.byref(rem), ctypes.byref(mod))
        assert sum(int(v) << (64 * i) for i, v in enumerate(prod[:npw])) == A * m
        assert sum(int(v) << (64 * i) for i, v in enumerate(quot)) == A // m
        assert rem.value == A % m and mod.value == A % m
