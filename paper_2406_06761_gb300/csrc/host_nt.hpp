// host_nt.hpp -- host-side number theory of the library: primes, roots of
// unity, NTT tables and the CRT constants of BFV/RNS (Sec. 2, Sec. 7).
#pragma once
#include <cstdint>
#include <vector>

namespace wally {

typedef unsigned __int128 u128;

uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t m);
uint64_t powmod_h(uint64_t a, uint64_t e, uint64_t m);
uint64_t invmod_h(uint64_t a, uint64_t p);  // p prime

// Deterministic Miller-Rabin for 64-bit integers (bases 2..37).
bool is_prime_u64(uint64_t n);
// Largest prime p < below with p = 1 (mod step); 0 if none.
uint64_t prime_1mod_below(uint64_t below, uint64_t step);
// A primitive 2N-th root of unity mod prime p = 1 mod 2N, from a generator
// of the multiplicative group (found by testing p-1's prime factors).
uint64_t root_2n(uint64_t p, uint32_t n);
// The slot root: the smallest x >= 2 with x^N = -1 (mod t).
uint64_t smallest_root_2n(uint64_t t, uint32_t n);
// floor(w * 2^64 / p)
inline uint64_t shoup_of(uint64_t w, uint64_t p) { return (uint64_t)(((u128)w << 64) / p); }
// -p^-1 mod 2^64 (p odd) by Newton iteration.
uint64_t mont_neg_inv(uint64_t p);

// Tables of one modulus: fwd[k] = psi^brv(k), inv[k] = psi^-brv(k), with
// Shoup companions.
struct NttTables {
    std::vector<uint64_t> fwd, fwd_s, inv, inv_s;
};
NttTables make_tables(uint64_t p, uint64_t psi, uint32_t log_n);

// Multi-precision helpers for Q = prod q_i (little-endian 64-bit limbs).
std::vector<uint64_t> big_mul_small(const std::vector<uint64_t> &a, uint64_t b);
std::vector<uint64_t> big_div_small(const std::vector<uint64_t> &a, uint64_t b, uint64_t *rem);
uint64_t big_mod_small(const std::vector<uint64_t> &a, uint64_t m);

}  // namespace wally
