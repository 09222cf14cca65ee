// host_nt.cpp -- number theory for parameter set-up (library side).
#include "host_nt.hpp"

namespace wally {

uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }

uint64_t powmod_h(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod_h(r, a, m);
        a = mulmod_h(a, a, m);
    }
    return r;
}

uint64_t invmod_h(uint64_t a, uint64_t p) { return powmod_h(a, p - 2, p); }

bool is_prime_u64(uint64_t n)
{
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t s : small) {
        if (n == s) return true;
        if (n % s == 0) return false;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (uint64_t a : small) {
        uint64_t x = powmod_h(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; i++) {
            x = mulmod_h(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

uint64_t prime_1mod_below(uint64_t below, uint64_t step)
{
    if (below <= step + 1) return 0;
    uint64_t c = below - 1 - ((below - 1 - 1) % step);  // largest value = 1 mod step that is <= below-1
    if (c >= below) c -= step;
    for (; c > step; c -= step)
        if (is_prime_u64(c)) return c;
    return 0;
}

static std::vector<uint64_t> prime_factors(uint64_t n)
{
    std::vector<uint64_t> f;
    for (uint64_t d = 2; d * d <= n; d += (d == 2 ? 1 : 2)) {
        if (n % d == 0) {
            f.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) f.push_back(n);
    return f;
}

uint64_t root_2n(uint64_t p, uint32_t n)
{
    std::vector<uint64_t> fs = prime_factors(p - 1);
    for (uint64_t g = 2; g < p; g++) {
        bool gen = true;
        for (uint64_t f : fs)
            if (powmod_h(g, (p - 1) / f, p) == 1) { gen = false; break; }
        if (gen) return powmod_h(g, (p - 1) / (2 * (uint64_t)n), p);
    }
    return 0;
}

uint64_t smallest_root_2n(uint64_t t, uint32_t n)
{
    for (uint64_t x = 2; x < t; x++)
        if (powmod_h(x, n, t) == t - 1) return x;
    return 0;
}

uint64_t mont_neg_inv(uint64_t p)
{
    uint64_t inv = p;  // correct to 3 bits for odd p
    for (int i = 0; i < 6; i++) inv *= 2 - p * inv;
    return (uint64_t)0 - inv;
}

static uint32_t bit_reverse(uint32_t x, uint32_t bits)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

NttTables make_tables(uint64_t p, uint64_t psi, uint32_t log_n)
{
    uint32_t n = 1u << log_n;
    NttTables t;
    t.fwd.resize(n);
    t.fwd_s.resize(n);
    t.inv.resize(n);
    t.inv_s.resize(n);
    std::vector<uint64_t> pw(n), ipw(n);
    uint64_t psi_inv = invmod_h(psi, p);
    pw[0] = ipw[0] = 1;
    for (uint32_t i = 1; i < n; i++) {
        pw[i] = mulmod_h(pw[i - 1], psi, p);
        ipw[i] = mulmod_h(ipw[i - 1], psi_inv, p);
    }
    for (uint32_t k = 0; k < n; k++) {
        uint32_t r = bit_reverse(k, log_n);
        t.fwd[k] = pw[r];
        t.inv[k] = ipw[r];
        t.fwd_s[k] = shoup_of(t.fwd[k], p);
        t.inv_s[k] = shoup_of(t.inv[k], p);
    }
    return t;
}

std::vector<uint64_t> big_mul_small(const std::vector<uint64_t> &a, uint64_t b)
{
    std::vector<uint64_t> r(a.size() + 1, 0);
    u128 carry = 0;
    for (size_t i = 0; i < a.size(); i++) {
        u128 v = (u128)a[i] * b + carry;
        r[i] = (uint64_t)v;
        carry = v >> 64;
    }
    r[a.size()] = (uint64_t)carry;
    while (r.size() > 1 && r.back() == 0) r.pop_back();
    return r;
}

std::vector<uint64_t> big_div_small(const std::vector<uint64_t> &a, uint64_t b, uint64_t *rem)
{
    std::vector<uint64_t> q(a.size(), 0);
    u128 r = 0;
    for (size_t i = a.size(); i-- > 0;) {
        u128 cur = (r << 64) | a[i];
        q[i] = (uint64_t)(cur / b);
        r = cur % b;
    }
    if (rem) *rem = (uint64_t)r;
    while (q.size() > 1 && q.back() == 0) q.pop_back();
    return q;
}

uint64_t big_mod_small(const std::vector<uint64_t> &a, uint64_t m)
{
    uint64_t r;
    big_div_small(a, m, &r);
    return r;
}

}  // namespace wally
