// common.cuh -- device-side building blocks of the Wally GB300 library:
// RNS modular arithmetic on 64-bit residues (primes below 2^61) and the
// negacyclic NTT of one polynomial held in shared memory by one CTA.
//
// Modular arithmetic follows published methods:
//  - Shoup's precomputed-quotient multiplication for constant operands
//    (twiddles, P^-1, Delta): w' = floor(w * 2^64 / p), q = hi64(x * w'),
//    r = x*w - q*p in [0, 2p) for any x < 2^64.
//  - Montgomery reduction (Montgomery 1985) with R = 2^64 for variable
//    products: operands stored pre-multiplied by R (keys, plaintexts), a
//    128-bit sum T < p * 2^64 reduces to T * R^-1 mod p with one REDC.  Lazy
//    sums of up to 2^12 products of residues < p (Sec. 7 "lazy reduction" in
//    sequential plaintext-ciphertext products) stay below that bound.
//  - Harvey's lazy butterflies (Harvey 2014, the NTT the paper's library uses,
//    Sec. 7), with a Shoup quotient taken from the three high 32x32 partial
//    products only (short by at most 2, so the product lies in [0, 4p)):
//    forward Cooley-Tukey values in [0, 8p), inverse Gentleman-Sande values in
//    [0, 4p).  With p < 2^50 every value stays below 2^53.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef uint64_t u64;
typedef unsigned int u32;

#ifndef WALLY_MAX_LIMBS
#define WALLY_MAX_LIMBS 8
#endif
#define WALLY_MAX_MODS (WALLY_MAX_LIMBS + 2)

// A twiddle factor w with its Shoup companion w' = floor(w * 2^64 / p).
struct __align__(16) Tw {
    u64 w, ws;
};

// One RNS modulus with its NTT tables (device pointers, N entries each):
// fwd[k] = psi^brv(k), inv[k] = psi^-brv(k), brv = bit reversal on log2 N bits.
struct Mod {
    u64 p, two_p, four_p;
    u64 np;            // 2^64 - p
    u64 mont_neg_inv;  // -p^-1 mod 2^64
    u64 r2;            // 2^128 mod p
    u64 n_inv, n_inv_s;
    const Tw *fwd, *inv;
    // The twiddles of the last radix-16 pass (stages log2 N - 4 .. log2 N - 1)
    // reordered k-major: entry k * N/16 + g is the k-th twiddle of group g
    // (k = 2^st - 1 + block for stage st), so that consecutive groups read
    // consecutive entries.
    const Tw *fwd_last, *inv_last;
};

// Everything a kernel needs about the parameter set (kept in device memory).
// Modulus index j: 0..L-1 ciphertext primes q_j, L = P, L+1 = t.
struct DevParams {
    int log_n, n, L;
    u32 d, d_pad, g, h;
    Mod m[WALLY_MAX_MODS];
    u64 pinv[WALLY_MAX_LIMBS], pinv_s[WALLY_MAX_LIMBS];    // P^-1 mod q_j
    u64 pmodq[WALLY_MAX_LIMBS], pmodq_s[WALLY_MAX_LIMBS];  // P mod q_j
    u64 delta[WALLY_MAX_LIMBS], delta_s[WALLY_MAX_LIMBS];  // [floor(Q/t)]_{q_j}
    u64 theta[WALLY_MAX_LIMBS], theta_s[WALLY_MAX_LIMBS];  // [(Q/q_j)^-1]_{q_j}
    u64 rs_inv[WALLY_MAX_LIMBS][WALLY_MAX_LIMBS];             // q_i^-1 mod q_j (response switch)
    u64 rs_inv_s[WALLY_MAX_LIMBS][WALLY_MAX_LIMBS];
    const u32 *slot_pos;      // [N] NTT position (mod t) of slot s
    const DevParams *self;    // device copy of this block (kernels read it there)
    // launch shape (host side only; no kernel reads these): dynamic shared
    // memory of the transform kernels (0 = what they need; more caps the CTAs
    // an SM holds) and resident CTAs per SM of the multiply-accumulate
    u32 ntt_smem, mac_ctas_per_sm;
    // transform core of the key-switch kernels: 0 = shared-memory radix-16
    // passes (three CTAs an SM), 1 = register-blocked passes (two CTAs an SM)
    u32 ks_core;
    // multiply-accumulate: 0 = whole tiles, one buffer; 1 = half tiles,
    // double-buffered with asynchronous copies
    u32 mac_halves;
};

__device__ __forceinline__ u64 csub(u64 x, u64 m) { return x >= m ? x - m : x; }

// x * w mod p up to one p: result in [0, 2p).  Requires p < 2^63.
__device__ __forceinline__ u64 shoup_mul(u64 x, u64 w, u64 ws, u64 p)
{
    u64 q = __umul64hi(x, ws);
    return x * w - q * p;
}

// (hi * 2^64 + lo) * 2^-64 mod p, for hi < p; canonical result.
__device__ __forceinline__ u64 mont_redc(u64 hi, u64 lo, const Mod &md)
{
    u64 m = lo * md.mont_neg_inv;
    u64 mh = __umul64hi(m, md.p);
    return csub(hi + mh + (lo != 0 ? 1ull : 0ull), md.p);
}

// a * b * 2^-64 mod p for a * b < p * 2^64 (e.g. a < 4p, b < p).
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, const Mod &md)
{
    return mont_redc(__umul64hi(a, b), a * b, md);
}

// Plain a * b mod p for canonical a, b (two REDCs).
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const Mod &md)
{
    return mont_mul(mont_mul(a, b, md), md.r2, md);
}

// 128-bit multiply-accumulate: (hi:lo) += a * b.
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

// Sums of up to 32 products of operands below 2^56, exactly: each operand split into 28-bit limbs a = a1 2^28 + a0,
// the four 32x32 -> 64-bit limb products accumulated in three columns of
// weight 1, 2^28 and 2^56 (each column stays below 2^63), combined into the
// 128-bit sum once at the end.  Four 32-bit multiply-adds a product instead
// of a 64x64 -> 128-bit multiply-accumulate.
struct Acc28 {
    u64 c0, c1, c2;
};

__device__ __forceinline__ void split28(u64 x, u32 &x0, u32 &x1)
{
    x0 = (u32)x & 0x0FFFFFFFu;
    x1 = (u32)(x >> 28);
}

// c0 + c1 2^28 + c2 2^56 as (hi, lo).
__device__ __forceinline__ void acc28_sum(const Acc28 &a, u64 &hi, u64 &lo)
{
    const u64 t1 = a.c1 << 28, t1h = a.c1 >> 36, t2 = a.c2 << 56, t2h = a.c2 >> 8;
    asm("add.cc.u64 %0, %2, %3;\n\t"
        "addc.u64 %1, %4, 0;\n\t"
        "add.cc.u64 %0, %0, %5;\n\t"
        "addc.u64 %1, %1, %6;"
        : "=l"(lo), "=l"(hi)
        : "l"(a.c0), "l"(t1), "l"(t1h), "l"(t2), "l"(t2h));
}

__device__ __forceinline__ void acc28_zero(Acc28 &a) { a.c0 = a.c1 = a.c2 = 0; }

__device__ __forceinline__ void mac28(Acc28 &acc, u32 a0, u32 a1, u32 b0, u32 b1)
{
    acc.c0 += (u64)a0 * b0;
    acc.c1 += (u64)a0 * b1;
    acc.c1 += (u64)a1 * b0;
    acc.c2 += (u64)a1 * b1;
}

// acc += a * b with a given in limbs and b whole.
__device__ __forceinline__ void mac28(Acc28 &acc, u32 a0, u32 a1, u64 b)
{
    u32 b0, b1;
    split28(b, b0, b1);
    mac28(acc, a0, a1, b0, b1);
}

// The accumulated sum times 2^-64 mod p (Montgomery reduction); the sum's
// high word must be below p.
__device__ __forceinline__ u64 acc28_redc(const Acc28 &a, const Mod &md)
{
    u64 hi, lo;
    acc28_sum(a, hi, lo);
    return mont_redc(hi, lo, md);
}

__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 p) { return csub(a + b, p); }
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 p) { return a >= b ? a - b : a + p - b; }

// --------------------------------------------------------------------------- NTT
// One CTA of N/32 threads transforms one polynomial held in shared memory.
// Shared memory holds the N words with an XOR swizzle inside each 16-word row
// (spos), so that every access pattern below is free of bank conflicts
// without padding.
//
// Passes: a remainder pass of R = log2 N mod 4 stages first (if any), then
// radix-16 passes of 4 stages.  A pass loads groups of 2^R elements into
// registers, runs its stages, and stores them back.  Every radix-16 pass runs
// the same code with a run-time first stage S0, which keeps the instruction
// footprint small.  Stage s uses twiddle entries [2^s, 2^(s+1)); those of all
// passes but the last (entries below 2^(log2 N - 4), at most 16 KB) are
// copied into a shared cache at the start of each transform, the last pass
// reads its group's 15 twiddles from global memory before the group's data.

__host__ __device__ constexpr int smem_words(int n) { return n; }
__device__ __forceinline__ int spos(int x) { return x ^ ((x >> 4) & 15); }

template <int LOGN>
struct NttShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 32;           // threads per CTA
    static constexpr int RR = LOGN % 4;        // stages of the remainder pass
    static constexpr int TW_CACHE = 1 << (LOGN - 4);
    // register budget: three CTAs share an SM at N = 8192 (85 registers)
    static constexpr int MIN_BLOCKS = (LOGN == 12) ? 4 : (LOGN == 13 ? 3 : 1);
};

// Shared-memory words of a transform kernel: the polynomial and the cache.
template <int LOGN>
__host__ __device__ constexpr int ntt_smem_words()
{
    return smem_words(1 << LOGN) + 2 * NttShape<LOGN>::TW_CACHE;
}

// x * w mod p up to 3p: a value in [0, 4p) for any x < 2^64.  The quotient
// x * w' / 2^64 is built from x1*s1, hi(x1*s0) and hi(x0*s1) (x = x1:x0,
// w' = s1:s0 in 32-bit halves); the dropped terms add less than 3 * 2^32 to
// the middle column, so it is short by at most 2.  np = 2^64 - p.
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 ws, u64 np)
{
    const u32 x0 = (u32)x, x1 = (u32)(x >> 32), s0 = (u32)ws, s1 = (u32)(ws >> 32);
    const u64 q = (u64)x1 * s1 + __umulhi(x1, s0) + __umulhi(x0, s1);
    return x * w + q * np;
}

// Forward butterfly, values in [0, 8p).
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, u64 w, u64 ws, u64 np, u64 four_p)
{
    u64 x = csub(X, four_p);
    u64 t = shoup_lazy(Y, w, ws, np);
    X = x + t;
    Y = x - t + four_p;
}

// Inverse butterfly, values in [0, 4p).
__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, u64 w, u64 ws, u64 np, u64 four_p)
{
    u64 x = X, y = Y;
    X = csub(x + y, four_p);
    Y = shoup_lazy(x - y + four_p, w, ws, np);
}

// Copy table entries [0, TW_CACHE) into the shared cache.
template <int LOGN>
__device__ __forceinline__ void load_tw_cache(Tw *dst, const Tw *__restrict__ src)
{
    constexpr int C = NttShape<LOGN>::TW_CACHE, T = NttShape<LOGN>::T;
    for (int i = threadIdx.x; i < C; i += T) dst[i] = src[i];
}

// Stage ST (0-based inside a pass of R stages) on the 2^R registers v of a
// group; tw holds the group's twiddles in stage order (1, 2, 4, ... entries).
// Stage ST pairs registers 2^(R-1-ST) apart; block b uses tw[2^ST - 1 + b].
template <int R, int ST, bool FWD>
__device__ __forceinline__ void group_stage(u64 *v, const Tw *tw, u64 p, u64 two_p)
{
    constexpr int HD = 1 << (R - 1 - ST);
    constexpr int NB = 1 << ST;
#pragma unroll
    for (int blk = 0; blk < NB; blk++) {
        const Tw t = tw[(NB - 1) + blk];
#pragma unroll
        for (int j = 0; j < HD; j++) {
            if (FWD) ct_bfly(v[blk * 2 * HD + j], v[blk * 2 * HD + j + HD], t.w, t.ws, p, two_p);
            else gs_bfly(v[blk * 2 * HD + j], v[blk * 2 * HD + j + HD], t.w, t.ws, p, two_p);
        }
    }
}

template <int R, int ST, bool FWD>
__device__ __forceinline__ void group_stages(u64 *v, const Tw *tw, u64 p, u64 two_p)
{
    if constexpr (FWD) {
        if constexpr (ST < R) {
            group_stage<R, ST, true>(v, tw, p, two_p);
            group_stages<R, ST + 1, true>(v, tw, p, two_p);
        }
    } else {
        if constexpr (ST >= 0) {
            group_stage<R, ST, false>(v, tw, p, two_p);
            group_stages<R, ST - 1, false>(v, tw, p, two_p);
        }
    }
}

// One pass: stages S0 .. S0+R-1 (forward) or in reverse order (inverse) on
// all groups.  Group gi covers elements base + (k << BLO), k < 2^R, with
// BLO = LOGN - R - S0 and base = (hi << (BLO + R)) | lo, hi = gi >> BLO,
// lo = gi mod 2^BLO; the twiddle of its block at stage S0+st is entry
// 2^(S0+st) + ((hi << st) | block), taken from `tws` (shared cache or global
// table: a generic pointer).
template <int LOGN, int R, bool FWD>
__device__ __forceinline__ void ntt_pass(u64 *sm, int S0, const Tw *tws, u64 p, u64 two_p)
{
    constexpr int T = NttShape<LOGN>::T;
    constexpr int G = 1 << R;
    constexpr int NG = 32 / G;
    const int BLO = LOGN - R - S0;
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int u = 0; u < NG; u++) {
        const int gi = tid + T * u;
        const int lo = gi & ((1 << BLO) - 1);
        const int hi = gi >> BLO;
        const int base = (hi << (BLO + R)) | lo;
        Tw tw[G - 1];
#pragma unroll
        for (int st = 0, k = 0; st < R; st++)
#pragma unroll
            for (int blk = 0; blk < (1 << st); blk++, k++) tw[k] = tws[(1 << (S0 + st)) + ((hi << st) | blk)];
        u64 v[G];
#pragma unroll
        for (int k = 0; k < G; k++) v[k] = sm[spos(base + (k << BLO))];
        if constexpr (FWD) group_stages<R, 0, true>(v, tw, p, two_p);
        else group_stages<R, R - 1, false>(v, tw, p, two_p);
#pragma unroll
        for (int k = 0; k < G; k++) sm[spos(base + (k << BLO))] = v[k];
    }
}

// Forward negacyclic NTT in place: natural-order coefficients (any values
// < 8p) -> evaluations at psi^(2*brv(i)+1) in bit-reversed position i, values
// in [0, 8p).  cache: TW_CACHE shared entries (reloaded here).  Starts and
// ends with __syncthreads().
template <int LOGN>
__device__ __forceinline__ void ntt_fwd(u64 *sm, Tw *cache, const Mod &md)
{
    using S = NttShape<LOGN>;
    const u64 p = md.np, two_p = md.four_p;  // the butterflies take (2^64 - p, 4p)
    __syncthreads();
    load_tw_cache<LOGN>(cache, md.fwd);
    __syncthreads();
    if constexpr (S::RR > 0) {
        ntt_pass<LOGN, S::RR, true>(sm, 0, cache, p, two_p);
        __syncthreads();
    }
#pragma unroll 1
    for (int s0 = S::RR; s0 < LOGN - 4; s0 += 4) {
        ntt_pass<LOGN, 4, true>(sm, s0, cache, p, two_p);
        __syncthreads();
    }
    ntt_pass<LOGN, 4, true>(sm, LOGN - 4, md.fwd, p, two_p);
    __syncthreads();
}

// Inverse: bit-reversed evaluations (values < 4p) -> natural-order
// coefficients times N (values in [0, 4p)); callers scale by N^-1 with
// inv_finish().  Starts and ends with __syncthreads().
template <int LOGN>
__device__ __forceinline__ void ntt_inv(u64 *sm, Tw *cache, const Mod &md)
{
    using S = NttShape<LOGN>;
    const u64 p = md.np, two_p = md.four_p;  // the butterflies take (2^64 - p, 4p)
    __syncthreads();
    load_tw_cache<LOGN>(cache, md.inv);
    ntt_pass<LOGN, 4, false>(sm, LOGN - 4, md.inv, p, two_p);
    __syncthreads();
#pragma unroll 1
    for (int s0 = LOGN - 8; s0 >= S::RR; s0 -= 4) {
        ntt_pass<LOGN, 4, false>(sm, s0, cache, p, two_p);
        __syncthreads();
    }
    if constexpr (S::RR > 0) {
        ntt_pass<LOGN, S::RR, false>(sm, 0, cache, p, two_p);
        __syncthreads();
    }
}

// [0, 8p) -> [0, p)
__device__ __forceinline__ u64 fwd_finish(u64 x, const Mod &md) { return csub(csub(csub(x, md.four_p), md.two_p), md.p); }
// N^-1 scaling after ntt_inv, canonical result.
__device__ __forceinline__ u64 inv_finish(u64 x, const Mod &md) { return csub(shoup_mul(x, md.n_inv, md.n_inv_s, md.p), md.p); }

__device__ __forceinline__ u32 brv(u32 x, int log_n) { return __brev(x) >> (32 - log_n); }

// Position, in the bit-reversed NTT order, of the evaluation that the Galois
// automorphism sigma_k moves to position j: (sigma_k a)(w) = a(w^k), and
// position j holds the evaluation at psi^(2 brv(j) + 1).
__device__ __forceinline__ u32 galois_src(u32 j, u64 k, int log_n)
{
    const u32 mask2n = (2u << log_n) - 1;
    u32 e = (u32)(((u64)(2 * brv(j, log_n) + 1) * k) & mask2n);
    return brv((e - 1) >> 1, log_n);
}

// --------------------------------------------------------------------------- element IO
// Elementwise sweeps use pairs: thread t owns elements 2(t + T*u) and
// 2(t + T*u) + 1 for u < 16, so that global accesses are 16-byte and
// coalesced.  Both elements of a pair sit in the same 16-word smem row, at
// spos(e) and spos(e) ^ 1.
template <int LOGN>
__device__ __forceinline__ int pair_elem(int u)
{
    return 2 * ((int)threadIdx.x + NttShape<LOGN>::T * u);
}

__device__ __forceinline__ ulonglong2 ldg2(const u64 *p) { return __ldg(reinterpret_cast<const ulonglong2 *>(p)); }

// L2 policy for data read once and not again soon (the keys of a key
// switch): evicted first, so that the data a kernel parks in global memory
// and reads back (transformed digits, key products) stays in L2.
__device__ __forceinline__ u64 l2_evict_first_policy()
{
    u64 pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 16-byte read-only load under an L2 policy.
__device__ __forceinline__ ulonglong2 ldg2_hint(const u64 *p, u64 pol)
{
    ulonglong2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(v.x), "=l"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, u64 a, u64 b) { *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a, b); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// The same copy of data read once (an L2 eviction policy, as ldg2_hint).
__device__ __forceinline__ void cp_async16_hint(void *dst, const void *src, u64 pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most PENDING of this thread's committed copy groups are
// still in flight.
template <int PENDING>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2 by the
// copy engine of the SM (TMA), without waiting: the data a CTA needs only
// after its transforms is requested at its start.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Global polynomial -> shared buffer (any values), 16-byte loads.  COHERENT:
// the data was written earlier by this kernel (read through the coherent
// path, not the read-only cache).
template <int LOGN, bool COHERENT = false>
__device__ __forceinline__ void poly_load(u64 *sm, const u64 *g)
{
#pragma unroll 4
    for (int u = 0; u < 16; u++) {
        const int e = pair_elem<LOGN>(u);
        const ulonglong2 v = COHERENT ? ld2(g + e) : ldg2(g + e);
        const int s = spos(e);
        sm[s] = v.x;
        sm[s ^ 1] = v.y;
    }
}
