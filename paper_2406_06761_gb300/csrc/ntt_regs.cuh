// ntt_regs.cuh -- register-blocked negacyclic NTT of one polynomial per CTA.
//
// One CTA of T = N/V threads; every thread holds V coefficients in
// registers.  A transform is a few passes, each a run of R butterfly stages
// on the thread's own registers, with the polynomial exchanged through an
// XOR-swizzled shared buffer of N words (free of bank conflicts) between
// passes.  In a pass of R stages starting at stage S0 the thread holds
// V / 2^R groups of 2^R elements spaced D = 2^(log2 N - S0 - R) apart:
// register k = jj 2^R + m holds element
//     ((g >> log D) << (log D + R)) | (g mod D) | (m << log D),  g = t + T jj.
// The first pass therefore reads natural-order coefficients with a warp
// covering 256 contiguous bytes per register, and the last pass (D = 1)
// leaves each group of 2^R contiguous bit-reversed evaluations in a thread
// (16-byte accesses).  Pointwise work between transforms runs in the last
// pass's layout, coefficient-domain work in the first pass's.
//
// Twiddles: table entries [2^s, 2^(s+1)) serve stage s.  Entries below
// 2^CACHE_LOG are read from a shared copy (loaded once per CTA and
// direction), the rest from the global table through the read-only cache.
//
// Arithmetic (Harvey's lazy butterflies, which Sec. 7 of the paper names):
// the forward Cooley-Tukey butterfly X' = X + wY, Y' = X + 4p - wY with wY
// in [0, 4p) from a Shoup product does no conditional subtraction, so values
// grow by 4p a stage: inputs below B leave the transform below
// B + 4p log2 N (below 2^57 for p < 2^50 and B < 8p); the Shoup product
// accepts any 64-bit input.  The inverse Gentleman-Sande butterfly keeps its
// values in [0, 4p) (one conditional subtraction on the sum).
//
// The Shoup product w*y mod p for a twiddle w with w' = floor(w 2^64 / p):
// the quotient estimate q = y1*s1 + hi(y1*s0) + hi(y0*s1) (y = y1:y0,
// w' = s1:s0 in 32-bit halves) is short of floor(y w' / 2^64) by at most 2,
// and y*w - q*p (computed mod 2^64 as y*w + q*(2^64 - p)) lies in [0, 4p).
// It is written out in 32-bit multiply-adds: two mul.hi and one mad.wide for
// q, two mad.wide and four mad.lo for the result -- the multiplier issue
// cost that bounds every transform.
#pragma once
#include "common.cuh"

namespace wally {

__device__ __forceinline__ u64 shoup_mul32(u64 y, u64 w, u64 ws, u64 np)
{
    u64 t;
    asm("{\n\t"
        ".reg .u32 y0, y1, s0, s1, w0, w1, n0, n1, a, b, c0, c1, q0, q1, tl, th;\n\t"
        ".reg .u64 q, c;\n\t"
        "mov.b64 {y0, y1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {s0, s1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.hi.u32 a, y1, s0;\n\t"
        "mul.hi.u32 b, y0, s1;\n\t"
        "add.cc.u32 c0, a, b;\n\t"
        "addc.u32 c1, 0, 0;\n\t"
        "mov.b64 c, {c0, c1};\n\t"
        "mad.wide.u32 q, y1, s1, c;\n\t"
        "mov.b64 {q0, q1}, q;\n\t"
        "mul.wide.u32 %0, y0, w0;\n\t"
        "mad.wide.u32 %0, q0, n0, %0;\n\t"
        "mov.b64 {tl, th}, %0;\n\t"
        "mad.lo.u32 th, y0, w1, th;\n\t"
        "mad.lo.u32 th, y1, w0, th;\n\t"
        "mad.lo.u32 th, q0, n1, th;\n\t"
        "mad.lo.u32 th, q1, n0, th;\n\t"
        "mov.b64 %0, {tl, th};\n\t"
        "}"
        : "=l"(t)
        : "l"(y), "l"(w), "l"(ws), "l"(np));
    return t;
}

// Forward butterfly without reduction: X' = X + wY, Y' = X + 4p - wY.
__device__ __forceinline__ void ct_grow(u64 &X, u64 &Y, u64 w, u64 ws, u64 np, u64 four_p)
{
    const u64 x = X;
    const u64 m = shoup_mul32(Y, w, ws, np);
    X = x + m;
    Y = x + four_p - m;
}

// Inverse butterfly, inputs and outputs in [0, 4p).
__device__ __forceinline__ void gs_keep(u64 &X, u64 &Y, u64 w, u64 ws, u64 np, u64 four_p)
{
    const u64 x = X, y = Y;
    X = csub(x + y, four_p);
    Y = shoup_mul32(x + four_p - y, w, ws, np);
}

// Pass plans, swizzles and launch shapes per (log2 N, V).  Every plan's
// passes and swizzle were checked on the host: each layout is a bijection
// onto [0, N) and every half-warp's 64-bit shared accesses of every layout
// fall in 16 distinct bank pairs.  With 32 coefficients a thread the
// transform needs about 128 registers, so two CTAs share an SM; twiddles
// past the first 32 entries come from global memory (a shared copy of more
// of the table costs more to load than it saves in a one-transform CTA).
template <int LOGN, int V>
struct NttV;

#define WALLY_NTT_PLAN(LG, VV, NPASS, R0, R1, R2, R3_, SA, SB, MB, CL)                          \
    template <>                                                                             \
    struct NttV<LG, VV> {                                                                   \
        static constexpr int LOGN = LG, N = 1 << LG, V = VV, T = N / VV, NP = NPASS;        \
        static constexpr int MIN_BLOCKS = MB, CACHE_LOG = CL;                               \
        static constexpr int SWZ_A = SA, SWZ_B = SB;                                        \
        __host__ __device__ static constexpr int R(int p)                                   \
        {                                                                                   \
            return p == 0 ? R0 : p == 1 ? R1 : p == 2 ? R2 : R3_;                           \
        }                                                                                   \
    };

//             logN  V  passes  R0 R1 R2 R3  swizzle  CTAs/SM  cached entries (log2)
WALLY_NTT_PLAN(12, 32, 3, 5, 4, 3, 0, 3, 7, 4, 5)
WALLY_NTT_PLAN(13, 32, 3, 5, 5, 3, 0, 3, 8, 2, 5)
WALLY_NTT_PLAN(14, 32, 3, 5, 5, 4, 0, 4, -1, 1, 5)
#undef WALLY_NTT_PLAN

template <class P>
__host__ __device__ constexpr int pass_start(int p)
{
    int s = 0;
    for (int i = 0; i < p; i++) s += P::R(i);
    return s;
}

// Element held in register k by thread t during pass p.
template <class P, int PASS>
__device__ __forceinline__ int elem_of(int t, int k)
{
    constexpr int R = P::R(PASS);
    constexpr int LD = P::LOGN - pass_start<P>(PASS) - R;
    const int jj = k >> R, m = k & ((1 << R) - 1);
    const int g = t + P::T * jj;
    return ((g >> LD) << (LD + R)) | (g & ((1 << LD) - 1)) | (m << LD);
}

// Shared-memory word of element e.
template <class P>
__device__ __forceinline__ int phys(int e)
{
    int x = e ^ ((e >> P::SWZ_A) & 15);
    if constexpr (P::SWZ_B >= 0) x ^= ((e >> P::SWZ_B) & 1) << 3;
    return x;
}

template <bool GLOBAL>
__device__ __forceinline__ Tw tw_load(const Tw *p)
{
    if constexpr (GLOBAL) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        return Tw{v.x, v.y};
    } else {
        return *p;
    }
}

// Stage LS of a run of R stages on the 2^R registers v[0 ..]: pairs
// 2^(R-1-LS) apart, block b of the stage uses twiddle tb[b].
template <int R, int LS, bool FWD, bool GLOBAL>
__device__ __forceinline__ void run_stage(u64 *v, const Tw *tb, u64 np, u64 four_p)
{
    constexpr int H = 1 << (R - 1 - LS);
#pragma unroll
    for (int b = 0; b < (1 << LS); b++) {
        const Tw t = tw_load<GLOBAL>(tb + b);
#pragma unroll
        for (int j = 0; j < H; j++) {
            if constexpr (FWD) ct_grow(v[b * 2 * H + j], v[b * 2 * H + j + H], t.w, t.ws, np, four_p);
            else gs_keep(v[b * 2 * H + j], v[b * 2 * H + j + H], t.w, t.ws, np, four_p);
        }
    }
}

// All R stages of one group (absolute stages S0 .. S0+R-1); stage S0+LS
// uses entries 2^(S0+LS) + (grp << LS) + block, from the shared copy when
// they lie below 2^CACHE_LOG.
template <class P, int S0, int R, int LS, bool FWD>
__device__ __forceinline__ void run_group(u64 *v, const Tw *cache, const Tw *tab, int grp, u64 np, u64 four_p)
{
    if constexpr (LS < R) {
        constexpr bool GL = (S0 + LS + 1) > P::CACHE_LOG;
        const Tw *tb = (GL ? tab : cache) + (1 << (S0 + LS)) + (grp << LS);
        if constexpr (FWD) {
            run_stage<R, LS, true, GL>(v, tb, np, four_p);
            run_group<P, S0, R, LS + 1, true>(v, cache, tab, grp, np, four_p);
        } else {
            run_group<P, S0, R, LS + 1, false>(v, cache, tab, grp, np, four_p);
            run_stage<R, LS, false, GL>(v, tb, np, four_p);
        }
    }
}

// The butterflies of pass PASS on all of the thread's groups.
template <class P, int PASS, bool FWD>
__device__ __forceinline__ void run_pass(u64 (&v)[P::V], const Tw *cache, const Tw *tab, u64 np, u64 four_p)
{
    constexpr int R = P::R(PASS), S0 = pass_start<P>(PASS);
    constexpr int LD = P::LOGN - S0 - R;
    const int t = threadIdx.x;
#pragma unroll
    for (int jj = 0; jj < (P::V >> R); jj++)
        run_group<P, S0, R, 0, FWD>(v + (jj << R), cache, tab, (t + P::T * jj) >> LD, np, four_p);
}

template <class P, int PASS>
__device__ __forceinline__ void sm_store(u64 *sm, const u64 (&v)[P::V])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k++) sm[phys<P>(elem_of<P, PASS>(t, k))] = v[k];
}

template <class P, int PASS>
__device__ __forceinline__ void sm_load(u64 (&v)[P::V], const u64 *sm)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k++) v[k] = sm[phys<P>(elem_of<P, PASS>(t, k))];
}

template <class P, int PASS>
__device__ __forceinline__ void fwd_from(u64 (&v)[P::V], u64 *sm, const Tw *cache, const Tw *tab, u64 np, u64 fp)
{
    if constexpr (PASS < P::NP) {
        if constexpr (PASS > 0) {
            sm_load<P, PASS>(v, sm);
        }
        run_pass<P, PASS, true>(v, cache, tab, np, fp);
        if constexpr (PASS + 1 < P::NP) {
            if constexpr (PASS == 0) __syncthreads();  // earlier users of sm are done
            sm_store<P, PASS>(sm, v);  // later passes store where they loaded: no barrier before
            __syncthreads();
            fwd_from<P, PASS + 1>(v, sm, cache, tab, np, fp);
        }
    }
}

template <class P, int PASS>
__device__ __forceinline__ void inv_from(u64 (&v)[P::V], u64 *sm, const Tw *cache, const Tw *tab, u64 np, u64 fp)
{
    if constexpr (PASS >= 0) {
        if constexpr (PASS < P::NP - 1) {
            sm_load<P, PASS>(v, sm);
        }
        run_pass<P, PASS, false>(v, cache, tab, np, fp);
        if constexpr (PASS > 0) {
            if constexpr (PASS == P::NP - 1) __syncthreads();
            sm_store<P, PASS>(sm, v);
            __syncthreads();
            inv_from<P, PASS - 1>(v, sm, cache, tab, np, fp);
        }
    }
}

// Forward negacyclic NTT.  v: natural-order coefficients in the first
// pass's layout, each below B; on return bit-reversed evaluations (position
// i = evaluation at psi^(2 brv(i) + 1)) in the last pass's layout, each
// below B + 4p log2 N.  cache: shared copy of the forward table's entries
// [0, 2^CACHE_LOG); tab: the global forward table.  sm: N words of shared
// memory; the first store into it is preceded by a barrier.
template <class P>
__device__ __forceinline__ void ntt_fwd_v(u64 (&v)[P::V], u64 *sm, const Tw *cache, const Tw *tab, const Mod &md)
{
    fwd_from<P, 0>(v, sm, cache, tab, md.np, md.four_p);
}

// Inverse: bit-reversed evaluations in the last pass's layout (values < 4p)
// -> natural coefficients times N in the first pass's layout (values < 4p).
// cache / tab: the inverse table.
template <class P>
__device__ __forceinline__ void ntt_inv_v(u64 (&v)[P::V], u64 *sm, const Tw *cache, const Tw *tab, const Mod &md)
{
    inv_from<P, P::NP - 1>(v, sm, cache, tab, md.np, md.four_p);
}

// Global <-> registers in the first pass's layout (coefficients).
template <class P, bool COHERENT = false>
__device__ __forceinline__ void gload_first(u64 (&v)[P::V], const u64 *g)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k++) {
        const int e = elem_of<P, 0>(t, k);
        v[k] = COHERENT ? g[e] : __ldg(g + e);
    }
}

template <class P>
__device__ __forceinline__ void gstore_first(u64 *g, const u64 (&v)[P::V])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k++) g[elem_of<P, 0>(t, k)] = v[k];
}

// Global <-> registers in the last pass's layout (evaluations): registers
// 2i, 2i+1 are adjacent elements.
template <class P, bool COHERENT = false>
__device__ __forceinline__ void gload_last(u64 (&v)[P::V], const u64 *g)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k += 2) {
        const u64 *a = g + elem_of<P, P::NP - 1>(t, k);
        const ulonglong2 x = COHERENT ? ld2(a) : ldg2(a);
        v[k] = x.x;
        v[k + 1] = x.y;
    }
}

template <class P>
__device__ __forceinline__ void gstore_last(u64 *g, const u64 (&v)[P::V])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < P::V; k += 2) st2(g + elem_of<P, P::NP - 1>(t, k), v[k], v[k + 1]);
}

template <class P>
__device__ __forceinline__ int elem_last(int t, int k)
{
    return elem_of<P, P::NP - 1>(t, k);
}

template <class P>
__device__ __forceinline__ void sm_store_last(u64 *sm, const u64 (&v)[P::V])
{
    sm_store<P, P::NP - 1>(sm, v);
}

// Shared copy of table entries [0, 2^CACHE_LOG) (all threads take part; the
// caller places a barrier before its first use).
template <class P>
__device__ __forceinline__ void load_tw_cache_v(Tw *dst, const Tw *src)
{
    constexpr int C = 1 << P::CACHE_LOG;
    const ulonglong2 *s = reinterpret_cast<const ulonglong2 *>(src);
    ulonglong2 *d = reinterpret_cast<ulonglong2 *>(dst);
    for (int i = threadIdx.x; i < C; i += P::T) d[i] = __ldg(s + i);
}

// ---------------------------------------------------------------------------
// The shared-memory transform core (common.cuh: the polynomial in a swizzled
// shared buffer, a remainder pass then radix-16 passes, each thread taking
// its groups of 2^R elements from the buffer) with this file's butterflies:
// the forward one without conditional subtractions (values grow by 4p a
// stage) and both with the Shoup product in 32-bit multiply-adds.  The
// twiddles of the passes served by the shared cache are read where they are
// used rather than preloaded into registers, which frees registers for the
// compiler to interleave a thread's two groups; the last pass (global table)
// still loads its group's 15 twiddles first.

template <int R, int ST, bool FWD, bool PRE>
__device__ __forceinline__ void sgroup_stage(u64 *v, const Tw *tw, const Tw *tws, int S0, int hi, u64 np, u64 fp)
{
    constexpr int HD = 1 << (R - 1 - ST);
    constexpr int NB = 1 << ST;
#pragma unroll
    for (int blk = 0; blk < NB; blk++) {
        const Tw t = PRE ? tw[(NB - 1) + blk] : tws[(1 << (S0 + ST)) + ((hi << ST) | blk)];
#pragma unroll
        for (int j = 0; j < HD; j++) {
            if constexpr (FWD) ct_grow(v[blk * 2 * HD + j], v[blk * 2 * HD + j + HD], t.w, t.ws, np, fp);
            else gs_keep(v[blk * 2 * HD + j], v[blk * 2 * HD + j + HD], t.w, t.ws, np, fp);
        }
    }
}

template <int R, int ST, bool FWD, bool PRE>
__device__ __forceinline__ void sgroup_stages(u64 *v, const Tw *tw, const Tw *tws, int S0, int hi, u64 np, u64 fp)
{
    if constexpr (FWD) {
        if constexpr (ST < R) {
            sgroup_stage<R, ST, true, PRE>(v, tw, tws, S0, hi, np, fp);
            sgroup_stages<R, ST + 1, true, PRE>(v, tw, tws, S0, hi, np, fp);
        }
    } else {
        if constexpr (ST >= 0) {
            sgroup_stage<R, ST, false, PRE>(v, tw, tws, S0, hi, np, fp);
            sgroup_stages<R, ST - 1, false, PRE>(v, tw, tws, S0, hi, np, fp);
        }
    }
}

// One pass of the shared-memory core (the group and twiddle indexing of
// common.cuh's ntt_pass).  PRE: the last radix-16 pass (S0 = log2 N - 4,
// one group per 16 contiguous elements), whose 15 twiddles a group are
// preloaded from the k-major table `tws` (Mod::fwd_last / inv_last):
// coalesced loads, a warp reading 32 consecutive entries at a time.
template <int LOGN, int R, bool FWD, bool PRE>
__device__ __forceinline__ void spass(u64 *sm, int S0, const Tw *tws, u64 np, u64 fp)
{
    static_assert(!PRE || R == 4, "the preloaded pass is the last radix-16 pass");
    constexpr int T = NttShape<LOGN>::T;
    constexpr int G = 1 << R;
    constexpr int NG = 32 / G;
    const int BLO = LOGN - R - S0;
    const int tid = threadIdx.x;
#pragma unroll 2
    for (int u = 0; u < NG; u++) {
        const int gi = tid + T * u;
        const int lo = gi & ((1 << BLO) - 1);
        const int hi = gi >> BLO;
        const int base = (hi << (BLO + R)) | lo;
        Tw tw[PRE ? G - 1 : 1];
        if constexpr (PRE) {
#pragma unroll
            for (int k = 0; k < G - 1; k++) tw[k] = tws[k * (1 << (LOGN - 4)) + hi];
        }
        u64 v[G];
#pragma unroll
        for (int k = 0; k < G; k++) v[k] = sm[spos(base + (k << BLO))];
        if constexpr (FWD) sgroup_stages<R, 0, true, PRE>(v, tw, tws, S0, hi, np, fp);
        else sgroup_stages<R, R - 1, false, PRE>(v, tw, tws, S0, hi, np, fp);
#pragma unroll
        for (int k = 0; k < G; k++) sm[spos(base + (k << BLO))] = v[k];
    }
}

// Transforms with their remainder stages (the RR = log2 N mod 4 stages that
// pair elements N/2 and N/4 apart) fused into the global load (forward) or
// store (inverse): a thread that loads an element together with its
// partners runs them before the polynomial first reaches shared memory, and
// after it last leaves it.

// Load of the input with the forward remainder stages: element e of the
// buffer gets f(src[e], e) transformed by stages 0 .. RR-1 (values grow by
// 4p a stage).  Ends with a barrier, after which ntt_fwd_grow_rest runs the
// remaining passes.  Loads the shared twiddle cache.
template <int LOGN, bool COHERENT, class F>
__device__ __forceinline__ void fwd_load_first(u64 *sm, Tw *cache, const u64 *src, F f, const Mod &md)
{
    using S = NttShape<LOGN>;
    constexpr int N = 1 << LOGN, T = S::T;
    const u64 np = md.np, fp = md.four_p;
    const int t = threadIdx.x;
    __syncthreads();  // earlier users of sm and the cache are done
    load_tw_cache<LOGN>(cache, md.fwd);
    auto ld = [&](int e) { return COHERENT ? ld2(src + e) : ldg2(src + e); };
    if constexpr (S::RR == 0) {
#pragma unroll 4
        for (int u = 0; u < 16; u++) {
            const int e = 2 * (t + T * u), sp = spos(e);
            const ulonglong2 a = ld(e);
            sm[sp] = f(a.x, e);
            sm[sp ^ 1] = f(a.y, e + 1);
        }
    } else if constexpr (S::RR == 1) {
        const Tw w1 = md.fwd[1];
#pragma unroll 2
        for (int u = 0; u < N / (4 * T); u++) {
            const int e = 2 * (t + T * u), sp = spos(e), sq = spos(e + N / 2);
            const ulonglong2 a = ld(e), b = ld(e + N / 2);
            u64 x0 = f(a.x, e), x1 = f(a.y, e + 1), y0 = f(b.x, e + N / 2), y1 = f(b.y, e + 1 + N / 2);
            ct_grow(x0, y0, w1.w, w1.ws, np, fp);
            ct_grow(x1, y1, w1.w, w1.ws, np, fp);
            sm[sp] = x0;
            sm[sp ^ 1] = x1;
            sm[sq] = y0;
            sm[sq ^ 1] = y1;
        }
    } else {
        const Tw w1 = md.fwd[1], w2 = md.fwd[2], w3 = md.fwd[3];
#pragma unroll 1
        for (int u = 0; u < N / (8 * T); u++) {
            const int e0 = 2 * (t + T * u);
            u64 v[2][4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const ulonglong2 a = ld(e0 + q * (N / 4));
                v[0][q] = f(a.x, e0 + q * (N / 4));
                v[1][q] = f(a.y, e0 + 1 + q * (N / 4));
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                ct_grow(v[h][0], v[h][2], w1.w, w1.ws, np, fp);  // stage 0: N/2 apart
                ct_grow(v[h][1], v[h][3], w1.w, w1.ws, np, fp);
                ct_grow(v[h][0], v[h][1], w2.w, w2.ws, np, fp);  // stage 1: N/4 apart, two blocks
                ct_grow(v[h][2], v[h][3], w3.w, w3.ws, np, fp);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int sp = spos(e0 + q * (N / 4));
                sm[sp] = v[0][q];
                sm[sp ^ 1] = v[1][q];
            }
        }
    }
    __syncthreads();
}

// The forward passes after fwd_load_first.  Ends with a barrier.
template <int LOGN>
__device__ __forceinline__ void ntt_fwd_grow_rest(u64 *sm, const Tw *cache, const Mod &md)
{
    using S = NttShape<LOGN>;
    const u64 np = md.np, fp = md.four_p;
#pragma unroll 1
    for (int s0 = S::RR; s0 < LOGN - 4; s0 += 4) {
        spass<LOGN, 4, true, false>(sm, s0, cache, np, fp);
        __syncthreads();
    }
    spass<LOGN, 4, true, true>(sm, LOGN - 4, md.fwd_last, np, fp);
    __syncthreads();
}

// The inverse transform up to its remainder stages, its input loaded from
// global memory (values < 4p; coalesced, COHERENT: written earlier by this
// kernel).  Loads the shared twiddle cache; ends with a barrier, after which
// inv_store_last finishes.
template <int LOGN, bool COHERENT>
__device__ __forceinline__ void ntt_inv_keep_from(u64 *sm, Tw *cache, const u64 *src, const Mod &md)
{
    using S = NttShape<LOGN>;
    const u64 np = md.np, fp = md.four_p;
    __syncthreads();  // earlier users of sm and the cache are done
    load_tw_cache<LOGN>(cache, md.inv);
    poly_load<LOGN, COHERENT>(sm, src);
    __syncthreads();
    spass<LOGN, 4, false, true>(sm, LOGN - 4, md.inv_last, np, fp);
    __syncthreads();
#pragma unroll 1
    for (int s0 = LOGN - 8; s0 >= S::RR; s0 -= 4) {
        spass<LOGN, 4, false, false>(sm, s0, cache, np, fp);
        __syncthreads();
    }
}

// The inverse's remainder stages fused with the store: coefficient e (times
// N, scaled back by N^-1) to dst[e], canonical.
template <int LOGN>
__device__ __forceinline__ void inv_store_last(const u64 *sm, u64 *dst, const Mod &md)
{
    using S = NttShape<LOGN>;
    constexpr int N = 1 << LOGN, T = S::T;
    const u64 np = md.np, fp = md.four_p;
    const int t = threadIdx.x;
    if constexpr (S::RR == 0) {
#pragma unroll 4
        for (int u = 0; u < 16; u++) {
            const int e = 2 * (t + T * u), sp = spos(e);
            st2(dst + e, inv_finish(sm[sp], md), inv_finish(sm[sp ^ 1], md));
        }
    } else if constexpr (S::RR == 1) {
        const Tw w1 = md.inv[1];
#pragma unroll 2
        for (int u = 0; u < N / (4 * T); u++) {
            const int e = 2 * (t + T * u), sp = spos(e), sq = spos(e + N / 2);
            u64 x0 = sm[sp], x1 = sm[sp ^ 1], y0 = sm[sq], y1 = sm[sq ^ 1];
            gs_keep(x0, y0, w1.w, w1.ws, np, fp);
            gs_keep(x1, y1, w1.w, w1.ws, np, fp);
            st2(dst + e, inv_finish(x0, md), inv_finish(x1, md));
            st2(dst + e + N / 2, inv_finish(y0, md), inv_finish(y1, md));
        }
    } else {
        const Tw w1 = md.inv[1], w2 = md.inv[2], w3 = md.inv[3];
#pragma unroll 1
        for (int u = 0; u < N / (8 * T); u++) {
            const int e0 = 2 * (t + T * u);
            u64 v[2][4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int sp = spos(e0 + q * (N / 4));
                v[0][q] = sm[sp];
                v[1][q] = sm[sp ^ 1];
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                gs_keep(v[h][0], v[h][1], w2.w, w2.ws, np, fp);  // stage 1 first
                gs_keep(v[h][2], v[h][3], w3.w, w3.ws, np, fp);
                gs_keep(v[h][0], v[h][2], w1.w, w1.ws, np, fp);  // then stage 0
                gs_keep(v[h][1], v[h][3], w1.w, w1.ws, np, fp);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) st2(dst + e0 + q * (N / 4), inv_finish(v[0][q], md), inv_finish(v[1][q], md));
        }
    }
}

// x < 64p -> [0, p)
__device__ __forceinline__ u64 reduce64p(u64 x, const Mod &md)
{
    const u64 p = md.p;
    x = csub(x, p << 5);
    x = csub(x, p << 4);
    x = csub(x, p << 3);
    x = csub(x, md.four_p);
    x = csub(x, md.two_p);
    return csub(x, p);
}

}  // namespace wally
