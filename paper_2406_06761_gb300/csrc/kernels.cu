// kernels.cu -- device kernels of the Wally GB300 library (evaluation path).
//
// Paper steps (arXiv 2406.06761) and where they run:
//   a0 grouping of the batch by cluster ......... k_hist / k_scan_clusters / k_scatter, k_gather_wave, k_wave_plan
//   a1 inputs to NTT form ....................... k_to_ntt
//   a2/a4 rotations Rot_k (Sec. 2 CtRotate, hybrid key switching Sec. 7)
//        ......................................... k_ks_a (automorphism + INTT of c1 -> digits; first of a chain)
//                                                  k_ks_b (digit NTTs + inner product with the key)
//                                                  k_ks_c (ModDown, + sigma(c0), + T_i for Horner; then the
//                                                          next rotation's automorphism and digits)
//   a3 plaintext x ciphertext products (Alg. "Server Computation") ... k_mac
//   a5 output to coefficient form ............... k_output
#include <cstdio>
#include "kernels.hpp"
#include "ntt_regs.cuh"

namespace wally {

namespace {

__device__ __forceinline__ void load_mod(Mod *s, const DevParams *dpp, int j)
{
    if (threadIdx.x < sizeof(Mod) / 8) ((u64 *)s)[threadIdx.x] = ((const u64 *)&dpp->m[j])[threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ u32 item_count(u32 n_max, const u32 *n_dev)
{
    if (!n_dev) return n_max;
    u32 c = *n_dev;
    return c < n_max ? c : n_max;
}

// Two transform cores: the register-blocked one of ntt_regs.cuh (32
// coefficients a thread, two CTAs an SM) for the kernels that transform one
// polynomial per CTA (inputs, outputs, chain starts), and the shared-memory
// one of common.cuh (three CTAs an SM) for the key-switch kernels, whose
// memory-bound phases (key inner products, ModDown) need the extra resident
// CTAs to hide their latency.
template <int LOGN>
using RP = NttV<LOGN, 32>;
#define NTT_LB(LOGN) __launch_bounds__(RP<LOGN>::T, RP<LOGN>::MIN_BLOCKS)

// Shared memory of the transform kernels: one polynomial buffer and the
// twiddle cache.
template <int LOGN>
struct Smem {
    u64 *poly;
    Tw *twf, *twi;
    __device__ __forceinline__ explicit Smem(u64 *base)
    {
        poly = base;
        twf = reinterpret_cast<Tw *>(base + smem_words(1 << LOGN));
        twi = twf;  // one cache, reloaded by every transform
    }
};

#define OLD_LB(LOGN) __launch_bounds__(NttShape<LOGN>::T, NttShape<LOGN>::MIN_BLOCKS)

// Parameters of modulus j and the shared copies of the first 32 entries of
// its forward and inverse twiddle tables (the register core reads the other
// entries from global memory); ends with a barrier.
struct ModSmem {
    Mod md;
    Tw twf[32], twi[32];
};

__device__ __forceinline__ void load_mod_tw(ModSmem &ms, const DevParams *dpp, int j)
{
    if (threadIdx.x < sizeof(Mod) / 8) ((u64 *)&ms.md)[threadIdx.x] = ((const u64 *)&dpp->m[j])[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 32) ms.twf[threadIdx.x] = ms.md.fwd[threadIdx.x];
    else if (threadIdx.x < 64) ms.twi[threadIdx.x - 32] = ms.md.inv[threadIdx.x - 32];
    __syncthreads();
}

// ---------------------------------------------------------------- a1: to NTT form
// Item x, polynomial z (modulus z % mod_cycle): forward NTT of the input
// (coefficients < 8p), canonical output, optionally times 2^64 (Montgomery).
template <int LOGN>
__global__ void NTT_LB(LOGN) k_to_ntt(const DevParams *dpp, const u64 *const *src_ptrs, const u64 *src,
                                      size_t src_stride, u64 *dst, size_t dst_stride, u32 mod_cycle, u32 n_max,
                                      const u32 *n_dev, bool mont)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    const u32 x = blockIdx.x;
    if (x >= item_count(n_max, n_dev)) return;
    const u32 z = blockIdx.y;
    const u64 *s = (src_ptrs ? src_ptrs[x] : src + x * src_stride) + (size_t)z * N;
    u64 v[32];
    gload_first<P>(v, s);
    load_mod_tw(ms, dpp, z % mod_cycle);
    const Mod &md = ms.md;
    ntt_fwd_v<P>(v, sm, ms.twf, md.fwd, md);
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = mont ? mont_mul(v[k], md.r2, md) : reduce64p(v[k], md);
    gstore_last<P>(dst + x * dst_stride + (size_t)z * N, v);
}

// Inverse NTT, canonical coefficients.
template <int LOGN>
__global__ void NTT_LB(LOGN) k_from_ntt(const DevParams *dpp, const u64 *src, u64 *dst, u32 polys, u32 mod_cycle)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    const u32 x = blockIdx.x, z = blockIdx.y;
    u64 v[32];
    gload_last<P>(v, src + ((size_t)x * polys + z) * N);
    load_mod_tw(ms, dpp, z % mod_cycle);
    const Mod &md = ms.md;
    ntt_inv_v<P>(v, sm, ms.twi, md.inv, md);
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = inv_finish(v[k], md);
    gstore_first<P>(dst + ((size_t)x * polys + z) * N, v);
}

// ---------------------------------------------------------------- a2/a4: rotations
// k_ks_a, CTA (item x, limb j, component c): first rotation of a chain.
// Limb j of component c of the input (NTT form) is permuted by sigma_k (a
// permutation of the evaluation positions, through shared memory) into sc;
// for c = 1 its inverse transform gives the digit d_j = [sigma(c1)]_{q_j} in
// [0, q_j) (reading R3: non-centred), written to dg.
template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_a(const DevParams *dpp, RotArgs a)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    // the 2L CTAs of an item are adjacent in the grid (they share its data in L2)
    const int L = dpp->L;
    const u32 x = blockIdx.x / (2 * L);
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int y = (int)(blockIdx.x % (2 * L)), j = y % L, c = y / L;
    u64 v[32];
    gload_last<P>(v, a.src + x * a.src_stride + ((size_t)c * L + j) * N);
    load_mod_tw(ms, dpp, j);
    sm_store_last<P>(sm, v);
    __syncthreads();
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < 32; r++) v[r] = sm[phys<P>((int)galois_src((u32)elem_last<P>(t, r), a.galois, LOGN))];
    gstore_last<P>(a.sc + ((size_t)x * 2 * L + c * L + j) * N, v);
    if (c == 1) {
        ntt_inv_v<P>(v, sm, ms.twi, ms.md.inv, ms.md);
#pragma unroll
        for (int r = 0; r < 32; r++) v[r] = inv_finish(v[r], ms.md);
        gstore_first<P>(a.dg + ((size_t)x * L + j) * N, v);
    }
}

// The fused part of k_ks_c (shared-memory transform core).  The buffer holds limb
// j of component c of a ciphertext (NTT form); write sigma_k of it to sc and,
// for c = 1, the digit d_j = [sigma(c1)]_{q_j} in [0, q_j) (reading R3:
// non-centred) to dg.  sigma_k is a permutation of the NTT positions.
template <int LOGN>
__device__ __forceinline__ void permute_and_digit_smem(const Smem<LOGN> &S, const Mod &md, u64 k, int c, u64 *sc_cj,
                                                  u64 *dg_j)
{
    __syncthreads();
#pragma unroll 4
    for (int u = 0; u < 16; u++) {
        const int e = pair_elem<LOGN>(u);
        st2(sc_cj + e, S.poly[spos(galois_src(e, k, LOGN))], S.poly[spos(galois_src(e + 1, k, LOGN))]);
    }
    if (c == 1) {
        // the inverse reads its first pass from sc_cj (this CTA's own writes,
        // visible after the barrier it starts with) and stores the digit
        ntt_inv_keep_from<LOGN, true>(S.poly, S.twi, sc_cj, md);
        inv_store_last<LOGN>(S.poly, dg_j, md);
    }
}

// k_ks_b, CTA (item x, modulus j in q_0..q_{L-1}, P):
//   u_j = sum_i NTT_j(d_i) * key_{i,j}  for both key components,
// as one lazy 128-bit sum per output and a single Montgomery reduction (the
// key is stored times 2^64).  NTT_j(d_j) = sigma(c1)_j is already known; the
// other digits are transformed here (lazy values below 56 p_j; a sum of L
// products with keys below p_j stays below p_j 2^64), all but the last one
// parked in dd.  For
// j = P the sums are brought back to coefficients (r = [u]_P) for ModDown.
template <int LOGN>
__global__ void OLD_LB(LOGN) k_ks_b(const DevParams *dpp, RotArgs a)
{
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 smraw[];
    Smem<LOGN> S(smraw);
    __shared__ Mod md;
    // the L+1 CTAs of an item are adjacent in the grid, so that the digits
    // they all read are served from L2; within an item the CTA of j = P
    // (which also runs two inverse transforms) comes first
    const int L = dpp->L;
    const u32 x = blockIdx.x / (L + 1);
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int j = L - (int)(blockIdx.x % (L + 1));
    load_mod(&md, dpp, j);
    const u64 *kx = a.key + (size_t)(a.key_map ? a.key_map[x] : x) * a.key_stride;
    const u64 pol = l2_evict_first_policy();  // keys: read once a key switch
    u64 *dd = a.dd + ((size_t)x * (L + 1) + j) * L * N;
    for (int i = 0; i < L; i++) {
        if (i == j) continue;
        // digit i (< q_i < 2 p_j), its first stage fused into the load
        fwd_load_first<LOGN, false>(S.poly, S.twf, a.dg + ((size_t)x * L + i) * N, [](u64 v, int) { return v; }, md);
        ntt_fwd_grow_rest<LOGN>(S.poly, S.twf, md);  // lazy, < 56 p_j
        u64 *di = dd + (size_t)i * N;
#pragma unroll 4
        for (int u = 0; u < 16; u++) {
            const int e = pair_elem<LOGN>(u), sp = spos(e);
            st2(di + e, S.poly[sp], S.poly[sp ^ 1]);  // lazy
        }
    }
    u64 *u0 = a.u + ((size_t)x * 2 + 0) * (L + 1) * N + (size_t)j * N;
    u64 *u1 = a.u + ((size_t)x * 2 + 1) * (L + 1) * N + (size_t)j * N;
    const u64 *sc1 = a.sc + ((size_t)x * 2 * L + L + j) * N;
    // The inner product streams its operands -- per step (u, i) the thread's
    // pair of digit i (this thread's own writes to dd, or sigma(c1) for
    // i = j) and of the two key components -- through a ring of KS stages of
    // cp.async copies in the shared memory the transforms used (the buffer
    // and the twiddle cache: exactly KS stages of 3 x 16 bytes a thread).
    // Every thread reads only its own copies, so the ring needs no barrier.
    constexpr int T = NttShape<LOGN>::T, KS = 6, SW = 6 * T;  // SW: words a stage
    static_assert(KS * SW == ntt_smem_words<LOGN>(), "the ring fills the transform's shared memory");
    __syncthreads();  // every thread has stored its part of the last digit
    u64 *ring = smraw + 2 * threadIdx.x;
    const int steps = 16 * L;
    int iu = 0, ii = 0, is = 0;  // the next step to copy
    auto copy_next = [&]() {
        if (is < steps) {
            const int e = pair_elem<LOGN>(iu);
            u64 *slot = ring + (size_t)(is % KS) * SW;
            cp_async16(slot, (ii == j ? sc1 : dd + (size_t)ii * N) + e);
            cp_async16_hint(slot + 2 * T, kx + (((size_t)ii * 2 + 0) * (L + 1) + j) * N + e, pol);
            cp_async16_hint(slot + 4 * T, kx + (((size_t)ii * 2 + 1) * (L + 1) + j) * N + e, pol);
            if (++ii == L) ii = 0, ++iu;
        }
        ++is;
        cp_async_commit();  // one group a step, empty past the end
    };
    for (int k = 0; k < KS; k++) copy_next();
    int s = 0;
    for (int u = 0; u < 16; u++) {
        const int e = pair_elem<LOGN>(u);
        Acc28 s0a, s0b, s1a, s1b;  // digits < 56 p_j, keys < p_j, L <= 32 terms
        acc28_zero(s0a), acc28_zero(s0b), acc28_zero(s1a), acc28_zero(s1b);
        for (int i = 0; i < L; i++, s++) {
            cp_async_wait<KS - 1>();  // step s has landed
            const u64 *slot = ring + (size_t)(s % KS) * SW;
            const ulonglong2 d = ld2(slot), kb = ld2(slot + 2 * T), ka = ld2(slot + 4 * T);
            copy_next();  // step s + KS, into the slot just read
            u32 a0, a1, b0, b1;
            split28(d.x, a0, a1);
            split28(d.y, b0, b1);
            mac28(s0a, a0, a1, kb.x);
            mac28(s0b, b0, b1, kb.y);
            mac28(s1a, a0, a1, ka.x);
            mac28(s1b, b0, b1, ka.y);
        }
        st2(u0 + e, acc28_redc(s0a, md), acc28_redc(s0b, md));
        st2(u1 + e, acc28_redc(s1a, md), acc28_redc(s1b, md));
    }
    cp_async_wait<0>();
    if (j == L) {
        for (int c = 0; c < 2; c++) {
            u64 *uc = c ? u1 : u0;
            ntt_inv_keep_from<LOGN, true>(S.poly, S.twi, uc, md);  // this CTA's own writes
            inv_store_last<LOGN>(S.poly, uc, md);
        }
    }
}

// k_ks_c, CTA (item x, limb j, component c): ModDown (reading R4: round to
// nearest through the centred residue r_c of u mod P):
//   u'_j = (u_j - NTT_j(r_c)) * P^-1 mod q_j,
//   out_0 = sigma(c0)_j + u0'_j [+ T0_j],  out_1 = u1'_j [+ T1_j].
// With next_galois set, the output is also prepared as the input of the next
// rotation of the chain (its automorphism and, for c = 1, its digit).
template <int LOGN>
__global__ void OLD_LB(LOGN) k_ks_c(const DevParams *dpp, RotArgs a)
{
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 smraw[];
    Smem<LOGN> S(smraw);
    __shared__ Mod md;
    // the 2L CTAs of an item are adjacent in the grid (they share the residue
    // mod P in L2); component 1 first: its CTAs also run the next rotation's
    // digit INTT
    const int L = dpp->L;
    const u32 x = blockIdx.x / (2 * L);
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int y = (int)(blockIdx.x % (2 * L)), j = y % L, c = 1 - y / L;
    load_mod(&md, dpp, j);
    const u64 q = md.p, P = dpp->m[L].p, half = (P - 1) / 2;
    const u64 pinv = dpp->pinv[j], pinv_s = dpp->pinv_s[j];
    const u64 q64 = q << 6;
    const u64 *r = a.u + (((size_t)x * 2 + c) * (L + 1) + L) * N;
    // r_c mod q_j (< 2q), the first forward stage fused into the load
    fwd_load_first<LOGN, false>(S.poly, S.twf, r, [=](u64 v, int) { return v > half ? q - (P - v) : v; }, md);
    ntt_fwd_grow_rest<LOGN>(S.poly, S.twf, md);  // < 58q
    const u64 *uj = a.u + (((size_t)x * 2 + c) * (L + 1) + j) * N;
    u64 *sc_cj = a.sc + ((size_t)x * 2 * L + c * L + j) * N;
    const u64 *ad = a.add ? a.add + x * a.add_stride + ((size_t)c * L + j) * N : nullptr;
    u64 *dst = a.dst + x * a.dst_stride + ((size_t)c * L + j) * N;
#pragma unroll 4
    for (int u = 0; u < 16; u++) {
        const int e = pair_elem<LOGN>(u), sp = spos(e);
        const ulonglong2 uv = ldg2(uj + e);
        u64 v0 = csub(shoup_mul(uv.x + q64 - S.poly[sp], pinv, pinv_s, q), q);
        u64 v1 = csub(shoup_mul(uv.y + q64 - S.poly[sp ^ 1], pinv, pinv_s, q), q);
        if (c == 0) {
            const ulonglong2 s0 = ld2(sc_cj + e);
            v0 = addmod(v0, s0.x, q);
            v1 = addmod(v1, s0.y, q);
        }
        if (ad) {
            const ulonglong2 t = ldg2(ad + e);
            v0 = addmod(v0, t.x, q);
            v1 = addmod(v1, t.y, q);
        }
        st2(dst + e, v0, v1);
        S.poly[sp] = v0;  // same thread, same positions: the output replaces NTT(r)
        S.poly[sp ^ 1] = v1;
    }
    if (a.next_galois)
        permute_and_digit_smem<LOGN>(S, md, a.next_galois, c, sc_cj, a.dg + ((size_t)x * L + j) * N);
}

// The same two key-switch kernels on the register core (two CTAs an SM): the
// digits' transforms read their input straight into registers and leave
// the evaluations there for the inner product, and ModDown's transform
// feeds the pointwise step without a pass through shared memory.
template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_b_reg(const DevParams *dpp, RotArgs a)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    const int L = dpp->L;
    const u32 x = blockIdx.x / (L + 1);
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int j = L - (int)(blockIdx.x % (L + 1));
    const int last = (j == L - 1) ? L - 2 : L - 1;
    u64 v[32];
    const int i0 = (j == 0) ? 1 : 0;
    if (i0 < L) gload_first<P>(v, a.dg + ((size_t)x * L + i0) * N);
    load_mod_tw(ms, dpp, j);
    for (int i = i0; i < L; i++) {
        if (i == j) continue;
        if (i != i0) gload_first<P>(v, a.dg + ((size_t)x * L + i) * N);  // < q_i < 2 p_j
        ntt_fwd_v<P>(v, sm, ms.twf, ms.md.fwd, ms.md);                 // lazy, < 56 p_j
        if (i != last) gstore_last<P>(a.dd + (((size_t)x * (L + 1) + j) * L + i) * N, v);
    }
    const Mod &md = ms.md;
    const u64 *kx = a.key + (size_t)(a.key_map ? a.key_map[x] : x) * a.key_stride;
    const u64 pol = l2_evict_first_policy();  // keys: read once a key switch
    const u64 *dd = a.dd + ((size_t)x * (L + 1) + j) * L * N;
    u64 *u0 = a.u + ((size_t)x * 2 + 0) * (L + 1) * N + (size_t)j * N;
    u64 *u1 = a.u + ((size_t)x * 2 + 1) * (L + 1) * N + (size_t)j * N;
    const u64 *sc1 = a.sc + ((size_t)x * 2 * L + L + j) * N;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        const int e = elem_last<P>(t, k);
        Acc28 s0a, s0b, s1a, s1b;  // digits < 56 p_j, keys < p_j, L <= 32 terms
        acc28_zero(s0a), acc28_zero(s0b), acc28_zero(s1a), acc28_zero(s1b);
        for (int i = 0; i < L; i++) {
            u64 da, db;
            if (i == j) {
                const ulonglong2 q = ld2(sc1 + e);
                da = q.x;
                db = q.y;
            } else if (i == last) {
                da = v[k];
                db = v[k + 1];
            } else {
                const ulonglong2 q = ld2(dd + (size_t)i * N + e);  // this thread's own writes
                da = q.x;
                db = q.y;
            }
            const ulonglong2 kb = ldg2_hint(kx + (((size_t)i * 2 + 0) * (L + 1) + j) * N + e, pol);
            const ulonglong2 ka = ldg2_hint(kx + (((size_t)i * 2 + 1) * (L + 1) + j) * N + e, pol);
            u32 a0, a1, b0, b1;
            split28(da, a0, a1);
            split28(db, b0, b1);
            mac28(s0a, a0, a1, kb.x);
            mac28(s0b, b0, b1, kb.y);
            mac28(s1a, a0, a1, ka.x);
            mac28(s1b, b0, b1, ka.y);
        }
        st2(u0 + e, acc28_redc(s0a, md), acc28_redc(s0b, md));
        st2(u1 + e, acc28_redc(s1a, md), acc28_redc(s1b, md));
    }
    if (j == L) {
        for (int c = 0; c < 2; c++) {
            u64 *uc = c ? u1 : u0;
            gload_last<P, true>(v, uc);  // this thread's own writes
            ntt_inv_v<P>(v, sm, ms.twi, md.inv, md);
#pragma unroll
            for (int k = 0; k < 32; k++) v[k] = inv_finish(v[k], md);
            gstore_first<P>(uc, v);
        }
    }
}

template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_c_reg(const DevParams *dpp, RotArgs a)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    const int L = dpp->L;
    const u32 x = blockIdx.x / (2 * L);
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int y = (int)(blockIdx.x % (2 * L)), j = y % L, c = 1 - y / L;
    u64 v[32];
    gload_first<P>(v, a.u + (((size_t)x * 2 + c) * (L + 1) + L) * N);  // r = [u]_P, coefficients
    load_mod_tw(ms, dpp, j);
    const Mod &md = ms.md;
    const u64 q = md.p, Pm = dpp->m[L].p, half = (Pm - 1) / 2;
    const u64 pinv = dpp->pinv[j], pinv_s = dpp->pinv_s[j];
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = v[k] > half ? q - (Pm - v[k]) : v[k];  // r_c mod q_j, < 2q
    ntt_fwd_v<P>(v, sm, ms.twf, md.fwd, md);  // < 58q
    const u64 *uj = a.u + (((size_t)x * 2 + c) * (L + 1) + j) * N;
    u64 *sc_cj = a.sc + ((size_t)x * 2 * L + c * L + j) * N;
    const u64 *ad = a.add ? a.add + x * a.add_stride + ((size_t)c * L + j) * N : nullptr;
    u64 *dst = a.dst + x * a.dst_stride + ((size_t)c * L + j) * N;
    const u64 q64 = q << 6;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        const int e = elem_last<P>(t, k);
        const ulonglong2 uv = ldg2(uj + e);
        u64 v0 = csub(shoup_mul(uv.x + q64 - v[k], pinv, pinv_s, q), q);
        u64 v1 = csub(shoup_mul(uv.y + q64 - v[k + 1], pinv, pinv_s, q), q);
        if (c == 0) {
            const ulonglong2 s0 = ld2(sc_cj + e);
            v0 = addmod(v0, s0.x, q);
            v1 = addmod(v1, s0.y, q);
        }
        if (ad) {
            const ulonglong2 tt = ldg2(ad + e);
            v0 = addmod(v0, tt.x, q);
            v1 = addmod(v1, tt.y, q);
        }
        v[k] = v0;
        v[k + 1] = v1;
    }
    gstore_last<P>(dst, v);
    if (a.next_galois) {
        __syncthreads();  // every thread has read sigma(c0) from sc_cj before it is replaced
        sm_store_last<P>(sm, v);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; r++)
            v[r] = sm[phys<P>((int)galois_src((u32)elem_last<P>(t, r), a.next_galois, LOGN))];
        gstore_last<P>(sc_cj, v);
        if (c == 1) {
            ntt_inv_v<P>(v, sm, ms.twi, md.inv, md);
#pragma unroll
            for (int r = 0; r < 32; r++) v[r] = inv_finish(v[r], md);
            gstore_first<P>(a.dg + ((size_t)x * L + j) * N, v);
        }
    }
}

// ---------------------------------------------------------------- a3: PtCt products
// For every (segment of one cluster in the wave, chunk k, limb l, tile of ts
// slot positions): load the tile of P'_{k,i,b} (d_pad x ts words) into shared
// memory once, then for every query of the segment
//   T_i[c] = sum_b P'_{k,i,b} * ct'[b][c]  (i < h, c = 0, 1)
// with exact lazy accumulation (28-bit limb columns) and one Montgomery
// reduction per output
// (plaintexts are stored times 2^64, Sec. 7 lazy reduction).
template <int G, int CPT>
__global__ void __launch_bounds__(256, 2) k_mac(const DevParams *dpp, ClusterStore cs, WavePlan wp, const u64 *ctp,
                                             u64 *Tout, u32 m_max)
{
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const int L = dpp->L, log_n = dpp->log_n, N = 1 << log_n;
    const int h = dpp->h, dp_ = dpp->d_pad;
    const int ts = cs.ts, tiles = N / ts;
    const size_t ctw = (size_t)2 * L * N;
    const u32 nseg = wp.counts[2];
    const u64 total = (u64)nseg * m_max * L * tiles;
    const int slot_in = threadIdx.x % ts;
    const int rest = threadIdx.x / ts;
    const int comp = (CPT == 2) ? 0 : (rest & 1);
    const int ql = (CPT == 2) ? rest : (rest >> 1);
    const int QL = (CPT == 2) ? (256 / ts) : (128 / ts);
    for (u64 v = blockIdx.x; v < total; v += gridDim.x) {
        const int tile = (int)(v % tiles);
        u64 r = v / tiles;
        const int l = (int)(r % L);
        r /= L;
        const int k = (int)(r % m_max);
        const u32 seg = (u32)(r / m_max);
        const u32 cl = wp.seg_cluster[seg];
        if (k >= (int)cs.chunks[cl]) continue;  // uniform across the CTA
        __syncthreads();
        if (threadIdx.x == 0) md = dpp->m[l];
        const u32 z = cs.chunk0[cl] + k;
        const uint4 *tsrc = (const uint4 *)(cs.ptxt + (((size_t)z * L + l) * tiles + tile) * ((size_t)dp_ * ts));
        uint4 *tdst = (uint4 *)sm;
        const int words2 = dp_ * ts / 2;
        for (int w = threadIdx.x; w < words2; w += 256) tdst[w] = tsrc[w];
        __syncthreads();
        const int s = tile * ts + slot_in;
        const u32 sb = wp.seg_begin[seg], se = wp.seg_end[seg];
        // a segment with fewer queries than query lanes also spreads the
        // giant-step rows i over the idle lanes (IG row groups)
        int IG = 1;
        while (IG * 2 <= QL && IG * 2 <= h && (u32)(QL / (IG * 2)) >= se - sb) IG *= 2;
        const int QLp = QL / IG, qlane = ql % QLp, ig = ql / QLp;
        for (u32 pos = sb + qlane; pos < se; pos += QLp) {
            const u64 *cq = ctp + (size_t)pos * G * ctw + (size_t)l * N + s;
            u32 cb0[G][CPT], cb1[G][CPT];  // in 28-bit limbs
#pragma unroll
            for (int b = 0; b < G; b++)
#pragma unroll
                for (int c = 0; c < CPT; c++) split28(cq[(size_t)b * ctw + (size_t)(c + comp) * L * N], cb0[b][c], cb1[b][c]);
            const u32 p = wp.pair_off[pos] + k;
            u64 *to = Tout + (size_t)p * h * ctw + (size_t)l * N + s;
            for (int i = ig; i < h; i += IG) {
                Acc28 acc[CPT];  // operands < p, G <= 32 terms
#pragma unroll
                for (int c = 0; c < CPT; c++) acc28_zero(acc[c]);
                const u64 *prow = sm + (size_t)i * G * ts + slot_in;
#pragma unroll
                for (int b = 0; b < G; b++) {
                    u32 p0, p1;
                    split28(prow[b * ts], p0, p1);
#pragma unroll
                    for (int c = 0; c < CPT; c++) mac28(acc[c], p0, p1, cb0[b][c], cb1[b][c]);
                }
#pragma unroll
                for (int c = 0; c < CPT; c++) to[(size_t)i * ctw + (size_t)(c + comp) * L * N] = acc28_redc(acc[c], md);
            }
        }
    }
}

// The same products with the tile's two halves (ts/2 slot positions each)
// as the unit of work, double-buffered: while a half is multiplied, the
// next unit's half is copied into the other buffer with cp.async, so that
// short segments (one query a cluster, as in the serving loop's waves) no
// longer wait for their tile.  Two buffers of d_pad x ts/2 words take the
// same shared memory as one whole tile.

template <int G>
__global__ void __launch_bounds__(256, 2) k_mac_halves(const DevParams *dpp, ClusterStore cs, WavePlan wp,
                                                    const u64 *ctp, u64 *Tout, u32 m_max)
{
    extern __shared__ __align__(16) u64 sm[];
    const int L = dpp->L, log_n = dpp->log_n, N = 1 << log_n;
    const int h = dpp->h, dp_ = dpp->d_pad;
    const int ts = cs.ts, hts = ts / 2, tiles = N / ts;
    const size_t ctw = (size_t)2 * L * N;
    const u32 nseg = wp.counts[2];
    const u64 total = (u64)nseg * m_max * L * tiles * 2;  // units: (item, half)
    const int slot_in = threadIdx.x % hts;
    const int ql = threadIdx.x / hts;
    const int QL = 256 / hts;
    const size_t buf_words = (size_t)dp_ * hts;
    // the unit's item, or false when its chunk does not exist (uniform)
    auto decode = [&](u64 w, int &half, int &tile, int &l, int &k, u32 &seg, u32 &cl) {
        half = (int)(w & 1);
        u64 v = w >> 1;
        tile = (int)(v % tiles);
        u64 r = v / tiles;
        l = (int)(r % L);
        r /= L;
        k = (int)(r % m_max);
        seg = (u32)(r / m_max);
        cl = wp.seg_cluster[seg];
        return k < (int)cs.chunks[cl];
    };
    auto next_valid = [&](u64 w) {
        int half, tile, l, k;
        u32 seg, cl;
        while (w < total && !decode(w, half, tile, l, k, seg, cl)) w += gridDim.x;
        return w;
    };
    auto issue = [&](u64 w, u64 *buf) {
        int half, tile, l, k;
        u32 seg, cl;
        decode(w, half, tile, l, k, seg, cl);
        const u32 z = cs.chunk0[cl] + k;
        const u64 *tsrc = cs.ptxt + (((size_t)z * L + l) * tiles + tile) * ((size_t)dp_ * ts) + half * hts;
        const int per_row = hts / 2;  // 16-byte pieces a row
        for (int q = threadIdx.x; q < dp_ * per_row; q += 256) {
            const int row = q / per_row, col = (q % per_row) * 2;
            cp_async16(buf + (size_t)row * hts + col, tsrc + (size_t)row * ts + col);
        }
    };
    u64 w = next_valid(blockIdx.x);
    int b = 0;
    if (w < total) issue(w, sm);
    asm volatile("cp.async.commit_group;" ::: "memory");
    while (w < total) {
        const u64 wn = next_valid(w + gridDim.x);
        if (wn < total) issue(wn, sm + (b ^ 1) * buf_words);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        int half, tile, l, k;
        u32 seg, cl;
        decode(w, half, tile, l, k, seg, cl);
        const u64 p = dpp->m[l].p, mni = dpp->m[l].mont_neg_inv;
        const u64 *buf = sm + b * buf_words;
        const int s = tile * ts + half * hts + slot_in;
        const u32 sb = wp.seg_begin[seg], se = wp.seg_end[seg];
        int IG = 1;
        while (IG * 2 <= QL && IG * 2 <= h && (u32)(QL / (IG * 2)) >= se - sb) IG *= 2;
        const int QLp = QL / IG, qlane = ql % QLp, ig = ql / QLp;
        for (u32 pos = sb + qlane; pos < se; pos += QLp) {
            const u64 *cq = ctp + (size_t)pos * G * ctw + (size_t)l * N + s;
            u32 cb0[G][2], cb1[G][2];  // in 28-bit limbs
#pragma unroll
            for (int bb = 0; bb < G; bb++)
#pragma unroll
                for (int c = 0; c < 2; c++) split28(cq[(size_t)bb * ctw + (size_t)c * L * N], cb0[bb][c], cb1[bb][c]);
            const u32 pr = wp.pair_off[pos] + k;
            u64 *to = Tout + (size_t)pr * h * ctw + (size_t)l * N + s;
            for (int i = ig; i < h; i += IG) {
                Acc28 s0, s1;  // operands < p, G <= 16 terms
                acc28_zero(s0), acc28_zero(s1);
                const u64 *prow = buf + (size_t)i * G * hts + slot_in;
#pragma unroll
                for (int bb = 0; bb < G; bb++) {
                    u32 p0, p1;
                    split28(prow[bb * hts], p0, p1);
                    mac28(s0, p0, p1, cb0[bb][0], cb1[bb][0]);
                    mac28(s1, p0, p1, cb0[bb][1], cb1[bb][1]);
                }
                Mod md;
                md.p = p;
                md.mont_neg_inv = mni;
                to[(size_t)i * ctw] = acc28_redc(s0, md);
                to[(size_t)i * ctw + (size_t)L * N] = acc28_redc(s1, md);
            }
        }
        __syncthreads();  // the buffer is read out before the next prefetch refills it
        w = wn;
        b ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The same products for the other splits, mainly those with more than 32 baby
// steps (the plain diagonal split g = d_pad, h = 1 of Sec. 5 for clusters of
// sqrt(d) chunks or more): the g ciphertexts are streamed from global memory
// instead of held in registers; one thread per (slot of the tile, component,
// query).
__global__ void __launch_bounds__(256) k_mac_wide(const DevParams *dpp, ClusterStore cs, WavePlan wp, const u64 *ctp,
                                                  u64 *Tout, u32 m_max)
{
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const int L = dpp->L, log_n = dpp->log_n, N = 1 << log_n;
    const int g = dpp->g, h = dpp->h, dp_ = dpp->d_pad;
    const int ts = cs.ts, tiles = N / ts;
    const size_t ctw = (size_t)2 * L * N;
    const u32 nseg = wp.counts[2];
    const u64 total = (u64)nseg * m_max * L * tiles;
    const int slot_in = threadIdx.x % ts;
    const int rest = threadIdx.x / ts;
    const int comp = rest & 1, ql = rest >> 1, QL = 128 / ts;
    for (u64 v = blockIdx.x; v < total; v += gridDim.x) {
        const int tile = (int)(v % tiles);
        u64 r = v / tiles;
        const int l = (int)(r % L);
        r /= L;
        const int k = (int)(r % m_max);
        const u32 seg = (u32)(r / m_max);
        const u32 cl = wp.seg_cluster[seg];
        if (k >= (int)cs.chunks[cl]) continue;  // uniform across the CTA
        __syncthreads();
        if (threadIdx.x == 0) md = dpp->m[l];
        const u32 z = cs.chunk0[cl] + k;
        const uint4 *tsrc = (const uint4 *)(cs.ptxt + (((size_t)z * L + l) * tiles + tile) * ((size_t)dp_ * ts));
        uint4 *tdst = (uint4 *)sm;
        const int words2 = dp_ * ts / 2;
        for (int w = threadIdx.x; w < words2; w += 256) tdst[w] = tsrc[w];
        __syncthreads();
        if (ql >= QL) continue;
        const int s = tile * ts + slot_in;
        const u32 sb = wp.seg_begin[seg], se = wp.seg_end[seg];
        for (u32 pos = sb + ql; pos < se; pos += QL) {
            const u64 *cq = ctp + (size_t)pos * g * ctw + (size_t)comp * L * N + (size_t)l * N + s;
            const u32 p = wp.pair_off[pos] + k;
            u64 *to = Tout + (size_t)p * h * ctw + (size_t)comp * L * N + (size_t)l * N + s;
            for (int i = 0; i < h; i++) {
                u64 hi = 0, lo = 0;
                const u64 *prow = sm + (size_t)i * g * ts + slot_in;
#pragma unroll 8
                for (int b = 0; b < g; b++) mac128(hi, lo, prow[b * ts], cq[(size_t)b * ctw]);
                to[(size_t)i * ctw] = mont_redc(hi, lo, md);
            }
        }
    }
}

// ---------------------------------------------------------------- a5: output
template <int LOGN>
__global__ void NTT_LB(LOGN) k_output(const DevParams *dpp, WavePlan wp, const u64 *S_, size_t S_stride, u32 n_max)
{
    using P = RP<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ u64 sm[];
    __shared__ ModSmem ms;
    const u32 p = blockIdx.x;
    if (p >= item_count(n_max, wp.counts + 1)) return;
    const int L = dpp->L;
    const int z = blockIdx.y, l = z % L;
    u64 v[32];
    gload_last<P>(v, S_ + p * S_stride + (size_t)z * N);
    load_mod_tw(ms, dpp, l);
    ntt_inv_v<P>(v, sm, ms.twi, ms.md.inv, ms.md);
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = inv_finish(v[k], ms.md);
    gstore_first<P>(wp.dst_out[wp.pair_pos[p]] + (size_t)wp.pair_k[p] * 2 * L * N + (size_t)z * N, v);
}

// ---------------------------------------------------------------- a0: grouping
__global__ void k_hist(const u32 *ids, u32 n, u32 K, u32 *counts, u32 *err)
{
    for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        u32 c = ids[q];
        if (c < K) atomicAdd(&counts[c], 1u);
        else atomicOr(err, 1u);
    }
}

// Exclusive prefix sum of counts[0..K) into cstart[0..K] and reset fill.
// One CTA of 1024 threads, each owning a contiguous run.
__global__ void __launch_bounds__(1024) k_scan_clusters(const u32 *counts, u32 K, u32 *cstart, u32 *fill)
{
    __shared__ u32 part[1024];
    const u32 per = (K + 1023) / 1024;
    const u32 b = threadIdx.x * per, e = min(K, b + per);
    u32 s = 0;
    for (u32 i = b; i < e; i++) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        u32 add = threadIdx.x >= (u32)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    u32 run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (u32 i = b; i < e; i++) {
        cstart[i] = run;
        fill[i] = 0;
        run += counts[i];
    }
    if (threadIdx.x == 1023) cstart[K] = part[1023];
}

__global__ void k_scatter(const u32 *ids, u32 n, u32 K, const u32 *cstart, u32 *fill, u32 *sorted_q)
{
    for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        u32 c = ids[q];
        if (c < K) sorted_q[cstart[c] + atomicAdd(&fill[c], 1u)] = q;
    }
}

// Wave positions [wave_begin, wave_begin + wave_len) of the cluster-sorted
// order, clipped to the valid queries: fill the per-wave arrays.
__global__ void k_gather_wave(WavePlan wp, const u32 *sorted_q, const u32 *ids, const u32 *cstart, u32 K,
                              u32 wave_begin, u32 wave_len, const u64 *cts, const u64 *keys, const u32 *input_index,
                              const u64 *out_offsets, u64 *out, size_t ct_words, size_t keys_words)
{
    const u32 valid = cstart[K];
    const u32 end = min(valid, wave_begin + wave_len);
    const u32 nw = end > wave_begin ? end - wave_begin : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) wp.counts[0] = nw;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        u32 q = sorted_q[wave_begin + i];
        u32 src = input_index ? input_index[q] : q;
        wp.cluster[i] = ids[q];
        wp.src_ct[i] = cts + (size_t)src * ct_words;
        wp.src_key[i] = keys + (size_t)src * keys_words;
        wp.dst_out[i] = out + out_offsets[q] * ct_words;
    }
}

// Segments (maximal runs of one cluster) and (query, chunk) pairs of a wave
// whose positions are grouped by cluster.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_wave_plan(WavePlan wp, const u32 *cluster_chunks)
{
    __shared__ u32 part[1024];
    __shared__ u32 nseg;
    const u32 nw = wp.counts[0];
    if (threadIdx.x == 0) nseg = 0;
    const u32 per = (nw + 1023) / 1024;
    const u32 b = threadIdx.x * per, e = min(nw, b + per);
    u32 s = 0;
    for (u32 i = b; i < e; i++) s += cluster_chunks[wp.cluster[i]];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        u32 add = threadIdx.x >= (u32)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    u32 run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (u32 i = b; i < e; i++) {
        u32 c = wp.cluster[i];
        u32 m = cluster_chunks[c];
        wp.pair_off[i] = run;
        for (u32 k = 0; k < m; k++) {
            wp.pair_pos[run + k] = i;
            wp.pair_k[run + k] = k;
        }
        run += m;
        if (i == 0 || wp.cluster[i - 1] != c) {
            u32 sidx = atomicAdd(&nseg, 1u);
            u32 end = i + 1;
            while (end < nw && wp.cluster[end] == c) end++;
            wp.seg_cluster[sidx] = c;
            wp.seg_begin[sidx] = i;
            wp.seg_end[sidx] = end;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        wp.pair_off[nw] = part[1023];
        wp.counts[1] = part[1023];
        wp.counts[2] = nseg;
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// the transform kernels may be launched with more shared memory than they
// use (fewer CTAs per SM): up to 225 KB, which with their static shared
// memory stays within the 227 KB a CTA may opt in to
constexpr size_t kMaxDynSmem = 225 * 1024;

template <int LOGN>
cudaError_t set_attrs_logn()
{
    const size_t sb = kMaxDynSmem;
    cudaError_t e = cudaSuccess;
#define SA(k) if (e == cudaSuccess) e = set_smem(k<LOGN>, sb)
    SA(k_to_ntt);
    SA(k_from_ntt);
    SA(k_ks_a);
    SA(k_ks_b);
    SA(k_ks_c);
    SA(k_ks_b_reg);
    SA(k_ks_c_reg);
    SA(k_output);
#undef SA
    return e;
}

}  // namespace

#define DISPATCH_LOGN(log_n, CALL)                  \
    switch (log_n) {                                \
    case 12: { constexpr int LG = 12; CALL; break; } \
    case 13: { constexpr int LG = 13; CALL; break; } \
    case 14: { constexpr int LG = 14; CALL; break; } \
    default: return cudaErrorInvalidValue;          \
    }

// dynamic shared memory of a transform kernel: its need, or the tuned size
#define SMEM(LG) (dp.ntt_smem > (8u << LG) ? (size_t)dp.ntt_smem : (size_t)8 << LG)
#define SMEM_OLD(LG) (dp.ntt_smem > ntt_smem_words<LG>() * 8 ? (size_t)dp.ntt_smem : (size_t)ntt_smem_words<LG>() * 8)
static inline int ntt_threads(int log_n) { return (1 << log_n) / 32; }

cudaError_t set_client_kernel_attributes(int log_n);

cudaError_t set_kernel_attributes(int log_n, u32 g)
{
    cudaError_t e;
    DISPATCH_LOGN(log_n, e = set_attrs_logn<LG>());
    if (e == cudaSuccess) e = set_client_kernel_attributes(log_n);
    if (e != cudaSuccess) return e;
    (void)g;
    e = set_smem(k_mac<16, 2>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac_halves<16>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac_halves<8>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac_halves<4>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac<8, 2>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac<4, 2>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac<32, 1>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac_wide, 64 * 1024);
    return e;
}

size_t ntt_smem_need(int log_n)
{
    switch (log_n) {
    case 12: return ntt_smem_words<12>() * 8;
    case 13: return ntt_smem_words<13>() * 8;
    case 14: return ntt_smem_words<14>() * 8;
    default: return 0;
    }
}

// The parameter block is read from device memory by every kernel.
static inline const DevParams *device_params_of(const DevParams &dp) { return dp.self; }

struct ProfScope {
    Profiler *pr;
    int kind;
    cudaStream_t st;
    ProfScope(Profiler *p, int k, cudaStream_t s) : pr(p), kind(k), st(s)
    {
        if (pr) pr->begin(kind, st);
    }
    ~ProfScope()
    {
        if (pr) pr->end(kind, st);
    }
};

cudaError_t launch_to_ntt(const DevParams &dp, const u64 *const *src_ptrs, const u64 *src, size_t src_stride,
                          u64 *dst, size_t dst_stride, u32 polys, u32 mod_cycle, u32 n_max, const u32 *n_dev,
                          bool mont, cudaStream_t st, Profiler *pr)
{
    if (n_max == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    dim3 grid(n_max, polys);
    ProfScope ps(pr, KK_TO_NTT, st);
    DISPATCH_LOGN(dp.log_n, (k_to_ntt<LG><<<grid, ntt_threads(LG), SMEM(LG), st>>>(
                                dpp, src_ptrs, src, src_stride, dst, dst_stride, mod_cycle, n_max, n_dev, mont)));
    return cudaGetLastError();
}

cudaError_t launch_from_ntt(const DevParams &dp, const u64 *src, u64 *dst, u32 polys, u32 mod_cycle, u32 n_items,
                            cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    dim3 grid(n_items, polys);
    DISPATCH_LOGN(dp.log_n, (k_from_ntt<LG><<<grid, ntt_threads(LG), SMEM(LG), st>>>(dpp, src, dst, polys, mod_cycle)));
    return cudaGetLastError();
}

cudaError_t launch_rotate(const DevParams &dp, const RotArgs &a, cudaStream_t st, Profiler *pr)
{
    if (a.n_max == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    const int L = dp.L;
    DISPATCH_LOGN(dp.log_n, ({
                      if (!a.prepared) {
                          ProfScope ps(pr, KK_KS_A, st);
                          k_ks_a<LG><<<a.n_max * 2 * L, ntt_threads(LG), SMEM(LG), st>>>(dpp, a);
                      }
                      if (dp.ks_core == 1) {
                          {
                              ProfScope ps(pr, KK_KS_B, st);
                              k_ks_b_reg<LG><<<a.n_max * (L + 1), ntt_threads(LG), SMEM(LG), st>>>(dpp, a);
                          }
                          ProfScope ps(pr, KK_KS_C, st);
                          k_ks_c_reg<LG><<<a.n_max * 2 * L, ntt_threads(LG), SMEM(LG), st>>>(dpp, a);
                      } else {
                          {
                              ProfScope ps(pr, KK_KS_B, st);
                              k_ks_b<LG><<<a.n_max * (L + 1), ntt_threads(LG), SMEM_OLD(LG), st>>>(dpp, a);
                          }
                          ProfScope ps(pr, KK_KS_C, st);
                          k_ks_c<LG><<<a.n_max * 2 * L, ntt_threads(LG), SMEM_OLD(LG), st>>>(dpp, a);
                      }
                  }));
    return cudaGetLastError();
}

cudaError_t launch_mac(const DevParams &dp, const ClusterStore &cs, const WavePlan &wp, const u64 *ctp, u64 *T,
                       u32 max_wave, u32 m_max, int num_sms, cudaStream_t st, Profiler *pr)
{
    const DevParams *dpp = device_params_of(dp);
    const size_t smem = (size_t)dp.d_pad * cs.ts * 8;
    // upper bound of work items: segments <= queries in the wave
    const u64 tiles = (u64)dp.n / cs.ts;
    u64 items = (u64)max_wave * m_max * dp.L * tiles;
    u64 grid = (u64)num_sms * (dp.mac_ctas_per_sm ? dp.mac_ctas_per_sm : 3);
    if (grid > items) grid = items;
    if (grid == 0) return cudaSuccess;
    ProfScope ps(pr, KK_MAC, st);
    const bool halves = dp.mac_halves && cs.ts % 4 == 0 && 256 % (cs.ts / 2) == 0;
    switch (dp.g) {
    case 4:
        if (halves) k_mac_halves<4><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        else k_mac<4, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        break;
    case 8:
        if (halves) k_mac_halves<8><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        else k_mac<8, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        break;
    case 16:
        if (halves) k_mac_halves<16><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        else k_mac<16, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        break;
    case 32: k_mac<32, 1><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max); break;
    default:
        if (128 % cs.ts) return cudaErrorInvalidValue;
        k_mac_wide<<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_output(const DevParams &dp, const WavePlan &wp, const u64 *S, size_t S_stride, u32 n_max,
                          cudaStream_t st, Profiler *pr)
{
    if (n_max == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    ProfScope ps(pr, KK_OUTPUT, st);
    DISPATCH_LOGN(dp.log_n, (k_output<LG><<<dim3(n_max, 2 * dp.L), ntt_threads(LG), SMEM(LG), st>>>(dpp, wp, S,
                                                                                                    S_stride, n_max)));
    return cudaGetLastError();
}

cudaError_t launch_group(const u32 *ids, u32 n, u32 num_clusters, u32 *counts, u32 *cstart, u32 *fill,
                         u32 *sorted_q, u32 *err, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(u32) * num_clusters, st);
    if (e != cudaSuccess) return e;
    const u32 blocks = n ? (n + 255) / 256 : 1;
    const u32 gb = blocks > 4096 ? 4096 : blocks;
    k_hist<<<gb, 256, 0, st>>>(ids, n, num_clusters, counts, err);
    k_scan_clusters<<<1, 1024, 0, st>>>(counts, num_clusters, cstart, fill);
    k_scatter<<<gb, 256, 0, st>>>(ids, n, num_clusters, cstart, fill, sorted_q);
    return cudaGetLastError();
}

cudaError_t launch_gather_wave(const WavePlan &wp, const u32 *sorted_q, const u32 *ids, const u32 *cstart,
                               u32 num_clusters, u32 wave_begin, u32 wave_len, const u64 *cts, const u64 *keys,
                               const u32 *input_index, const u64 *out_offsets, u64 *out, size_t ct_words,
                               size_t keys_words, cudaStream_t st)
{
    const u32 blocks = (wave_len + 255) / 256;
    k_gather_wave<<<blocks ? blocks : 1, 256, 0, st>>>(wp, sorted_q, ids, cstart, num_clusters, wave_begin, wave_len,
                                                        cts, keys, input_index, out_offsets, out, ct_words,
                                                        keys_words);
    return cudaGetLastError();
}

cudaError_t launch_wave_plan(const WavePlan &wp, const u32 *cluster_chunks, u32, cudaStream_t st, Profiler *pr)
{
    ProfScope ps(pr, KK_PLAN, st);
    k_wave_plan<<<1, 1024, 0, st>>>(wp, cluster_chunks);
    return cudaGetLastError();
}

}  // namespace wally
