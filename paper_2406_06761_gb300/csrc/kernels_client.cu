// kernels_client.cu -- set-up and client-side kernels of the Wally GB300
// library: cluster encoding (Alg. "Server Initialization"), its export back to
// coefficient form, and the client operations of Sec. 2 / Alg. "Client Query
// Generation" (query encoding, encryption, Galois keys, decryption).  Only the
// cluster encoding also runs on the server path, when the compact cluster
// store encodes each wave's chunks on the fly.
#include "kernels.hpp"
#include "pir.hpp"

namespace wally {

namespace {

typedef unsigned char u8_t;


__device__ __forceinline__ void load_mod(Mod *s, const DevParams *dpp, int j)
{
    if (threadIdx.x < sizeof(Mod) / 8) ((u64 *)s)[threadIdx.x] = ((const u64 *)&dpp->m[j])[threadIdx.x];
    __syncthreads();
}

#define NTT_LB(LOGN) __launch_bounds__(NttShape<LOGN>::T, NttShape<LOGN>::MIN_BLOCKS)
#define NTT_LB_WIDE(LOGN) __launch_bounds__(NttShape<LOGN>::T)

// ---------------------------------------------------------------- setup: cluster encoding
// CTA (plaintext (i, b), global chunk z): the slot vector of P'_{k,i,b}
// (diagonal j = g*i + b of the chunk's slices, rotated right by g*i within
// each row; Alg. "Server Initialization", Sec. 4.1) scattered to the NTT
// positions mod t, inverse NTT mod t (slot decoding), centred lift (reading
// R9), then per limb: forward NTT mod q_l, times 2^64, tile layout.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_encode_cluster(const DevParams *dpp, EncodeArgs a)
{
    constexpr int N = 1 << LOGN, T = N / 32, HALF = N / 2;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 z = blockIdx.y, ib = blockIdx.x;
    const int L = dpp->L;
    const u32 g = dpp->g, d = dpp->d, dpad = dpp->d_pad;
    const u32 i = ib / g, b = ib % g, j = g * i + b, shift = (g * i) % HALF;
    const u32 c = a.chunk_cluster[z], k = a.chunk_k[z], size = a.size[c];
    const u64 row0 = a.row0[c];
    if (a.chunk0_out && ib == 0 && k == 0 && threadIdx.x == 0) a.chunk0_out[c] = z;
    load_mod(&md, dpp, L + 1);
    const u64 t = md.p;
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const u32 s = threadIdx.x + T * u;
        const u32 rho = s / HALF, col = s % HALF;
        const u32 src = rho * HALF + (col + HALF - shift) % HALF;
        const u32 xx = src % dpad, cc = (xx + j) % dpad;
        const u64 ue = (u64)k * N + src;
        long v = (ue < size && cc < d) ? (long)a.emb[(row0 + ue) * d + cc] : 0;
        sm[spos(dpp->slot_pos[s])] = v < 0 ? (u64)(v + (long)t) : (u64)v;
    }
    ntt_inv<LOGN>(sm, twi, md);
    u64 mc[32];
#pragma unroll
    for (int u = 0; u < 32; u++) mc[u] = inv_finish(sm[spos(threadIdx.x + T * u)], md);
    const u32 ts = a.ts, tiles = N / ts;
    for (int l = 0; l < L; l++) {
        __syncthreads();
        load_mod(&md, dpp, l);
        const u64 q = md.p;
#pragma unroll
        for (int u = 0; u < 32; u++) sm[spos(threadIdx.x + T * u)] = mc[u] > (t - 1) / 2 ? q - (t - mc[u]) : mc[u];
        ntt_fwd<LOGN>(sm, twf, md);
        u64 *base = a.ptxt + ((size_t)z * L + l) * tiles * ((size_t)dpad * ts);
#pragma unroll 4
        for (int u = 0; u < 32; u++) {
            const u32 e = threadIdx.x + T * u;
            u64 v = mont_mul(fwd_finish(sm[spos(e)], md), md.r2, md);
            base[(size_t)(e / ts) * dpad * ts + (size_t)ib * ts + e % ts] = v;
        }
    }
}

// Back to coefficient form: CTA (plaintext ib, limb l, chunk k of the cluster).
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_export_cluster(const DevParams *dpp, ClusterStore cs, u32 cluster, u64 *out)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 ib = blockIdx.x, l = blockIdx.y, k = blockIdx.z;
    const int L = dpp->L;
    const u32 dpad = dpp->d_pad, ts = cs.ts, tiles = N / ts;
    load_mod(&md, dpp, l);
    const u32 zz = cs.chunk0[cluster] + k;
    const u64 *base = cs.ptxt + ((size_t)zz * L + l) * tiles * ((size_t)dpad * ts);
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const u32 e = threadIdx.x + T * u;
        sm[spos(e)] = mont_redc(0, base[(size_t)(e / ts) * dpad * ts + (size_t)ib * ts + e % ts], md);
    }
    ntt_inv<LOGN>(sm, twi, md);
    u64 *d = out + (((size_t)k * dpad + ib) * L + l) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const u32 e = threadIdx.x + T * u;
        d[e] = inv_finish(sm[spos(e)], md);
    }
}

// ---------------------------------------------------------------- client side
// Slot vector of the replicated query (slot beta*d_pad + x holds q[x] for
// x < d) -> plaintext polynomial mod t.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_encode_query(const DevParams *dpp, const int8_t *queries, u64 *m_out)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int L = dpp->L;
    const u32 d = dpp->d, dpad = dpp->d_pad;
    load_mod(&md, dpp, L + 1);
    const u64 t = md.p;
    const int8_t *qv = queries + (size_t)n * d;
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const u32 s = threadIdx.x + T * u, xx = s % dpad;
        long v = xx < d ? (long)qv[xx] : 0;
        sm[spos(dpp->slot_pos[s])] = v < 0 ? (u64)(v + (long)t) : (u64)v;
    }
    ntt_inv<LOGN>(sm, twi, md);
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const u32 e = threadIdx.x + T * u;
        m_out[(size_t)n * N + e] = inv_finish(sm[spos(e)], md);
    }
}

// sm <- NTT(a) * NTT(s) brought back by INTT: the negacyclic product a*s mod p.
// sv holds NTT(s) for the thread's 32 positions.
template <int LOGN>
__device__ __forceinline__ void poly_times_secret(u64 *sm, const u64 sv[32], const Mod &md, Tw *twf,
                                                  Tw *twi)
{
    constexpr int T = (1 << LOGN) / 32;
    ntt_fwd<LOGN>(sm, twf, md);
#pragma unroll
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = mulmod(fwd_finish(sm[spos(e)], md), sv[u], md);
    }
    ntt_inv<LOGN>(sm, twi, md);
}

template <int LOGN>
__device__ __forceinline__ void secret_ntt(u64 *sm, u64 sv[32], const int8_t *s, const Mod &md, Tw *twf)
{
    constexpr int T = (1 << LOGN) / 32;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        const int v = s[e];
        sm[spos(e)] = v < 0 ? md.p - 1 : (u64)v;
    }
    ntt_fwd<LOGN>(sm, twf, md);
#pragma unroll
    for (int u = 0; u < 32; u++) sv[u] = fwd_finish(sm[spos(threadIdx.x + T * u)], md);
    __syncthreads();
}

// CTA (client n, limb l): c1 = a, c0 = -a*s + e + Delta*m (reading R1).
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_encrypt(const DevParams *dpp, const int8_t *secret, const u64 *m, const u64 *enc_a,
                                       const int8_t *enc_e, u64 *cts)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int l = blockIdx.y, L = dpp->L;
    load_mod(&md, dpp, l);
    const u64 q = md.p;
    u64 sv[32];
    secret_ntt<LOGN>(sm, sv, secret + (size_t)n * N, md, twf);
    const u64 *a = enc_a + ((size_t)n * L + l) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = a[e];
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
    u64 *c0 = cts + ((size_t)n * 2 * L + l) * N, *c1 = cts + ((size_t)n * 2 * L + L + l) * N;
    const int8_t *ee = enc_e + (size_t)n * N;
    const u64 *mm = m + (size_t)n * N;
    const u64 dl = dpp->delta[l], dls = dpp->delta_s[l];
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        const u64 as = inv_finish(sm[spos(e)], md);
        const int ev = ee[e];
        u64 v = submod(ev < 0 ? q - (u64)(-ev) : (u64)ev, as, q);
        v = addmod(v, csub(shoup_mul(mm[e], dl, dls, q), q), q);
        c0[e] = v;
        c1[e] = a[e];
    }
}

// CTA (client n, modulus j, key kk * L + digit i): Galois key of element
// k = (kk ? kg : k1), s' = sigma_k(s):
//   b = -a*s + e + [i == j] P s'  (mod q_j),  b = -a*s + e (mod P).
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_keygen(const DevParams *dpp, const int8_t *secret, const u64 *key_a,
                                      const int8_t *key_e, KinvList kl, u64 *keys)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int j = blockIdx.y, L = dpp->L;
    const int kk = blockIdx.z / L, i = blockIdx.z % L, NK = kl.nk;
    load_mod(&md, dpp, j);
    const u64 p = md.p;
    const int8_t *s = secret + (size_t)n * N;
    u64 sv[32];
    secret_ntt<LOGN>(sm, sv, s, md, twf);
    const u64 *a = key_a + ((((size_t)n * NK + kk) * L + i) * (L + 1) + j) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = a[e];
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
    const int8_t *ee = key_e + (((size_t)n * NK + kk) * L + i) * N;
    u64 *kb = keys + (((((size_t)n * NK + kk) * L + i) * 2 + 0) * (L + 1) + j) * N;
    u64 *ka = keys + (((((size_t)n * NK + kk) * L + i) * 2 + 1) * (L + 1) + j) * N;
    const u64 kinv = kl.v[kk];
    const u32 mask2n = 2 * N - 1;
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        const u64 as = inv_finish(sm[spos(e)], md);
        const int ev = ee[e];
        u64 v = submod(ev < 0 ? p - (u64)(-ev) : (u64)ev, as, p);
        if (i == j) {
            // s'[e]: the coefficient n0 = e * k^-1 mod 2N of s moves to X^e
            // (sign + if n0 < N, else coefficient n0 - N with sign -).
            const u32 n0 = (u32)(((u64)e * kinv) & mask2n);
            int sp = n0 < (u32)N ? s[n0] : -s[n0 - N];
            const u64 pm = dpp->pmodq[j];
            if (sp > 0) v = addmod(v, pm, p);
            else if (sp < 0) v = submod(v, pm, p);
        }
        kb[e] = v;
        ka[e] = a[e];
    }
}

// Relinearisation key, CTA (client n, modulus j, digit i): the key
// switching key from s^2 to s (MulPIR's ciphertext products, Sec. 4.2):
// b_i = -a_i*s + e_i + [i == j] P s^2 (mod q_j), b_i = -a_i*s + e_i (mod P),
// with s^2 the negacyclic square of the secret, formed here mod p_j.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_relinkey(const DevParams *dpp, const int8_t *secret, const u64 *key_a,
                                        const int8_t *key_e, u64 *keys)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int j = blockIdx.y, L = dpp->L, i = blockIdx.z;
    load_mod(&md, dpp, j);
    const u64 p = md.p;
    const int8_t *s = secret + (size_t)n * N;
    u64 sv[32], s2[32];
    secret_ntt<LOGN>(sm, sv, s, md, twf);
#pragma unroll
    for (int u = 0; u < 32; u++) {
        const int v = s[threadIdx.x + T * u];
        sm[spos(threadIdx.x + T * u)] = v < 0 ? p - 1 : (u64)v;
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
#pragma unroll
    for (int u = 0; u < 32; u++) s2[u] = inv_finish(sm[spos(threadIdx.x + T * u)], md);
    __syncthreads();
    const u64 *a = key_a + (((size_t)n * L + i) * (L + 1) + j) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = a[e];
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
    const int8_t *ee = key_e + ((size_t)n * L + i) * N;
    u64 *kb = keys + ((((size_t)n * L + i) * 2 + 0) * (L + 1) + j) * N;
    u64 *ka = keys + ((((size_t)n * L + i) * 2 + 1) * (L + 1) + j) * N;
    const u64 pm = dpp->pmodq[j < L ? j : 0];
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        const u64 as = inv_finish(sm[spos(e)], md);
        const int ev = ee[e];
        u64 v = submod(ev < 0 ? p - (u64)(-ev) : (u64)ev, as, p);
        if (i == j) v = addmod(v, mulmod(pm, s2[u], md), p);
        kb[e] = v;
        ka[e] = a[e];
    }
}

// CTA (ciphertext n, limb l): x_l = [c0 + c1 s]_{q_l}, coefficient form.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_decrypt_residues(const DevParams *dpp, const int8_t *secret, const u32 *secret_index,
                                                const u64 *cts, u64 *xs)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int l = blockIdx.y, L = dpp->L;
    load_mod(&md, dpp, l);
    const u32 si = secret_index ? secret_index[n] : n;
    u64 sv[32];
    secret_ntt<LOGN>(sm, sv, secret + (size_t)si * N, md, twf);
    const u64 *c0 = cts + ((size_t)n * 2 * L + l) * N, *c1 = cts + ((size_t)n * 2 * L + L + l) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = c1[e];
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
    u64 *x = xs + ((size_t)n * L + l) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        x[e] = addmod(inv_finish(sm[spos(e)], md), c0[e], md.p);
    }
}

// CTA (ciphertext n): m = round(t x / Q) mod t from the residues x_l, then
// slot decoding (forward NTT mod t) and centring.  With y_l = x_l (Q/q_l)^-1
// mod q_l, t x / Q = sum_l y_l t / q_l - (a multiple of t), so m is the
// rounded sum of the integer parts and the 64-bit fractions of y_l t / q_l.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_decrypt_scale(const DevParams *dpp, const u64 *xs, int64_t *scores, bool slots)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int L = dpp->L;
    load_mod(&md, dpp, L + 1);
    const u64 t = md.p;
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        u64 ipart = 0;
        unsigned __int128 frac = 0;
        for (int l = 0; l < L; l++) {
            const u64 q = dpp->m[l].p;
            const u64 y = csub(shoup_mul(xs[((size_t)n * L + l) * N + e], dpp->theta[l], dpp->theta_s[l], q), q);
            const unsigned __int128 num = (unsigned __int128)y * t;
            const u64 quo = (u64)(num / q);
            const u64 rem = (u64)(num - (unsigned __int128)quo * q);
            ipart += quo;
            frac += (u64)(((unsigned __int128)rem << 64) / q);
        }
        const u64 rnd = (u64)((frac + ((unsigned __int128)1 << 63)) >> 64);
        sm[spos(e)] = (ipart + rnd) % t;
        if (!slots) scores[(size_t)n * N + e] = (int64_t)((ipart + rnd) % t);  // coefficient e of m, in [0, t)
    }
    if (!slots) return;
    ntt_fwd<LOGN>(sm, twf, md);
    for (int u = 0; u < 32; u++) {
        const int s = threadIdx.x + T * u;
        const u64 v = fwd_finish(sm[spos(dpp->slot_pos[s])], md);
        scores[(size_t)n * N + s] = v > t / 2 ? (int64_t)v - (int64_t)t : (int64_t)v;
    }
}

// ---------------------------------------------------------------- response compression
// Sec. 7 "Reducing the response size".  Per coefficient of both components:
// the chain of exact rescalings by q_0, ..., q_{L-2} (each step replaces c by
// round(c / q_i) = (c - centred [c]_{q_i}) * q_i^-1 on the remaining limbs),
// leaving the residue mod q' = q_{L-1}; then l low bits dropped with rounding
// to nearest.  Each group of 8 coefficients packs into b bytes (b bits each,
// little-endian bit order); component 0 then component 1.
__device__ __forceinline__ u64 switch_to_last_limb(const DevParams *dpp, const u64 *ct_c, int n, int N, int L)
{
    u64 v[WALLY_MAX_LIMBS];
    for (int j = 0; j < L; j++) v[j] = ct_c[(size_t)j * N + n];
    for (int i = 0; i + 1 < L; i++) {
        const u64 qi = dpp->m[i].p, r = v[i];
        const bool neg = r > (qi - 1) / 2;
        for (int j = i + 1; j < L; j++) {
            const u64 qj = dpp->m[j].p;
            // centred remainder mod q_j: |r_c| < q_i / 2 < q_j (primes of one size)
            const u64 rm = neg ? qj - (qi - r) : r;
            v[j] = csub(shoup_mul(v[j] + qj - rm, dpp->rs_inv[i][j], dpp->rs_inv_s[i][j], qj), qj);
        }
    }
    return v[L - 1];
}

__global__ void __launch_bounds__(256) k_compress(const DevParams *dpp, const u64 *cts, u8_t *out, u32 l0, u32 l1,
                                                  u32 b0, u32 b1)
{
    const int L = dpp->L, N = dpp->n;
    const u32 x = blockIdx.x;
    const u64 *ct = cts + (size_t)x * 2 * L * N;
    u8_t *o = out + (size_t)x * (N / 8) * (b0 + b1);
    for (int c = 0; c < 2; c++) {
        const u32 l = c ? l1 : l0, b = c ? b1 : b0;
        u8_t *base = o + (c ? (size_t)(N / 8) * b0 : 0);
        for (int g = threadIdx.x; g < N / 8; g += blockDim.x) {
            u64 buf = 0;
            int nb = 0;
            u8_t *dst = base + (size_t)g * b;
            for (int k = 0; k < 8; k++) {
                const u64 xv = switch_to_last_limb(dpp, ct + (size_t)c * L * N, 8 * g + k, N, L);
                const u64 val = l ? (xv + (1ull << (l - 1))) >> l : xv;
                buf |= val << nb;
                nb += b;
                while (nb >= 8) {  // fewer than 8 bits stay pending, so b <= 57 fits
                    *dst++ = (u8_t)buf;
                    buf >>= 8;
                    nb -= 8;
                }
            }
            // 8 values of b bits are exactly b bytes: nothing is left pending
        }
    }
}

// Value e (b bits) of a packed component.
__device__ __forceinline__ u64 unpack_at(const u8_t *base, int e, u32 b)
{
    const u64 bit = (u64)e * b;
    const u8_t *p = base + (bit >> 3);
    const int sh = (int)(bit & 7);
    const int nbytes = (sh + (int)b + 7) >> 3;
    u64 lo = 0, hi = 0;
    for (int i = 0; i < nbytes && i < 8; i++) lo |= (u64)p[i] << (8 * i);
    if (nbytes > 8) hi = p[8];
    u64 v = lo >> sh;
    if (sh) v |= hi << (64 - sh);
    return b >= 64 ? v : (v & ((1ull << b) - 1));
}

// CTA (response n): x = c0'' 2^l0 + c1'' 2^l1 s (mod q'), m = round(t x / q')
// mod t, slots decoded and centred.
template <int LOGN>
__global__ void NTT_LB_WIDE(LOGN) k_decrypt_compressed(const DevParams *dpp, const int8_t *secret,
                                                       const u32 *secret_index, const u8_t *packed, u32 l0, u32 l1,
                                                       u32 b0, u32 b1, int64_t *scores)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    Tw *twf = reinterpret_cast<Tw *>(sm + smem_words(1 << LOGN));
    Tw *twi = twf;  // one cache, reloaded by every transform
    __shared__ Mod md;
    const u32 n = blockIdx.x;
    const int L = dpp->L;
    load_mod(&md, dpp, L - 1);
    const u64 q = md.p;
    const u32 si = secret_index ? secret_index[n] : n;
    u64 sv[32];
    secret_ntt<LOGN>(sm, sv, secret + (size_t)si * N, md, twf);
    const u8_t *p0 = packed + (size_t)n * (N / 8) * (b0 + b1);
    const u8_t *p1 = p0 + (size_t)(N / 8) * b0;
    const u64 f1 = ((u64)1 << l1) % q, f0 = ((u64)1 << l0) % q;
    const u64 f1s = (u64)(((unsigned __int128)f1 << 64) / q), f0s = (u64)(((unsigned __int128)f0 << 64) / q);
#pragma unroll 4
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        sm[spos(e)] = csub(shoup_mul(unpack_at(p1, e, b1), f1, f1s, q), q);
    }
    poly_times_secret<LOGN>(sm, sv, md, twf, twi);
    const u64 t = dpp->m[L + 1].p;
    for (int u = 0; u < 32; u++) {
        const int e = threadIdx.x + T * u;
        const u64 c0 = csub(shoup_mul(unpack_at(p0, e, b0), f0, f0s, q), q);
        const u64 xv = addmod(c0, inv_finish(sm[spos(e)], md), q);
        sv[u] = (u64)((((unsigned __int128)t * xv) + q / 2) / q) % t;
    }
    __syncthreads();
    load_mod(&md, dpp, L + 1);
    for (int u = 0; u < 32; u++) sm[spos(threadIdx.x + T * u)] = sv[u];
    ntt_fwd<LOGN>(sm, twf, md);
    for (int u = 0; u < 32; u++) {
        const int s = threadIdx.x + T * u;
        const u64 v = fwd_finish(sm[spos(dpp->slot_pos[s])], md);
        scores[(size_t)n * N + s] = v > t / 2 ? (int64_t)v - (int64_t)t : (int64_t)v;
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int LOGN>
cudaError_t set_attrs_logn()
{
    const size_t sb = ntt_smem_words<LOGN>() * 8;
    cudaError_t e = cudaSuccess;
#define SA(k) if (e == cudaSuccess) e = set_smem(k<LOGN>, sb)
    SA(k_encode_cluster);
    SA(k_export_cluster);
    SA(k_encode_query);
    SA(k_encrypt);
    SA(k_keygen);
    SA(k_relinkey);
    SA(k_decrypt_residues);
    SA(k_decrypt_scale);
    SA(k_decrypt_compressed);
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

static inline size_t smem_bytes(int log_n)
{
    return log_n == 12 ? ntt_smem_words<12>() * 8 : log_n == 13 ? ntt_smem_words<13>() * 8 : ntt_smem_words<14>() * 8;
}
static inline int ntt_threads(int log_n) { return (1 << log_n) / 32; }

static inline const DevParams *device_params_of(const DevParams &dp) { return dp.self; }

cudaError_t set_client_kernel_attributes(int log_n)
{
    cudaError_t e;
    DISPATCH_LOGN(log_n, e = set_attrs_logn<LG>());
    return e;
}

static cudaError_t encode_dispatch(const DevParams *dpp, int log_n, dim3 grid, const EncodeArgs &a, cudaStream_t st)
{
    DISPATCH_LOGN(log_n, (k_encode_cluster<LG><<<grid, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, a)));
    return cudaGetLastError();
}

cudaError_t launch_encode_clusters(const DevParams &dp, const EncodeArgs &a, cudaStream_t st, Profiler *pr)
{
    if (a.total_chunks == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    dim3 grid(dp.g * dp.h, a.total_chunks);
    if (pr) pr->begin(KK_ENCODE, st);
    cudaError_t e = encode_dispatch(dpp, dp.log_n, grid, a, st);
    if (pr) pr->end(KK_ENCODE, st);
    return e;
}

cudaError_t launch_export_cluster(const DevParams &dp, const ClusterStore &cs, u32 cluster, u32 m, u64 *out,
                                  cudaStream_t st)
{
    const DevParams *dpp = device_params_of(dp);
    dim3 grid(dp.g * dp.h, dp.L, m);
    DISPATCH_LOGN(dp.log_n, (k_export_cluster<LG><<<grid, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, cs, cluster,
                                                                                                   out)));
    return cudaGetLastError();
}

cudaError_t launch_encode_queries(const DevParams &dp, const int8_t *queries, u32 n, u64 *m_out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, (k_encode_query<LG><<<n, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, queries, m_out)));
    return cudaGetLastError();
}

cudaError_t launch_encrypt(const DevParams &dp, const int8_t *secret, const u64 *m, const u64 *enc_a,
                           const int8_t *enc_e, u32 n, u64 *cts, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, (k_encrypt<LG><<<dim3(n, dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, secret, m, enc_a, enc_e, cts)));
    return cudaGetLastError();
}

cudaError_t launch_keygen(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e, u32 n,
                          u64, u64, u64 k1_inv, u64 kg_inv, u64 *keys, cudaStream_t st)
{
    KinvList kl;
    kl.nk = 2;
    kl.v[0] = k1_inv;
    kl.v[1] = kg_inv;
    return launch_keygen_list(dp, secret, key_a, key_e, n, kl, keys, st);
}

cudaError_t launch_keygen_list(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e,
                               u32 n, const KinvList &kl, u64 *keys, cudaStream_t st)
{
    if (n == 0 || kl.nk <= 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, (k_keygen<LG><<<dim3(n, dp.L + 1, kl.nk * dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, secret, key_a, key_e, kl, keys)));
    return cudaGetLastError();
}

cudaError_t launch_decrypt(const DevParams &dp, const int8_t *secret, const u32 *secret_index, const u64 *cts, u32 n,
                           u64 *xs, int64_t *scores, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, ({
                      k_decrypt_residues<LG><<<dim3(n, dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                          dpp, secret, secret_index, cts, xs);
                      k_decrypt_scale<LG><<<n, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, xs, scores, true);
                  }));
    return cudaGetLastError();
}

cudaError_t launch_relinkey(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e, u32 n,
                            u64 *keys, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, (k_relinkey<LG><<<dim3(n, dp.L + 1, dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, secret, key_a, key_e, keys)));
    return cudaGetLastError();
}

cudaError_t launch_decrypt_coeffs(const DevParams &dp, const int8_t *secret, const u32 *secret_index, const u64 *cts,
                                  u32 n, u64 *xs, int64_t *coeffs, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    DISPATCH_LOGN(dp.log_n, ({
                      k_decrypt_residues<LG><<<dim3(n, dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                          dpp, secret, secret_index, cts, xs);
                      k_decrypt_scale<LG><<<n, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, xs, coeffs, false);
                  }));
    return cudaGetLastError();
}

}  // namespace wally

namespace wally {
cudaError_t launch_compress(const DevParams &dp, const u64 *cts, u32 n, uint8_t *out, u32 l0, u32 l1, u32 b0, u32 b1,
                            cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_compress<<<n, 256, 0, st>>>(dp.self, cts, out, l0, l1, b0, b1);
    return cudaGetLastError();
}

cudaError_t launch_decrypt_compressed(const DevParams &dp, const int8_t *secret, const u32 *secret_index,
                                      const uint8_t *packed, u32 n, u32 l0, u32 l1, u32 b0, u32 b1, int64_t *scores,
                                      cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const DevParams *dpp = dp.self;
    DISPATCH_LOGN(dp.log_n, (k_decrypt_compressed<LG><<<n, ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, secret, secret_index, packed, l0, l1, b0, b1, scores)));
    return cudaGetLastError();
}
}  // namespace wally
