// kernels.cu -- device kernels of the Wally GB300 library.
//
// Paper steps (arXiv 2406.06761) and where they run:
//   a0 grouping of the batch by cluster ......... k_hist / k_scan_clusters / k_scatter, k_gather_wave, k_wave_plan
//   a1 inputs to NTT form ....................... k_to_ntt
//   a2/a4 rotations Rot_k (Sec. 2 CtRotate, hybrid key switching Sec. 7)
//        ......................................... k_ks_a (automorphism + INTT of c1 -> digits)
//                                                  k_ks_b (digit NTTs + inner product with the key)
//                                                  k_ks_c (ModDown, + sigma(c0), + T_i for Horner)
//   a3 plaintext x ciphertext products (Alg. "Server Computation") ... k_mac
//   a5 output to coefficient form ............... k_output
//   setup: cluster encoding (Alg. "Server Initialization") ... k_encode_cluster
//   client side: k_encode_query, k_encrypt, k_keygen, k_decrypt_*
#include <cstdio>
#include "kernels.hpp"

namespace wally {

namespace {

template <int LOGN>
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

#define NTT_LB(LOGN) __launch_bounds__(NttShape<LOGN>::T, NttShape<LOGN>::MIN_BLOCKS)
#define NTT_LB_WIDE(LOGN) __launch_bounds__(NttShape<LOGN>::T)

// ---------------------------------------------------------------- a1: to NTT form
// Item x, polynomial z (modulus z % mod_cycle): forward NTT of the input
// (coefficients < 4p), canonical output, optionally times 2^64 (Montgomery).
template <int LOGN>
__global__ void NTT_LB(LOGN) k_to_ntt(const DevParams *dpp, const u64 *const *src_ptrs, const u64 *src,
                                      size_t src_stride, u64 *dst, size_t dst_stride, u32 mod_cycle, u32 n_max,
                                      const u32 *n_dev, bool mont)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 x = blockIdx.x;
    if (x >= item_count(n_max, n_dev)) return;
    const u32 z = blockIdx.y;
    load_mod<LOGN>(&md, dpp, z % mod_cycle);
    const u64 *s = (src_ptrs ? src_ptrs[x] : src + x * src_stride) + (size_t)z * N;
    u64 *d = dst + x * dst_stride + (size_t)z * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        sm[pidx(e)] = s[e];
    }
    ntt_fwd<LOGN>(sm, md);
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        u64 v = fwd_finish(sm[pidx(e)], md);
        d[e] = mont ? mont_mul(v, md.r2, md) : v;
    }
}

// Inverse NTT, canonical coefficients.
template <int LOGN>
__global__ void NTT_LB(LOGN) k_from_ntt(const DevParams *dpp, const u64 *src, u64 *dst, u32 polys, u32 mod_cycle)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 x = blockIdx.x, z = blockIdx.y;
    load_mod<LOGN>(&md, dpp, z % mod_cycle);
    const u64 *s = src + ((size_t)x * polys + z) * N;
    u64 *d = dst + ((size_t)x * polys + z) * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        sm[pidx(e)] = s[e];
    }
    ntt_inv<LOGN>(sm, md);
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        d[e] = inv_finish(sm[pidx(e)], md);
    }
}

// ---------------------------------------------------------------- a2/a4: rotations
// k_ks_a, CTA (item x, limb i): sigma_k on limb i of both components (a
// permutation in the NTT domain), written to sc; INTT of sigma(c1)_i gives the
// digit d_i = [sigma(c1)]_{q_i} in [0, q_i) (reading R3: non-centred).
template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_a(const DevParams *dpp, RotArgs a)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 x = blockIdx.x;
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int i = blockIdx.y, L = dpp->L;
    load_mod<LOGN>(&md, dpp, i);
    const u64 *src = a.src + x * a.src_stride;
    u64 *sc = a.sc + (size_t)x * 2 * L * N;
    for (int c = 0; c < 2; c++) {
        const u64 *s = src + ((size_t)c * L + i) * N;
        __syncthreads();
#pragma unroll 8
        for (int u = 0; u < 32; u++) {
            int e = threadIdx.x + T * u;
            sm[pidx(e)] = s[e];
        }
        __syncthreads();
        u64 v[32];
#pragma unroll
        for (int u = 0; u < 32; u++) {
            int e = threadIdx.x + T * u;
            v[u] = sm[pidx(galois_src(e, a.galois, LOGN))];
        }
        u64 *dsc = sc + ((size_t)c * L + i) * N;
#pragma unroll
        for (int u = 0; u < 32; u++) dsc[threadIdx.x + T * u] = v[u];
        if (c == 1) {
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 32; u++) sm[pidx(threadIdx.x + T * u)] = v[u];
            ntt_inv<LOGN>(sm, md);
            u64 *dd = a.dg + ((size_t)x * L + i) * N;
#pragma unroll 8
            for (int u = 0; u < 32; u++) {
                int e = threadIdx.x + T * u;
                dd[e] = inv_finish(sm[pidx(e)], md);
            }
        }
    }
}

// k_ks_b, CTA (item x, modulus j in q_0..q_{L-1}, P): u_j = sum_i NTT_j(d_i) * key_{i,j}
// for both key components.  For j = P the sums are brought back to
// coefficients (r = [u]_P) for ModDown.
template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_b(const DevParams *dpp, RotArgs a)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 x = blockIdx.x;
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int j = blockIdx.y, L = dpp->L;
    load_mod<LOGN>(&md, dpp, j);
    const u64 *kx = a.key + (size_t)(a.key_map ? a.key_map[x] : x) * a.key_stride;
    u64 *u0 = a.u + ((size_t)x * 2 + 0) * (L + 1) * N + (size_t)j * N;
    u64 *u1 = a.u + ((size_t)x * 2 + 1) * (L + 1) * N + (size_t)j * N;
    const u64 p = md.p;
    for (int i = 0; i < L; i++) {
        const u64 *kb = kx + (((size_t)i * 2 + 0) * (L + 1) + j) * N;
        const u64 *ka = kx + (((size_t)i * 2 + 1) * (L + 1) + j) * N;
        const u64 *D = nullptr;
        if (i == j) {
            D = a.sc + ((size_t)x * 2 * L + L + i) * N;  // sigma(c1)_i, already NTT form mod q_i
        } else {
            const u64 *dg = a.dg + ((size_t)x * L + i) * N;
            __syncthreads();
#pragma unroll 8
            for (int u = 0; u < 32; u++) {
                int e = threadIdx.x + T * u;
                sm[pidx(e)] = dg[e];  // < q_i < 4p_j
            }
            ntt_fwd<LOGN>(sm, md);
        }
#pragma unroll 4
        for (int u = 0; u < 32; u++) {
            int e = threadIdx.x + T * u;
            u64 d = D ? D[e] : sm[pidx(e)];
            u64 t0 = mont_mul(d, kb[e], md), t1 = mont_mul(d, ka[e], md);
            if (i > 0) {
                t0 = addmod(t0, u0[e], p);
                t1 = addmod(t1, u1[e], p);
            }
            u0[e] = t0;
            u1[e] = t1;
        }
    }
    if (j == L) {
        for (int c = 0; c < 2; c++) {
            u64 *uc = c ? u1 : u0;
            __syncthreads();
#pragma unroll 8
            for (int u = 0; u < 32; u++) {
                int e = threadIdx.x + T * u;
                sm[pidx(e)] = uc[e];
            }
            ntt_inv<LOGN>(sm, md);
#pragma unroll 8
            for (int u = 0; u < 32; u++) {
                int e = threadIdx.x + T * u;
                uc[e] = inv_finish(sm[pidx(e)], md);
            }
        }
    }
}

// k_ks_c, CTA (item x, limb j): ModDown (reading R4: round to nearest through
// the centred residue r_c of u mod P): u'_j = (u_j - NTT_j(r_c)) * P^-1, then
// out = (sigma(c0)_j + u0'_j [+ T0_j], u1'_j [+ T1_j]).
template <int LOGN>
__global__ void NTT_LB(LOGN) k_ks_c(const DevParams *dpp, RotArgs a)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 x = blockIdx.x;
    if (x >= item_count(a.n_max, a.n_dev)) return;
    const int j = blockIdx.y, L = dpp->L;
    load_mod<LOGN>(&md, dpp, j);
    const u64 q = md.p, P = dpp->m[L].p, half = (P - 1) / 2;
    const u64 pinv = dpp->pinv[j], pinv_s = dpp->pinv_s[j];
    for (int c = 0; c < 2; c++) {
        const u64 *r = a.u + (((size_t)x * 2 + c) * (L + 1) + L) * N;
        __syncthreads();
#pragma unroll 8
        for (int u = 0; u < 32; u++) {
            int e = threadIdx.x + T * u;
            u64 rv = r[e];
            sm[pidx(e)] = rv > half ? q - (P - rv) : rv;  // r_c mod q_j, value < 4q
        }
        ntt_fwd<LOGN>(sm, md);
        const u64 *uj = a.u + (((size_t)x * 2 + c) * (L + 1) + j) * N;
        const u64 *s0 = a.sc + ((size_t)x * 2 * L + j) * N;
        const u64 *ad = a.add ? a.add + x * a.add_stride + ((size_t)c * L + j) * N : nullptr;
        u64 *dst = a.dst + x * a.dst_stride + ((size_t)c * L + j) * N;
#pragma unroll 4
        for (int u = 0; u < 32; u++) {
            int e = threadIdx.x + T * u;
            u64 R = fwd_finish(sm[pidx(e)], md);
            u64 v = csub(shoup_mul(uj[e] + q - R, pinv, pinv_s, q), q);
            if (c == 0) v = addmod(v, s0[e], q);
            if (ad) v = addmod(v, ad[e], q);
            dst[e] = v;
        }
    }
}

// ---------------------------------------------------------------- a3: PtCt products
// For every (segment of one cluster in the wave, chunk k, limb l, tile of ts
// slot positions): load the tile of P'_{k,i,b} (d_pad x ts words) into shared
// memory once, then for every query of the segment
//   T_i[c] = sum_b P'_{k,i,b} * ct'[b][c]  (i < h, c = 0, 1)
// with 128-bit lazy accumulation and one Montgomery reduction per output
// (plaintexts are stored times 2^64, Sec. 7 lazy reduction).
template <int G, int CPT>
__global__ void __launch_bounds__(256) k_mac(const DevParams *dpp, ClusterStore cs, WavePlan wp, const u64 *ctp,
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
        for (u32 pos = sb + ql; pos < se; pos += QL) {
            const u64 *cq = ctp + (size_t)pos * G * ctw + (size_t)l * N + s;
            u64 cb[G][CPT];
#pragma unroll
            for (int b = 0; b < G; b++)
#pragma unroll
                for (int c = 0; c < CPT; c++) cb[b][c] = cq[(size_t)b * ctw + (size_t)(c + comp) * L * N];
            const u32 p = wp.pair_off[pos] + k;
            u64 *to = Tout + (size_t)p * h * ctw + (size_t)l * N + s;
            for (int i = 0; i < h; i++) {
                u64 hi[CPT], lo[CPT];
#pragma unroll
                for (int c = 0; c < CPT; c++) hi[c] = lo[c] = 0;
                const u64 *prow = sm + (size_t)i * G * ts + slot_in;
#pragma unroll
                for (int b = 0; b < G; b++) {
                    const u64 pv = prow[b * ts];
#pragma unroll
                    for (int c = 0; c < CPT; c++) mac128(hi[c], lo[c], pv, cb[b][c]);
                }
#pragma unroll
                for (int c = 0; c < CPT; c++) to[(size_t)i * ctw + (size_t)(c + comp) * L * N] = mont_redc(hi[c], lo[c], md);
            }
        }
    }
}

// ---------------------------------------------------------------- a5: output
template <int LOGN>
__global__ void NTT_LB(LOGN) k_output(const DevParams *dpp, WavePlan wp, const u64 *S, size_t S_stride, u32 n_max)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    extern __shared__ u64 sm[];
    __shared__ Mod md;
    const u32 p = blockIdx.x;
    if (p >= item_count(n_max, wp.counts + 1)) return;
    const int L = dpp->L;
    const int z = blockIdx.y, l = z % L;
    load_mod<LOGN>(&md, dpp, l);
    const u64 *s = S + p * S_stride + (size_t)z * N;
    u64 *d = wp.dst_out[wp.pair_pos[p]] + (size_t)wp.pair_k[p] * 2 * L * N + (size_t)z * N;
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        sm[pidx(e)] = s[e];
    }
    ntt_inv<LOGN>(sm, md);
#pragma unroll 8
    for (int u = 0; u < 32; u++) {
        int e = threadIdx.x + T * u;
        d[e] = inv_finish(sm[pidx(e)], md);
    }
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

template <int LOGN>
cudaError_t set_attrs_logn()
{
    const size_t sb = smem_words(1 << LOGN) * 8;
    cudaError_t e = cudaSuccess;
#define SA(k) if (e == cudaSuccess) e = set_smem(k<LOGN>, sb)
    SA(k_to_ntt);
    SA(k_from_ntt);
    SA(k_ks_a);
    SA(k_ks_b);
    SA(k_ks_c);
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

static inline size_t smem_bytes(int log_n) { return smem_words(1 << log_n) * 8; }
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
    if (e == cudaSuccess) e = set_smem(k_mac<8, 2>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac<4, 2>, 64 * 1024);
    if (e == cudaSuccess) e = set_smem(k_mac<32, 1>, 64 * 1024);
    return e;
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
    DISPATCH_LOGN(dp.log_n, (k_to_ntt<LG><<<grid, ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, src_ptrs, src, src_stride, dst, dst_stride, mod_cycle, n_max, n_dev, mont)));
    return cudaGetLastError();
}

cudaError_t launch_from_ntt(const DevParams &dp, const u64 *src, u64 *dst, u32 polys, u32 mod_cycle, u32 n_items,
                            cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    dim3 grid(n_items, polys);
    DISPATCH_LOGN(dp.log_n, (k_from_ntt<LG><<<grid, ntt_threads(LG), smem_bytes(LG), st>>>(dpp, src, dst, polys,
                                                                                              mod_cycle)));
    return cudaGetLastError();
}

cudaError_t launch_rotate(const DevParams &dp, const RotArgs &a, cudaStream_t st, Profiler *pr)
{
    if (a.n_max == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    const int L = dp.L;
    DISPATCH_LOGN(dp.log_n, ({
                      {
                          ProfScope ps(pr, KK_KS_A, st);
                          k_ks_a<LG><<<dim3(a.n_max, L), ntt_threads(LG), smem_bytes(LG), st>>>(dpp, a);
                      }
                      {
                          ProfScope ps(pr, KK_KS_B, st);
                          k_ks_b<LG><<<dim3(a.n_max, L + 1), ntt_threads(LG), smem_bytes(LG), st>>>(dpp, a);
                      }
                      {
                          ProfScope ps(pr, KK_KS_C, st);
                          k_ks_c<LG><<<dim3(a.n_max, L), ntt_threads(LG), smem_bytes(LG), st>>>(dpp, a);
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
    u64 grid = (u64)num_sms * 3;
    if (grid > items) grid = items;
    if (grid == 0) return cudaSuccess;
    ProfScope ps(pr, KK_MAC, st);
    switch (dp.g) {
    case 4: k_mac<4, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max); break;
    case 8: k_mac<8, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max); break;
    case 16: k_mac<16, 2><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max); break;
    case 32: k_mac<32, 1><<<(unsigned)grid, 256, smem, st>>>(dpp, cs, wp, ctp, T, m_max); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_output(const DevParams &dp, const WavePlan &wp, const u64 *S, size_t S_stride, u32 n_max,
                          cudaStream_t st, Profiler *pr)
{
    if (n_max == 0) return cudaSuccess;
    const DevParams *dpp = device_params_of(dp);
    ProfScope ps(pr, KK_OUTPUT, st);
    DISPATCH_LOGN(dp.log_n, (k_output<LG><<<dim3(n_max, 2 * dp.L), ntt_threads(LG), smem_bytes(LG), st>>>(
                                dpp, wp, S, S_stride, n_max)));
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
