// pir.cu -- kernels of the index PIR under the keyword PIR of Sec. 4.2
// ("Details of keyword PIR": MulPIR): the server lifts the table's plaintexts
// into the ciphertext moduli, expands each query ciphertext obliviously into
// indicator ciphertexts (substitutions by N/2^a + 1 are the key switches of
// kernels.cu; this file adds the additions and the monomial X^(-2^a) of each
// level), and runs MulPIR's first dimension, sums of plaintext-ciphertext
// products over the rows of the table.
#include "pir.hpp"

namespace wally {

namespace {

__global__ void k_pir_lift(const DevParams *dpp, const u64 *src, u32 count, u64 *dst)
{
    const int L = dpp->L, N = dpp->n;
    const u64 t = dpp->m[L + 1].p;
    const size_t total = (size_t)count * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t p = idx / N;
        const int e = (int)(idx % N);
        const u64 v = src[idx];  // in [0, t): centred lift (reading R9)
        for (int l = 0; l < L; l++) {
            const u64 q = dpp->m[l].p;
            dst[(p * L + l) * N + e] = v > (t - 1) / 2 ? q - (t - v) : v;
        }
    }
}

__global__ void k_pir_qmap(u32 *map, u32 count, u32 shift)
{
    for (u32 x = blockIdx.x * blockDim.x + threadIdx.x; x < count; x += gridDim.x * blockDim.x) map[x] = x >> shift;
}

// One expansion level: C (cur) and S = sigma(C) (sig) give C + S and
// (C - S) X^(-2^a), both in NTT form (a pointwise product with the NTT of the
// monomial, stored times 2^64).
__global__ void k_pir_combine(const DevParams *dpp, const u64 *cur, const u64 *sig, u64 *next, const u64 *mono,
                              u32 count, u32 a)
{
    const int L = dpp->L, N = dpp->n;
    const size_t ctw = (size_t)2 * L * N;
    const size_t total = (size_t)count * ctw;
    const u32 lowmask = (1u << a) - 1;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const u32 x = (u32)(idx / ctw);
        const size_t r = idx % ctw;
        const int e = (int)(r % N), l = (int)((r / N) % L);
        const Mod &md = dpp->m[l];
        const u64 C = cur[idx], S = sig[idx];
        const size_t base = ((size_t)(x >> a) << (a + 1)) + (x & lowmask);
        next[base * ctw + r] = addmod(C, S, md.p);
        next[(base + (1u << a)) * ctw + r] = mont_mul(submod(C, S, md.p), mono[(size_t)l * N + e], md);
    }
}

// First dimension.  CTA (tile of 32 slots, column j and limb l, group of 4
// queries); thread (slot, component, query).  Rows are staged through shared
// memory 64 at a time; each thread keeps one lazy 128-bit sum and reduces it
// once (the table is stored times 2^64).
__global__ void __launch_bounds__(256) k_pir_dim1(const DevParams *dpp, const u64 *db, u32 rows, u32 cols,
                                                  const u64 *ind, u32 ind_stride, u32 n, u64 *out)
{
    constexpr int TS = 32, RB = 64;
    __shared__ u64 tile[RB][TS];
    const int L = dpp->L, N = dpp->n;
    const size_t ctw = (size_t)2 * L * N;
    const int ti = blockIdx.x, j = blockIdx.y / L, l = blockIdx.y % L;
    const int slot = threadIdx.x % TS, comp = (threadIdx.x / TS) & 1, qi = threadIdx.x / (2 * TS);
    const u32 q = blockIdx.z * 4 + qi;
    const int s = ti * TS + slot;
    u64 hi = 0, lo = 0;
    for (u32 r0 = 0; r0 < rows; r0 += RB) {
        const u32 rb = min((u32)RB, rows - r0);
        __syncthreads();
        for (u32 w = threadIdx.x; w < rb * TS; w += 256) {
            const u32 r = w / TS, sl = w % TS;
            tile[r][sl] = db[(((size_t)(r0 + r) * cols + j) * L + l) * N + (size_t)ti * TS + sl];
        }
        __syncthreads();
        if (q < n) {
            const u64 *ip = ind + ((size_t)q * ind_stride + r0) * ctw + (size_t)comp * L * N + (size_t)l * N + s;
            for (u32 r = 0; r < rb; r++) mac128(hi, lo, tile[r][slot], ip[(size_t)r * ctw]);
        }
    }
    if (q < n) out[((size_t)q * cols + j) * ctw + (size_t)comp * L * N + (size_t)l * N + s] = mont_redc(hi, lo, dpp->m[l]);
}

// ---- multiword integers: XW little-endian 64-bit words, non-negative
__device__ __forceinline__ void mw_zero(u64 *a)
{
#pragma unroll
    for (int i = 0; i < XW; i++) a[i] = 0;
}

// a += b * m
__device__ __forceinline__ void mw_mul_add(u64 *a, const u64 *b, u64 m)
{
    unsigned __int128 carry = 0;
#pragma unroll
    for (int i = 0; i < XW; i++) {
        const unsigned __int128 v = (unsigned __int128)b[i] * m + a[i] + carry;
        a[i] = (u64)v;
        carry = v >> 64;
    }
}

__device__ __forceinline__ int mw_cmp(const u64 *a, const u64 *b)
{
    for (int i = XW - 1; i >= 0; i--)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

// a -= b (a >= b)
__device__ __forceinline__ void mw_sub(u64 *a, const u64 *b)
{
    u64 borrow = 0;
#pragma unroll
    for (int i = 0; i < XW; i++) {
        const u64 x = a[i], y = b[i];
        const u64 d = x - y - borrow;
        borrow = (x < y) || (x == y && borrow) ? 1 : 0;
        a[i] = d;
    }
}

// a += b
__device__ __forceinline__ void mw_add(u64 *a, const u64 *b)
{
    u64 carry = 0;
#pragma unroll
    for (int i = 0; i < XW; i++) {
        const u64 s1 = a[i] + b[i];
        const u64 c1 = s1 < a[i];
        const u64 s2 = s1 + carry;
        carry = c1 | (s2 < s1);
        a[i] = s2;
    }
}

// a = floor(a / d), returns a mod d
__device__ __forceinline__ u64 mw_div_small(u64 *a, u64 d)
{
    unsigned __int128 rem = 0;
    for (int i = XW - 1; i >= 0; i--) {
        const unsigned __int128 cur = (rem << 64) | a[i];
        a[i] = (u64)(cur / d);
        rem = cur % d;
    }
    return (u64)rem;
}

__device__ __forceinline__ u64 mw_mod_small(const u64 *a, u64 d)
{
    unsigned __int128 rem = 0;
    for (int i = XW - 1; i >= 0; i--) rem = ((rem << 64) | a[i]) % d;
    return (u64)rem;
}

// 2a > b ?
__device__ __forceinline__ bool mw_twice_gt(const u64 *a, const u64 *b)
{
    u64 d[XW];
    u64 carry = 0;
#pragma unroll
    for (int i = 0; i < XW; i++) {
        d[i] = (a[i] << 1) | carry;
        carry = a[i] >> 63;
    }
    return carry || mw_cmp(d, b) > 0;
}

// Centred lift into the extension basis, one thread per coefficient: with
// y_i = [x_i theta_i]_{q_i}, S = sum_i y_i Q/q_i = A + k Q exactly
// (multiword), k chosen so that A lies in (-Q/2, Q/2]; then
// A mod b = sum_i y_i [Q/q_i]_b - k [Q]_b.
__global__ void k_lift_ext(const ExtConst *ec, const u64 *src, u32 count, u32 n, u64 *dst)
{
    const int L = ec->L, Lx = ec->Lx, Lr = ec->Lr;
    const size_t total = (size_t)count * n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t p = idx / n;
        const u32 e = (u32)(idx % n);
        u64 y[WALLY_MAX_LIMBS];
        u64 S[XW];
        mw_zero(S);
        for (int i = 0; i < L; i++) {
            const u64 x = src[(p * L + i) * n + e];
            dst[(p * Lr + i) * n + e] = x;
            y[i] = (u64)(((unsigned __int128)x * ec->theta[i]) % ec->q[i]);
            mw_mul_add(S, ec->qw[i], y[i]);
        }
        u32 k = 0;
        while (mw_cmp(S, ec->Q) >= 0) {
            mw_sub(S, ec->Q);
            k++;
        }
        if (mw_twice_gt(S, ec->Q)) k++;  // centred: A = S - Q < 0
        for (int j = 0; j < Lx; j++) {
            const u64 b = ec->b[j];
            unsigned __int128 acc = (unsigned __int128)k * (b - ec->Q_b[j]);
            for (int i = 0; i < L; i++) acc += (unsigned __int128)y[i] * ec->qdiv_b[i][j];
            dst[(p * Lr + L + j) * n + e] = (u64)(acc % b);
        }
    }
}

// Thread per (query, limb, coefficient) of the extension basis: three lazy
// 128-bit sums over the d2 pairs, reduced once.
__global__ void k_tensor_acc(const ExtConst *ec, const u64 *A, const u64 *B, u32 nq, u32 d2, u32 n, u64 *T)
{
    const int Lr = ec->Lr;
    const size_t per = (size_t)2 * Lr * n;  // one ciphertext
    const size_t total = (size_t)nq * Lr * n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const u32 q = (u32)(idx / ((size_t)Lr * n));
        const size_t le = idx % ((size_t)Lr * n);  // l * n + e
        const u64 p = ec->r[le / n];
        u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0, h2 = 0, l2 = 0;
        for (u32 j = 0; j < d2; j++) {
            const size_t base = ((size_t)q * d2 + j) * per + le;
            const u64 a0 = A[base], a1 = A[base + (size_t)Lr * n], b0 = B[base], b1 = B[base + (size_t)Lr * n];
            mac128(h0, l0, a0, b0);
            mac128(h1, l1, a0, b1);
            mac128(h1, l1, a1, b0);
            mac128(h2, l2, a1, b1);
        }
        const size_t o = (size_t)q * 3 * Lr * n + le;
        T[o] = (u64)((((unsigned __int128)h0 << 64) | l0) % p);
        T[o + (size_t)Lr * n] = (u64)((((unsigned __int128)h1 << 64) | l1) % p);
        T[o + (size_t)2 * Lr * n] = (u64)((((unsigned __int128)h2 << 64) | l2) % p);
    }
}

// Thread per (query, tensor component, coefficient): CRT over the extension
// basis to the centred integer V, then round(t V / Q) = floor((2tV + Q) / 2Q)
// by successive single-word divisions (2, q_0, ..., q_{L-1}), reduced mod q_i.
__global__ void k_scale_ext(const ExtConst *ec, const u64 *T, u32 nq, u32 n, u64 *X, u64 *ADD)
{
    const int L = ec->L, Lr = ec->Lr;
    const size_t total = (size_t)nq * 3 * n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const u32 q = (u32)(idx / ((size_t)3 * n));
        const int k = (int)((idx / n) % 3);
        const u32 e = (u32)(idx % n);
        u64 S[XW];
        mw_zero(S);
        for (int l = 0; l < Lr; l++) {
            const u64 v = T[(((size_t)q * 3 + k) * Lr + l) * n + e];
            const u64 y = (u64)(((unsigned __int128)v * ec->rinv[l]) % ec->r[l]);
            mw_mul_add(S, ec->rw[l], y);
        }
        while (mw_cmp(S, ec->R) >= 0) mw_sub(S, ec->R);
        const bool neg = mw_twice_gt(S, ec->R);
        u64 V[XW];
        if (neg) {
            for (int i = 0; i < XW; i++) V[i] = ec->R[i];
            mw_sub(V, S);  // |V| = R - S
        } else {
            for (int i = 0; i < XW; i++) V[i] = S[i];
        }
        u64 M[XW];
        mw_zero(M);
        mw_mul_add(M, V, 2 * ec->t);  // 2t |V|
        bool res_neg = false, zero = false;
        if (!neg) {
            mw_add(M, ec->Q);  // 2tV + Q >= 0: floor division
        } else if (mw_cmp(M, ec->Q) <= 0) {
            zero = true;  // 0 <= Q - 2t|V| <= Q < 2Q
        } else {
            mw_sub(M, ec->Q);      // m = 2t|V| - Q > 0
            mw_add(M, ec->twoQm1);  // ceil(m / 2Q) = floor((m + 2Q - 1) / 2Q)
            res_neg = true;
        }
        u64 res[WALLY_MAX_LIMBS];
        if (zero) {
            for (int i = 0; i < L; i++) res[i] = 0;
        } else {
            mw_div_small(M, 2);
            for (int i = 0; i < L; i++) mw_div_small(M, ec->q[i]);
            for (int i = 0; i < L; i++) {
                const u64 r = mw_mod_small(M, ec->q[i]);
                res[i] = (res_neg && r) ? ec->q[i] - r : r;
            }
        }
        // k = 0 -> c0 (X comp 0), k = 2 -> c2 (X comp 1), k = 1 -> c1 (ADD comp 1)
        for (int i = 0; i < L; i++) {
            const size_t o = ((size_t)q * 2 * L + i) * n + e;
            if (k == 0) X[o] = res[i];
            else if (k == 2) X[o + (size_t)L * n] = res[i];
            else {
                ADD[o] = 0;
                ADD[o + (size_t)L * n] = res[i];
            }
        }
    }
}

unsigned grid_for(size_t total)
{
    size_t b = (total + 255) / 256;
    return (unsigned)(b > 65535 ? 65535 : (b ? b : 1));
}

}  // namespace

cudaError_t launch_pir_lift(const DevParams &dp, const u64 *src, u32 count, u64 *dst, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    k_pir_lift<<<grid_for((size_t)count * dp.n), 256, 0, st>>>(dp.self, src, count, dst);
    return cudaGetLastError();
}

cudaError_t launch_pir_qmap(u32 *map, u32 count, u32 shift, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    k_pir_qmap<<<grid_for(count), 256, 0, st>>>(map, count, shift);
    return cudaGetLastError();
}

cudaError_t launch_pir_combine(const DevParams &dp, const u64 *cur, const u64 *sig, u64 *next, const u64 *mono,
                               u32 count, u32 a, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    k_pir_combine<<<grid_for((size_t)count * 2 * dp.L * dp.n), 256, 0, st>>>(dp.self, cur, sig, next, mono, count, a);
    return cudaGetLastError();
}

cudaError_t launch_lift_ext(const ExtConst *ec, const u64 *src, u32 count, u32 n, u64 *dst, cudaStream_t st)
{
    if (!count) return cudaSuccess;
    k_lift_ext<<<grid_for((size_t)count * n), 256, 0, st>>>(ec, src, count, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_tensor_acc(const ExtConst *ec, const u64 *A, const u64 *B, u32 nq, u32 d2, u32 n, u64 *T,
                              cudaStream_t st)
{
    if (!nq) return cudaSuccess;
    k_tensor_acc<<<grid_for((size_t)nq * WALLY_MAX_LIMBS * n), 256, 0, st>>>(ec, A, B, nq, d2, n, T);
    return cudaGetLastError();
}

cudaError_t launch_scale_ext(const ExtConst *ec, const u64 *T, u32 nq, u32 n, u64 *X, u64 *ADD, cudaStream_t st)
{
    if (!nq) return cudaSuccess;
    k_scale_ext<<<grid_for((size_t)nq * 3 * n), 256, 0, st>>>(ec, T, nq, n, X, ADD);
    return cudaGetLastError();
}

cudaError_t launch_pir_dim1(const DevParams &dp, const u64 *db, u32 rows, u32 cols, const u64 *ind, u32 ind_stride,
                            u32 n, u64 *out, cudaStream_t st)
{
    if (!n || !cols) return cudaSuccess;
    dim3 grid(dp.n / 32, cols * dp.L, (n + 3) / 4);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    k_pir_dim1<<<grid, 256, 0, st>>>(dp.self, db, rows, cols, ind, ind_stride, n, out);
    return cudaGetLastError();
}

}  // namespace wally
