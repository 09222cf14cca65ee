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
