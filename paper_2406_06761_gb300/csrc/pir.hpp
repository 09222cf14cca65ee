// pir.hpp -- launchers of the index PIR that serves the keyword PIR of
// Sec. 4.2 (oblivious query expansion and MulPIR's first dimension), and the
// client-side helpers it needs: Galois keys for a list of elements and
// decryption to plaintext coefficients.
#pragma once
#include "kernels.hpp"

namespace wally {

// Inverses mod 2N of the Galois elements of a key set (at most 16 keys).
struct KinvList {
    u64 v[16];
    int nk;
};

// keys [n][nk][L][2][L+1][N] from key_a [n][nk][L][L+1][N], key_e [n][nk][L][N]
cudaError_t launch_keygen_list(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e,
                               u32 n, const KinvList &kl, u64 *keys, cudaStream_t st);

// m = round(t [c0 + c1 s]_Q / Q) mod t per coefficient: coeffs [n][N] in [0, t)
cudaError_t launch_decrypt_coeffs(const DevParams &dp, const int8_t *secret, const u32 *secret_index, const u64 *cts,
                                  u32 n, u64 *xs, int64_t *coeffs, cudaStream_t st);

// dst [P][L][N] = centred lift of src [P][N] (coefficients in [0, t)) into every q_l
cudaError_t launch_pir_lift(const DevParams &dp, const u64 *src, u32 count, u64 *dst, cudaStream_t st);

// key_map[x] = x >> shift for x < count
cudaError_t launch_pir_qmap(u32 *map, u32 count, u32 shift, cudaStream_t st);

// One expansion level (NTT form): for x < count (= n 2^a), with S = sigma(C):
//   next[(x >> a) 2^(a+1) + (x & (2^a - 1))]       = C + S
//   next[(x >> a) 2^(a+1) + (x & (2^a - 1)) + 2^a] = (C - S) * X^(-2^a)
// mono: NTT(X^(-2^a)) per limb, times 2^64 mod q_l, [L][N].
cudaError_t launch_pir_combine(const DevParams &dp, const u64 *cur, const u64 *sig, u64 *next, const u64 *mono,
                               u32 count, u32 a, cudaStream_t st);

// MulPIR's first dimension (NTT form): out[q][j] = sum_{i < rows} db[i][j] * ind[q][i]
// db [rows][cols][L][N] times 2^64 (Montgomery), ind [n][ind_stride][2][L][N]
// canonical, out [n][cols][2][L][N] canonical.
cudaError_t launch_pir_dim1(const DevParams &dp, const u64 *db, u32 rows, u32 cols, const u64 *ind, u32 ind_stride,
                            u32 n, u64 *out, cudaStream_t st);

}  // namespace wally
