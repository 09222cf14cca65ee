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

// ---- MulPIR's second dimension: BFV ciphertext products (Sec. 2 CtCtMult)

// Relinearisation keys [n][L][2][L+1][N] (switching from s^2 to s) from
// key_a [n][L][L+1][N] and key_e [n][L][N].
cudaError_t launch_relinkey(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e, u32 n,
                            u64 *keys, cudaStream_t st);

constexpr int XW = 8;  // 64-bit words of the multiword integers (512 bits)

// Constants of the exact tensor: the extension basis r = (q_0..q_{L-1},
// b_0..b_{Lx-1}) whose product R bounds twice the largest tensor
// coefficient, and the CRT and division constants between it and Q.
struct ExtConst {
    int L, Lx, Lr;
    u64 q[WALLY_MAX_LIMBS], b[WALLY_MAX_LIMBS], r[WALLY_MAX_LIMBS];
    u64 theta[WALLY_MAX_LIMBS];          // (Q/q_i)^-1 mod q_i
    u64 qw[WALLY_MAX_LIMBS][XW];         // Q/q_i
    u64 Q[XW], twoQm1[XW];               // Q, 2Q - 1
    u64 qdiv_b[WALLY_MAX_LIMBS][WALLY_MAX_LIMBS];  // (Q/q_i) mod b_k
    u64 Q_b[WALLY_MAX_LIMBS];            // Q mod b_k
    u64 rw[WALLY_MAX_LIMBS][XW];         // R/r_l
    u64 rinv[WALLY_MAX_LIMBS];           // (R/r_l)^-1 mod r_l
    u64 R[XW];
    u64 t;
};

// Centred lifts of count polynomials (coefficient form mod q_0..q_{L-1},
// [count][L][N]) into the extension basis: dst [count][Lr][N].
cudaError_t launch_lift_ext(const ExtConst *ec, const u64 *src, u32 count, u32 n, u64 *dst, cudaStream_t st);

// T[q][k] = sum_j tensor_k(A[q][j], B[q][j]) mod each r_l, NTT form in the
// extension basis: A, B [nq][d2][2][Lr][N]; T [nq][3][Lr][N].
cudaError_t launch_tensor_acc(const ExtConst *ec, const u64 *A, const u64 *B, u32 nq, u32 d2, u32 n, u64 *T,
                              cudaStream_t st);

// From the tensor's residues (coefficient form, [nq][3][Lr][N]): the exact
// integers T_k, then round(t T_k / Q) mod q_i, written as X[q] = (c0, c2) and
// ADD[q] = (0, c1) ([nq][2][L][N] each).
cudaError_t launch_scale_ext(const ExtConst *ec, const u64 *T, u32 nq, u32 n, u64 *X, u64 *ADD, cudaStream_t st);

}  // namespace wally
