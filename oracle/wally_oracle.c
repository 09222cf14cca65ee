/*
 * wally_oracle.c -- plain, slow, CPU reference of Wally's server-side BFV
 * evaluation (arXiv 2406.06761) and of the client operations that feed it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the CPU
 * baseline / reference arm of the benchmark use it.  It shares no code,
 * header, table or constant generator with the CUDA library: primes are found
 * here by trial division (the library uses Miller-Rabin), NTT roots are found
 * by an exhaustive search of its own, and every product is a plain
 * unsigned __int128 product reduced with the C '%' operator.
 *
 * Notation follows the paper: ring R_Q = Z_Q[X]/(X^N+1) with Q = q_0...q_{L-1}
 * (RNS limbs, Sec. 7 "RNS variant of BFV"), plaintext modulus t = 1 mod 2N
 * (Sec. 2 "Vectorized SHE"), special key-switching prime P (hybrid RNS key
 * switching, Sec. 7), embedding dimension d padded to d_pad = g*h, baby step g,
 * giant step h (Sec. 4.1 BSGS; Alg. "Server Initialization"; Alg. "Server
 * Computation").
 *
 * Readings of the paper that fix ciphertext bits where the paper is silent
 * (each one is stated again at the function that takes it):
 *   R1 ct = (c0, c1) with c0 + c1*s = Delta*m + e   (Sec. 2 decryption formula)
 *   R2 one special prime P and one RNS limb per key-switching digit
 *   R3 digits are the non-centred residues [c1]_{q_i} in [0, q_i)
 *   R4 ModDown rounds to nearest through the centred residue mod P
 *   R5 baby steps are a chain of rotations by 1; giant steps use Horner's
 *      rule with rotations by g (only the two keys of Sec. 7 are sent)
 *   R6 Galois generator 3; left row rotation by r is X -> X^(3^r)
 *   R7 slot (row rho, column c) is the evaluation at zeta^(+-3^c) with zeta the
 *      smallest x with x^N = -1 (mod t)
 *   R8 d is padded to the next power of two; g = 2^ceil(log2(d_pad)/2)
 *   R9 plaintext polynomials are lifted centred before reduction mod q_i
 *   R16 the response switch to the last limb is a chain of exact rescalings
 *      by q_0, ..., q_{L-2}, each rounding to nearest; dropped bits round to
 *      nearest too
 *
 * Parity status: every function here is pinned by a test against something
 * other than itself (closed forms, Python big-integer re-derivations,
 * schoolbook products, decryption of the result).  None is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_MAX_MODS 18

typedef struct {
    uint32_t logN, N, L, d, d_pad, g, h, reserved;
    uint64_t mod[OR_MAX_MODS];   /* [0..L-1] = q_i, [L] = P, [L+1] = t */
    uint64_t psi[OR_MAX_MODS];   /* a primitive 2N-th root of unity per modulus */
    uint64_t delta[OR_MAX_MODS]; /* [floor(Q/t)]_{q_i} */
    uint64_t k1, kg;             /* Galois elements of left rotation by 1 and by g */
} or_params;

/* ---------------------------------------------------------------- integers */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a + b) % m); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a + m - (b % m)) % m); }
static uint64_t negmod(uint64_t a, uint64_t m) { return (m - (a % m)) % m; }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

/* Inverse modulo a prime by Fermat's little theorem. */
static uint64_t invmod(uint64_t a, uint64_t p) { return powmod(a, p - 2, p); }

/* Signed small integer to its residue mod m. */
static uint64_t smod(int64_t v, uint64_t m)
{
    i128 r = (i128)v % (i128)m;
    if (r < 0) r += m;
    return (uint64_t)r;
}

/* Primality by trial division: slow and obviously correct. */
int or_is_prime(uint64_t n)
{
    if (n < 2) return 0;
    if (n % 2 == 0) return n == 2;
    for (uint64_t f = 3; f <= n / f; f += 2)
        if (n % f == 0) return 0;
    return 1;
}

/* Largest prime p < below with p = 1 (mod step); 0 if none. */
uint64_t or_prev_prime_1mod(uint64_t below, uint64_t step)
{
    if (below <= step + 1) return 0;
    uint64_t c = ((below - 2) / step) * step + 1; /* largest 1 mod step that is < below */
    for (; c > step; c -= step)
        if (or_is_prime(c)) return c;
    return 0;
}

/* A primitive 2N-th root of unity mod p (p = 1 mod 2N): the first h = 2, 3, ...
 * whose power h^((p-1)/2N) satisfies x^N = -1.  Any such root gives the same
 * ring products; only the plaintext slot root (R7) changes ciphertext bits. */
static uint64_t find_psi(uint64_t p, uint32_t N)
{
    for (uint64_t h = 2; h < p; h++) {
        uint64_t x = powmod(h, (p - 1) / (2 * (uint64_t)N), p);
        if (powmod(x, N, p) == p - 1) return x;
    }
    return 0;
}

/* R7: the slot root zeta_t, the smallest x with x^N = -1 (mod t). */
uint64_t or_smallest_root(uint64_t t, uint32_t N)
{
    for (uint64_t x = 2; x < t; x++)
        if (powmod(x, N, t) == t - 1) return x;
    return 0;
}

/* --------------------------------------------------------------- parameters
 * Sec. 2 "Vectorized SHE" (t prime, t = 1 mod 2n), Sec. 7 "Parameters
 * Selection" (RNS limbs of a given bit size).  q_i: the L largest primes
 * = 1 mod 2N below 2^q_bits; P (R2): the next prime of that form below the
 * last q_i; t: the largest prime = 1 mod 2N below 2^t_bits.
 * Delta = floor(Q/t) (Sec. 2 ciphertext formula), stored as [Delta]_{q_i}:
 * with Q = t*Delta + rho, rho = Q mod t, and Q = 0 mod q_i it follows that
 * [Delta]_{q_i} = -rho * t^-1 mod q_i.
 * R8: d_pad = next power of two >= d, g = 2^ceil(log2(d_pad)/2), h = d_pad/g.
 */
int or_params_init(uint32_t logN, uint32_t L, uint32_t q_bits, uint32_t t_bits, uint32_t dim,
                   const uint64_t *q_override, uint64_t p_override, uint64_t t_override,
                   or_params *o)
{
    if (logN < 2 || logN > 17 || L < 1 || L + 2 > OR_MAX_MODS || q_bits > 61 || t_bits > 40) return -1;
    memset(o, 0, sizeof(*o));
    o->logN = logN;
    o->N = 1u << logN;
    o->L = L;
    uint64_t step = 2 * (uint64_t)o->N;
    uint64_t below = (uint64_t)1 << q_bits;
    for (uint32_t i = 0; i < L; i++) {
        uint64_t q = q_override ? q_override[i] : or_prev_prime_1mod(below, step);
        if (!q) return -2;
        o->mod[i] = q;
        below = q;
    }
    o->mod[L] = p_override ? p_override : or_prev_prime_1mod(below, step);
    o->mod[L + 1] = t_override ? t_override : or_prev_prime_1mod((uint64_t)1 << t_bits, step);
    if (!o->mod[L] || !o->mod[L + 1]) return -2;
    for (uint32_t j = 0; j < L + 1; j++) o->psi[j] = find_psi(o->mod[j], o->N);
    o->psi[L + 1] = or_smallest_root(o->mod[L + 1], o->N);
    for (uint32_t j = 0; j < L + 2; j++)
        if (!o->psi[j]) return -3;
    uint64_t t = o->mod[L + 1];
    uint64_t rho = 1 % t;
    for (uint32_t i = 0; i < L; i++) rho = mulmod(rho, o->mod[i] % t, t);
    for (uint32_t i = 0; i < L; i++) {
        uint64_t q = o->mod[i];
        o->delta[i] = mulmod(negmod(rho, q), invmod(t % q, q), q);
    }
    o->d = dim;
    uint32_t dp = 1, lg = 0;
    while (dp < dim) { dp <<= 1; lg++; }
    o->d_pad = dp;
    o->g = 1u << ((lg + 1) / 2);
    o->h = dp / o->g;
    if (dp > o->N / 2) return -4;
    o->k1 = 3;
    o->kg = powmod(3, o->g, step);
    return 0;
}

/* Another split of the diagonals into g baby steps and h = d_pad / g giant
 * steps.  Sec. 5: the plaintexts are pre-rotated for BSGS only while a
 * cluster has fewer than sqrt(d) chunks; for larger clusters the query is
 * rotated through every diagonal with no giant steps, which is the split
 * g = d_pad, h = 1 (the pre-rotation by g*i is then the identity).  g must be
 * a power of two dividing d_pad, at least 2. */
int or_params_set_split(or_params *o, uint32_t g)
{
    if (g < 2 || g > o->d_pad || (g & (g - 1)) || o->d_pad % g) return -1;
    o->g = g;
    o->h = o->d_pad / g;
    o->kg = powmod(3, g, 2 * (uint64_t)o->N);
    return 0;
}

/* ---------------------------------------------------------------- NTT
 * Negacyclic number-theoretic transform (Sec. 7 "Reducing the computation of
 * BFV operations"): A[i] = sum_k a[k] psi^((2i+1)k), natural order, i.e. the
 * evaluation of a(X) at the odd powers psi^(2i+1), the N roots of X^N + 1.
 * Computed textbook-style: twist by psi^k, then a cyclic radix-2 DFT with
 * omega = psi^2 (bit-reversal permutation followed by butterflies).
 */
static void dft_cyclic(uint64_t *a, uint32_t N, uint64_t p, uint64_t w)
{
    for (uint32_t i = 1, j = 0; i < N; i++) {
        uint32_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t tmp = a[i]; a[i] = a[j]; a[j] = tmp; }
    }
    uint64_t *pw = (uint64_t *)malloc(sizeof(uint64_t) * (N / 2 + 1));
    pw[0] = 1 % p;
    for (uint32_t i = 1; i <= N / 2; i++) pw[i] = mulmod(pw[i - 1], w, p);
    for (uint32_t len = 2; len <= N; len <<= 1) {
        uint32_t half = len / 2, stride = N / len;
        for (uint32_t i = 0; i < N; i += len)
            for (uint32_t j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + half], pw[j * stride], p);
                a[i + j] = addmod(u, v, p);
                a[i + j + half] = submod(u, v, p);
            }
    }
    free(pw);
}

static void ntt_fwd_raw(uint64_t *a, uint32_t N, uint64_t p, uint64_t psi)
{
    uint64_t pk = 1 % p;
    for (uint32_t k = 0; k < N; k++) { a[k] = mulmod(a[k], pk, p); pk = mulmod(pk, psi, p); }
    dft_cyclic(a, N, p, mulmod(psi, psi, p));
}

static void ntt_inv_raw(uint64_t *a, uint32_t N, uint64_t p, uint64_t psi)
{
    uint64_t psi_inv = invmod(psi, p);
    dft_cyclic(a, N, p, mulmod(psi_inv, psi_inv, p));
    uint64_t n_inv = invmod(N % p, p), pk = n_inv;
    for (uint32_t k = 0; k < N; k++) { a[k] = mulmod(a[k], pk, p); pk = mulmod(pk, psi_inv, p); }
}

void or_ntt_fwd(const or_params *o, uint32_t j, uint64_t *a) { ntt_fwd_raw(a, o->N, o->mod[j], o->psi[j]); }
void or_ntt_inv(const or_params *o, uint32_t j, uint64_t *a) { ntt_inv_raw(a, o->N, o->mod[j], o->psi[j]); }

/* Negacyclic product a*b mod (X^N + 1, p_j) by the definition (O(N^2)). */
void or_polymul_schoolbook(const or_params *o, uint32_t j, const uint64_t *a, const uint64_t *b, uint64_t *out)
{
    uint32_t N = o->N;
    uint64_t p = o->mod[j];
    for (uint32_t k = 0; k < N; k++) out[k] = 0;
    for (uint32_t x = 0; x < N; x++)
        for (uint32_t y = 0; y < N; y++) {
            uint64_t v = mulmod(a[x], b[y], p);
            if (x + y < N) out[x + y] = addmod(out[x + y], v, p);
            else out[x + y - N] = submod(out[x + y - N], v, p);
        }
}

/* Negacyclic product through the NTT: INTT(NTT(a) . NTT(b)). */
void or_polymul(const or_params *o, uint32_t j, const uint64_t *a, const uint64_t *b, uint64_t *out)
{
    uint32_t N = o->N;
    uint64_t p = o->mod[j];
    uint64_t *A = (uint64_t *)malloc(8 * (size_t)N), *B = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t k = 0; k < N; k++) { A[k] = a[k] % p; B[k] = b[k] % p; }
    ntt_fwd_raw(A, N, p, o->psi[j]);
    ntt_fwd_raw(B, N, p, o->psi[j]);
    for (uint32_t k = 0; k < N; k++) out[k] = mulmod(A[k], B[k], p);
    ntt_inv_raw(out, N, p, o->psi[j]);
    free(A);
    free(B);
}

/* Galois automorphism sigma_k : a(X) -> a(X^k) on a coefficient vector mod
 * p_j (Sec. 4.2 "Reducing evaluation key size"; Sec. 2 CtRotate).  The term
 * a_n X^n goes to X^(nk mod 2N), folded with X^N = -1. */
void or_automorphism(const or_params *o, uint32_t j, uint64_t k, const uint64_t *a, uint64_t *out)
{
    uint32_t N = o->N;
    uint64_t p = o->mod[j], twoN = 2 * (uint64_t)N;
    for (uint32_t n = 0; n < N; n++) {
        uint64_t e = ((uint64_t)n * k) % twoN;
        if (e < N) out[e] = a[n] % p;
        else out[e - N] = negmod(a[n], p);
    }
}

/* ---------------------------------------------------------------- slots
 * Sec. 2 "Vectorized SHE" and the CtRotate definition: N slots in two rows of
 * N/2.  R7: slot s = rho*N/2 + c holds m(zeta^e) with e = 3^c (rho = 0) or
 * e = -3^c (rho = 1) mod 2N.  With the NTT above, m(zeta^e) is entry (e-1)/2.
 */
static uint32_t slot_ntt_index(const or_params *o, uint32_t s)
{
    uint64_t twoN = 2 * (uint64_t)o->N;
    uint32_t half = o->N / 2, rho = s / half, c = s % half;
    uint64_t e = powmod(3, c, twoN);
    if (rho) e = twoN - e;
    return (uint32_t)((e - 1) / 2);
}

/* Encode: the unique m in Z_t[X]/(X^N+1) with the given slot values. */
void or_slots_encode(const or_params *o, const uint64_t *v, uint64_t *m)
{
    uint32_t N = o->N, jt = o->L + 1;
    for (uint32_t s = 0; s < N; s++) m[slot_ntt_index(o, s)] = v[s] % o->mod[jt];
    or_ntt_inv(o, jt, m);
}

void or_slots_decode(const or_params *o, const uint64_t *m, uint64_t *v)
{
    uint32_t N = o->N, jt = o->L + 1;
    uint64_t *A = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t k = 0; k < N; k++) A[k] = m[k] % o->mod[jt];
    or_ntt_fwd(o, jt, A);
    for (uint32_t s = 0; s < N; s++) v[s] = A[slot_ntt_index(o, s)];
    free(A);
}

/* Alg. "Client Query Generation": the query repeated n/d times.  Slot
 * s = beta*d_pad + x holds q[x] mod t for x < d and 0 for the padding.  A NULL
 * query is the all-zero vector of a fake query. */
void or_replicate_query(const or_params *o, const int32_t *q, uint64_t *v)
{
    uint64_t t = o->mod[o->L + 1];
    for (uint32_t s = 0; s < o->N; s++) {
        uint32_t x = s % o->d_pad;
        v[s] = (q && x < o->d) ? smod(q[x], t) : 0;
    }
}

/* ---------------------------------------------------------------- cluster encoding
 * Alg. "Server Initialization" with the packing of Sec. 4.1 ("Database and
 * query packing").  A cluster of `size` embeddings (rows of `emb`, d entries
 * each) fills m = ceil(size/N) chunks.  Chunk k, slot s = beta*d_pad + x,
 * belongs to embedding u = k*N + s (slice beta of the chunk, column x).
 * Diagonal j (Sec. 4.1 p_j): p_{k,j}[s] = E[u][(x + j) mod d_pad], zero past
 * the end of the cluster and in the padding of d.  BSGS pre-rotation (the
 * PtRotate by -g*a of the algorithm): P'_{k,i,b} = rowrot(p_{k,g*i+b}, -g*i),
 * i.e. slot (rho, c) takes p at (rho, c - g*i mod N/2).  Each P' is encoded
 * (slots -> polynomial mod t), lifted centred (R9) and reduced mod every q_l.
 * Output layout: [m][h][g][L][N], coefficient form.  Returns m.
 */
int or_encode_cluster(const or_params *o, uint32_t size, const int8_t *emb, uint64_t *out)
{
    uint32_t N = o->N, L = o->L, d = o->d, dp = o->d_pad, g = o->g, h = o->h, half = N / 2;
    uint64_t t = o->mod[L + 1];
    uint32_t m = (size + N - 1) / N;
    if (m == 0) m = 1;
    uint64_t *pj = (uint64_t *)malloc(8 * (size_t)N), *pr = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t *poly = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t k = 0; k < m; k++)
        for (uint32_t i = 0; i < h; i++)
            for (uint32_t b = 0; b < g; b++) {
                uint32_t j = g * i + b;
                for (uint32_t s = 0; s < N; s++) {
                    uint32_t x = s % dp, col = (x + j) % dp;
                    uint64_t u = (uint64_t)k * N + s;
                    pj[s] = (u < size && col < d) ? smod(emb[u * d + col], t) : 0;
                }
                uint32_t shift = (g * i) % half;
                for (uint32_t s = 0; s < N; s++) {
                    uint32_t rho = s / half, c = s % half;
                    pr[s] = pj[rho * half + (c + half - shift) % half];
                }
                or_slots_encode(o, pr, poly);
                for (uint32_t l = 0; l < L; l++) {
                    uint64_t q = o->mod[l];
                    uint64_t *dst = out + ((((size_t)k * h + i) * g + b) * L + l) * N;
                    for (uint32_t n = 0; n < N; n++) {
                        int64_t c = poly[n] > (t - 1) / 2 ? (int64_t)poly[n] - (int64_t)t : (int64_t)poly[n];
                        dst[n] = smod(c, q);
                    }
                }
            }
    free(pj);
    free(pr);
    free(poly);
    return (int)m;
}

/* ---------------------------------------------------------------- client side
 * Sec. 2 (RLWE SHE, decryption formula) and Sec. 5 "Query generation": fresh
 * keys per query, evaluation keys for rotation steps 1 and g.  All random
 * numbers are inputs: s ternary, a uniform residues, e small errors.
 */

/* Galois key for element k (R2, R3): s' = sigma_k(s).  For digit i < L, with
 * a_i uniform mod each of the L+1 moduli and e_i small:
 *   on q_j : b_i = -a_i*s + e_i + [i == j] * P * s'   (mod q_j)
 *   on P   : b_i = -a_i*s + e_i                       (mod P)
 * key layout [L digit][2: b, a][L+1 modulus][N], coefficient form. */
void or_keygen(const or_params *o, const int8_t *s, uint64_t k, const uint64_t *a_rand,
               const int8_t *e_rand, uint64_t *key)
{
    uint32_t N = o->N, L = o->L;
    uint64_t *sj = (uint64_t *)malloc(8 * (size_t)N), *spj = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t *as = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t j = 0; j <= L; j++) {
        uint64_t p = o->mod[j];
        for (uint32_t n = 0; n < N; n++) sj[n] = smod(s[n], p);
        or_automorphism(o, j, k, sj, spj);
        uint64_t Pmod = o->mod[L] % p;
        for (uint32_t i = 0; i < L; i++) {
            const uint64_t *a = a_rand + ((size_t)i * (L + 1) + j) * N;
            const int8_t *e = e_rand + (size_t)i * N;
            uint64_t *b_out = key + (((size_t)i * 2 + 0) * (L + 1) + j) * N;
            uint64_t *a_out = key + (((size_t)i * 2 + 1) * (L + 1) + j) * N;
            or_polymul(o, j, a, sj, as);
            for (uint32_t n = 0; n < N; n++) {
                uint64_t v = submod(smod(e[n], p), as[n], p);
                if (j == i) v = addmod(v, mulmod(Pmod, spj[n], p), p);
                b_out[n] = v;
                a_out[n] = a[n] % p;
            }
        }
    }
    free(sj);
    free(spj);
    free(as);
}

/* Relinearisation key (the key switching key from s^2 to s): as or_keygen
 * with s' = s^2, the negacyclic square of the secret, in place of
 * sigma_k(s):  b_i = -a_i*s + e_i + [i == j] P s^2 (mod q_j),  b_i = -a_i*s + e_i (mod P). */
void or_relinkey(const or_params *o, const int8_t *s, const uint64_t *a_rand, const int8_t *e_rand, uint64_t *key)
{
    uint32_t N = o->N, L = o->L;
    uint64_t *sj = (uint64_t *)malloc(8 * (size_t)N), *s2 = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t *as = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t j = 0; j <= L; j++) {
        uint64_t p = o->mod[j];
        for (uint32_t n = 0; n < N; n++) sj[n] = smod(s[n], p);
        or_polymul(o, j, sj, sj, s2);
        uint64_t Pmod = o->mod[L] % p;
        for (uint32_t i = 0; i < L; i++) {
            const uint64_t *a = a_rand + ((size_t)i * (L + 1) + j) * N;
            const int8_t *e = e_rand + (size_t)i * N;
            uint64_t *b_out = key + (((size_t)i * 2 + 0) * (L + 1) + j) * N;
            uint64_t *a_out = key + (((size_t)i * 2 + 1) * (L + 1) + j) * N;
            or_polymul(o, j, a, sj, as);
            for (uint32_t n = 0; n < N; n++) {
                uint64_t v = submod(smod(e[n], p), as[n], p);
                if (j == i) v = addmod(v, mulmod(Pmod, s2[n], p), p);
                b_out[n] = v;
                a_out[n] = a[n] % p;
            }
        }
    }
    free(sj);
    free(s2);
    free(as);
}

/* Encryption (R1): c1 = a, c0 = -a*s + e + Delta*m (mod q_i), m in [0, t). */
void or_encrypt(const or_params *o, const int8_t *s, const uint64_t *m_poly, const uint64_t *a_rand,
                const int8_t *e, uint64_t *ct)
{
    uint32_t N = o->N, L = o->L;
    uint64_t *sj = (uint64_t *)malloc(8 * (size_t)N), *as = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t i = 0; i < L; i++) {
        uint64_t q = o->mod[i];
        const uint64_t *a = a_rand + (size_t)i * N;
        for (uint32_t n = 0; n < N; n++) sj[n] = smod(s[n], q);
        or_polymul(o, i, a, sj, as);
        uint64_t *c0 = ct + (size_t)i * N, *c1 = ct + ((size_t)L + i) * N;
        for (uint32_t n = 0; n < N; n++) {
            uint64_t v = submod(smod(e[n], q), as[n], q);
            c0[n] = addmod(v, mulmod(o->delta[i], m_poly[n], q), q);
            c1[n] = a[n] % q;
        }
    }
    free(sj);
    free(as);
}

/* Decryption, first half (Sec. 2): x_i = [c0 + c1*s]_{q_i} for every limb.
 * The CRT composition and the scaling by t/Q are done with big integers by
 * the Python wrapper. */
void or_decrypt_residues(const or_params *o, const int8_t *s, const uint64_t *ct, uint64_t *x)
{
    uint32_t N = o->N, L = o->L;
    uint64_t *sj = (uint64_t *)malloc(8 * (size_t)N), *cs = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t i = 0; i < L; i++) {
        uint64_t q = o->mod[i];
        for (uint32_t n = 0; n < N; n++) sj[n] = smod(s[n], q);
        or_polymul(o, i, ct + ((size_t)L + i) * N, sj, cs);
        for (uint32_t n = 0; n < N; n++) x[(size_t)i * N + n] = addmod(ct[(size_t)i * N + n], cs[n], q);
    }
    free(sj);
    free(cs);
}

/* ---------------------------------------------------------------- server side */

/* Key in NTT form: every polynomial of a key transformed once per query. */
static uint64_t *key_to_ntt(const or_params *o, const uint64_t *key)
{
    uint32_t N = o->N, L = o->L;
    size_t n = (size_t)L * 2 * (L + 1) * N;
    uint64_t *kn = (uint64_t *)malloc(8 * n);
    memcpy(kn, key, 8 * n);
    for (uint32_t i = 0; i < L; i++)
        for (uint32_t c = 0; c < 2; c++)
            for (uint32_t j = 0; j <= L; j++) or_ntt_fwd(o, j, kn + (((size_t)i * 2 + c) * (L + 1) + j) * N);
    return kn;
}

/* Rotation Rot_k = automorphism + hybrid key switching (Sec. 2 CtRotate,
 * Sec. 7 hybrid RNS key switching), key in NTT form:
 *   1. (c0, c1) -> (sigma_k(c0), sigma_k(c1)).
 *   2. R3: digit d_i = [sigma(c1)]_{q_i} in [0, q_i), read as an integer and
 *      reduced mod every modulus of q_0..q_{L-1}, P.
 *   3. (u0, u1) = sum_i d_i * (b_i, a_i) over all L+1 moduli.
 *   4. R4 ModDown: r = [u]_P, r_c = r - P if r > (P-1)/2 else r;
 *      u'_j = (u_j - r_c) * P^-1 mod q_j.
 *   5. result (sigma(c0) + u0', u1').
 */
static void rotate_nttkey(const or_params *o, uint64_t k, const uint64_t *keyn, const uint64_t *ct, uint64_t *out)
{
    uint32_t N = o->N, L = o->L;
    uint64_t P = o->mod[L];
    uint64_t *sc = (uint64_t *)malloc(8 * (size_t)2 * L * N);
    for (uint32_t c = 0; c < 2; c++)
        for (uint32_t i = 0; i < L; i++)
            or_automorphism(o, i, k, ct + ((size_t)c * L + i) * N, sc + ((size_t)c * L + i) * N);
    const uint64_t *sc0 = sc, *sc1 = sc + (size_t)L * N;
    uint64_t *u = (uint64_t *)malloc(8 * (size_t)2 * (L + 1) * N); /* [2][L+1][N] */
    uint64_t *D = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t j = 0; j <= L; j++) {
        uint64_t p = o->mod[j];
        uint64_t *u0 = u + (size_t)j * N, *u1 = u + ((size_t)(L + 1) + j) * N;
        memset(u0, 0, 8 * (size_t)N);
        memset(u1, 0, 8 * (size_t)N);
        for (uint32_t i = 0; i < L; i++) {
            for (uint32_t n = 0; n < N; n++) D[n] = sc1[(size_t)i * N + n] % p;
            or_ntt_fwd(o, j, D);
            const uint64_t *kb = keyn + (((size_t)i * 2 + 0) * (L + 1) + j) * N;
            const uint64_t *ka = keyn + (((size_t)i * 2 + 1) * (L + 1) + j) * N;
            for (uint32_t n = 0; n < N; n++) {
                u0[n] = addmod(u0[n], mulmod(D[n], kb[n], p), p);
                u1[n] = addmod(u1[n], mulmod(D[n], ka[n], p), p);
            }
        }
        or_ntt_inv(o, j, u0);
        or_ntt_inv(o, j, u1);
    }
    for (uint32_t j = 0; j < L; j++) {
        uint64_t q = o->mod[j], pinv = invmod(P % q, q);
        for (uint32_t c = 0; c < 2; c++) {
            const uint64_t *uj = u + ((size_t)c * (L + 1) + j) * N;
            const uint64_t *uP = u + ((size_t)c * (L + 1) + L) * N;
            uint64_t *dst = out + ((size_t)c * L + j) * N;
            for (uint32_t n = 0; n < N; n++) {
                int64_t rc = uP[n] > (P - 1) / 2 ? (int64_t)uP[n] - (int64_t)P : (int64_t)uP[n];
                uint64_t v = mulmod(submod(uj[n], smod(rc, q), q), pinv, q);
                dst[n] = c == 0 ? addmod(sc0[(size_t)j * N + n], v, q) : v;
            }
        }
    }
    free(sc);
    free(u);
    free(D);
}

/* One rotation with a key in coefficient form ([L][2][L+1][N]). */
void or_rotate(const or_params *o, uint64_t k, const uint64_t *key, const uint64_t *ct, uint64_t *out)
{
    uint64_t *kn = key_to_ntt(o, key);
    rotate_nttkey(o, k, kn, ct, out);
    free(kn);
}

/* Plaintext-ciphertext products T = sum_b P_b * ct_b, both ciphertext
 * components, as ring products mod each q_l (Sec. 2 PtCtMult, CtCtAdd). */
void or_ptct_sum(const or_params *o, uint32_t count, const uint64_t *ptxt /*[count][L][N]*/,
                 const uint64_t *cts /*[count][2][L][N]*/, uint64_t *out /*[2][L][N]*/)
{
    uint32_t N = o->N, L = o->L;
    uint64_t *A = (uint64_t *)malloc(8 * (size_t)N), *B = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t *acc = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t c = 0; c < 2; c++)
        for (uint32_t l = 0; l < L; l++) {
            uint64_t q = o->mod[l];
            memset(acc, 0, 8 * (size_t)N);
            for (uint32_t b = 0; b < count; b++) {
                memcpy(A, ptxt + ((size_t)b * L + l) * N, 8 * (size_t)N);
                memcpy(B, cts + (((size_t)b * 2 + c) * L + l) * N, 8 * (size_t)N);
                or_ntt_fwd(o, l, A);
                or_ntt_fwd(o, l, B);
                for (uint32_t n = 0; n < N; n++) acc[n] = addmod(acc[n], mulmod(A[n], B[n], q), q);
            }
            or_ntt_inv(o, l, acc);
            memcpy(out + ((size_t)c * L + l) * N, acc, 8 * (size_t)N);
        }
    free(A);
    free(B);
    free(acc);
}

/* Server computation (Alg. "Server Computation", Sec. 5 "Server
 * computation") for one query, with plaintexts already in NTT form
 * ([m][h][g][L][N]) and keys in coefficient form ([2][L][2][L+1][N], key for
 * rotation by 1 first, then by g).  R5:
 *   ct'[0] = ct; ct'[j] = Rot_1(ct'[j-1]) for j < g            (baby steps)
 *   per chunk k: T_i = sum_b P'_{k,i,b} * ct'[b]               (i < h)
 *                S = T_{h-1}; S = Rot_g(S) + T_i for i = h-2 .. 0
 * Output [m][2][L][N], coefficient form, residues in [0, q_l). */
static void eval_one(const or_params *o, uint32_t m, const uint64_t *ptxt_ntt, const uint64_t *ct,
                     const uint64_t *keys, uint64_t *out)
{
    uint32_t N = o->N, L = o->L, g = o->g, h = o->h;
    size_t ctsz = (size_t)2 * L * N, keysz = (size_t)L * 2 * (L + 1) * N;
    uint64_t *k1n = key_to_ntt(o, keys), *kgn = key_to_ntt(o, keys + keysz);
    uint64_t *ctp = (uint64_t *)malloc(8 * ctsz * g);
    memcpy(ctp, ct, 8 * ctsz);
    for (uint32_t j = 1; j < g; j++) rotate_nttkey(o, o->k1, k1n, ctp + (j - 1) * ctsz, ctp + j * ctsz);
    /* NTT form of the rotated queries, for the products */
    uint64_t *ctpn = (uint64_t *)malloc(8 * ctsz * g);
    memcpy(ctpn, ctp, 8 * ctsz * g);
    for (uint32_t j = 0; j < g; j++)
        for (uint32_t c = 0; c < 2; c++)
            for (uint32_t l = 0; l < L; l++) or_ntt_fwd(o, l, ctpn + j * ctsz + ((size_t)c * L + l) * N);
    uint64_t *T = (uint64_t *)malloc(8 * ctsz * h), *S = (uint64_t *)malloc(8 * ctsz);
    uint64_t *R = (uint64_t *)malloc(8 * ctsz);
    for (uint32_t k = 0; k < m; k++) {
        for (uint32_t i = 0; i < h; i++)
            for (uint32_t c = 0; c < 2; c++)
                for (uint32_t l = 0; l < L; l++) {
                    uint64_t q = o->mod[l];
                    uint64_t *acc = T + i * ctsz + ((size_t)c * L + l) * N;
                    memset(acc, 0, 8 * (size_t)N);
                    for (uint32_t b = 0; b < g; b++) {
                        const uint64_t *pt = ptxt_ntt + ((((size_t)k * h + i) * g + b) * L + l) * N;
                        const uint64_t *cb = ctpn + b * ctsz + ((size_t)c * L + l) * N;
                        for (uint32_t n = 0; n < N; n++) acc[n] = addmod(acc[n], mulmod(pt[n], cb[n], q), q);
                    }
                    or_ntt_inv(o, l, acc);
                }
        memcpy(S, T + (size_t)(h - 1) * ctsz, 8 * ctsz);
        for (int i = (int)h - 2; i >= 0; i--) {
            rotate_nttkey(o, o->kg, kgn, S, R);
            for (uint32_t c = 0; c < 2; c++)
                for (uint32_t l = 0; l < L; l++) {
                    uint64_t q = o->mod[l];
                    size_t off = ((size_t)c * L + l) * N;
                    for (uint32_t n = 0; n < N; n++) S[off + n] = addmod(R[off + n], T[(size_t)i * ctsz + off + n], q);
                }
        }
        memcpy(out + (size_t)k * ctsz, S, 8 * ctsz);
    }
    free(k1n);
    free(kgn);
    free(ctp);
    free(ctpn);
    free(T);
    free(S);
    free(R);
}

/* Plaintexts of one cluster ([m][h][g][L][N], coefficient form) to NTT form. */
void or_ptxt_to_ntt(const or_params *o, uint32_t m, const uint64_t *ptxt, uint64_t *out)
{
    uint32_t N = o->N, L = o->L;
    size_t cnt = (size_t)m * o->h * o->g;
    memcpy(out, ptxt, 8 * cnt * L * N);
    for (size_t x = 0; x < cnt; x++)
        for (uint32_t l = 0; l < L; l++) or_ntt_fwd(o, l, out + (x * L + l) * N);
}

int or_eval(const or_params *o, uint32_t m, const uint64_t *ptxt, const uint64_t *ct, const uint64_t *keys,
            uint64_t *out)
{
    if (m == 0 || m >= o->g) return -1; /* BSGS only while chunks < sqrt(d) (Sec. 5) */
    size_t n = (size_t)m * o->h * o->g * o->L * o->N;
    uint64_t *pn = (uint64_t *)malloc(8 * n);
    or_ptxt_to_ntt(o, m, ptxt, pn);
    eval_one(o, m, pn, ct, keys, out);
    free(pn);
    return 0;
}

/* Many queries over several clusters, one POSIX thread per worker, queries
 * handed out through an atomic counter.  ptxt_ntt[c] is cluster c's plaintext
 * set in NTT form (or_ptxt_to_ntt), chunks[c] its chunk count; query q uses
 * cluster ids[q], ciphertext cts[q], keys keys[q], and writes chunk offset
 * out_offsets[q] of `out`. */
typedef struct {
    const or_params *o;
    const uint32_t *chunks;
    const uint64_t *const *ptxt_ntt;
    uint32_t nq;
    const uint32_t *ids;
    const uint64_t *cts, *keys, *out_offsets;
    uint64_t *out;
    uint32_t next;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *b = (batch_job *)arg;
    const or_params *o = b->o;
    size_t ctsz = (size_t)2 * o->L * o->N, keysz = (size_t)2 * o->L * 2 * (o->L + 1) * o->N;
    for (;;) {
        uint32_t q = __atomic_fetch_add(&b->next, 1, __ATOMIC_RELAXED);
        if (q >= b->nq) break;
        uint32_t c = b->ids[q];
        eval_one(o, b->chunks[c], b->ptxt_ntt[c], b->cts + q * ctsz, b->keys + q * keysz,
                 b->out + b->out_offsets[q] * ctsz);
    }
    return NULL;
}

int or_eval_batch(const or_params *o, uint32_t n_clusters, const uint32_t *chunks, const uint64_t *const *ptxt_ntt,
                  uint32_t nq, const uint32_t *ids, const uint64_t *cts, const uint64_t *keys,
                  const uint64_t *out_offsets, uint64_t *out, uint32_t nthreads)
{
    for (uint32_t q = 0; q < nq; q++)
        if (ids[q] >= n_clusters || chunks[ids[q]] == 0 || chunks[ids[q]] >= o->g) return -1;
    batch_job job = {o, chunks, ptxt_ntt, nq, ids, cts, keys, out_offsets, out, 0};
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (uint32_t i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, batch_worker, &job);
    for (uint32_t i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

/* ---------------------------------------------------------------- response compression
 * Sec. 7 "Reducing the response size": switch the response to its last RNS
 * limb q' = q_{L-1} and drop low bits of both polynomials.
 * Reading R16: the switch is a chain of exact rescalings by q_0, ..., q_{L-2};
 * each step replaces c by round(c / q_i), computed as
 * (c - [c]_{q_i, centred}) * q_i^-1 on the remaining limbs.  Then l0 low bits
 * of c0 and l1 of c1 are dropped with rounding to nearest:
 * c'' = floor((c' + 2^(l-1)) / 2^l).  Output [2][N] integers. */
void or_compress(const or_params *o, const uint64_t *ct, uint32_t l0, uint32_t l1, uint64_t *out)
{
    uint32_t N = o->N, L = o->L;
    int64_t v[OR_MAX_MODS];
    for (uint32_t c = 0; c < 2; c++)
        for (uint32_t n = 0; n < N; n++) {
            for (uint32_t j = 0; j < L; j++) v[j] = (int64_t)ct[((size_t)c * L + j) * N + n];
            for (uint32_t i = 0; i + 1 < L; i++) {
                uint64_t qi = o->mod[i];
                int64_t rc = (uint64_t)v[i] > (qi - 1) / 2 ? v[i] - (int64_t)qi : v[i];
                for (uint32_t j = i + 1; j < L; j++) {
                    uint64_t qj = o->mod[j];
                    uint64_t d = submod((uint64_t)v[j], smod(rc, qj), qj);
                    v[j] = (int64_t)mulmod(d, invmod(qi % qj, qj), qj);
                }
            }
            uint64_t x = (uint64_t)v[L - 1];
            uint32_t l = c ? l1 : l0;
            out[(size_t)c * N + n] = l ? (x + ((uint64_t)1 << (l - 1))) >> l : x;
        }
}

/* Decryption of a compressed response, first half: x = c0'' 2^l0 +
 * c1'' 2^l1 s (mod q'); the scaling round(t x / q') is left to the caller. */
void or_decompress_residue(const or_params *o, const int8_t *s, const uint64_t *cc, uint32_t l0, uint32_t l1,
                           uint64_t *x)
{
    uint32_t N = o->N, L = o->L;
    uint64_t q = o->mod[L - 1];
    uint64_t *c1 = (uint64_t *)malloc(8 * (size_t)N), *sj = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t *p = (uint64_t *)malloc(8 * (size_t)N);
    for (uint32_t n = 0; n < N; n++) {
        c1[n] = mulmod(cc[N + n] % q, powmod(2, l1, q), q);
        sj[n] = smod(s[n], q);
    }
    or_polymul(o, L - 1, c1, sj, p);
    for (uint32_t n = 0; n < N; n++) x[n] = addmod(mulmod(cc[n] % q, powmod(2, l0, q), q), p[n], q);
    free(c1);
    free(sj);
    free(p);
}
