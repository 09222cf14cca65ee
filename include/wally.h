/*
 * wally.h -- C ABI of the GB300 library for Wally's server-side encrypted
 * similarity computation (arXiv 2406.06761, "Wally: Batched Private Nearest
 * Neighbor Search at Scale").
 *
 * The server holds a database of embeddings split into clusters.  Each query
 * is a BFV ciphertext of the client's embedding (replicated across the slots)
 * plus two fresh Galois keys, and names one cluster.  The server returns, per
 * chunk of that cluster, one ciphertext whose slots are the dot products of
 * the query with every embedding of the chunk (Sec. 4.1, Sec. 5 "Server
 * computation", Alg. "Server Computation").
 *
 * Conventions shared by every call:
 *  - N ring degree, L ciphertext limbs q_0..q_{L-1}, P the special prime of
 *    hybrid key switching (Sec. 7), t the plaintext modulus, d the embedding
 *    dimension, d_pad = g*h its padding, g baby steps, h giant steps.
 *  - Polynomials are N consecutive uint64_t residues in [0, modulus), in
 *    COEFFICIENT form (coefficient of X^n at index n) at the boundary.
 *  - ciphertext  : uint64_t [2][L][N]             (c0, c1 with c0 + c1*s = Delta*m + e)
 *  - galois keys : uint64_t [2][L][2][L+1][N]     (key for left rotation by 1, then by g;
 *                  per key: digit i < L, component (b, a), modulus q_0..q_{L-1}, P)
 *  - "device" pointers are CUDA device memory of the context's device;
 *    "host" pointers are ordinary host memory.  Pointers must be 16-byte
 *    aligned.  The caller owns every buffer it passes; no call keeps a caller
 *    pointer after it returns (asynchronous calls: after the stream reaches
 *    the work, i.e. after wally_sync).
 *  - Every call returns WALLY_OK or an error code; wally_last_error() gives a
 *    thread-local message.  Nothing throws across the ABI.  Device-side
 *    problems of asynchronous calls (a cluster id out of range) are recorded
 *    in the context and reported by wally_sync.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef WALLY_H
#define WALLY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    WALLY_OK = 0,
    WALLY_EINVAL = 1,   /* bad argument: shape, range, null pointer, unsupported size */
    WALLY_ENOMEM = 2,   /* device or host allocation failed */
    WALLY_ECUDA = 3,    /* a CUDA runtime call failed */
    WALLY_ETIMEOUT = 4, /* a bounded device-side wait gave up (reserved: no call waits on the device) */
    WALLY_ESTATE = 5    /* call out of order (e.g. eval before load_clusters) */
};

#define WALLY_MAX_LIMBS 8

typedef struct wally_ctx wally_ctx;

/* Parameter request (Sec. 7 "Parameters Selection"; the configurations this
 * library is measured on use N = 4096/8192/16384 and 36- or 50-bit limbs).
 * q_i = the num_q largest primes = 1 mod 2N below 2^q_bits, P = the next such
 * prime below q_{L-1}, t = the largest such prime below 2^t_bits, unless the
 * explicit overrides are given. */
typedef struct {
    uint32_t log_n;        /* 12, 13 or 14 */
    uint32_t num_q;        /* L, 1..WALLY_MAX_LIMBS-1 */
    uint32_t q_bits;       /* bit size of the ciphertext primes, <= 61 */
    uint32_t t_bits;       /* bit size of the plaintext prime, <= 30 */
    uint32_t dim;          /* embedding dimension d; d_pad = next power of two */
    int32_t device;        /* CUDA device ordinal */
    const uint64_t *q;     /* optional [num_q] explicit primes, NULL = derive */
    uint64_t p_special;    /* optional explicit P, 0 = derive */
    uint64_t t;            /* optional explicit t, 0 = derive */
    uint32_t max_wave;     /* queries per internal wave of wally_eval_batch, 0 = 1024 */
    uint32_t store;        /* cluster store: WALLY_STORE_AUTO / _NTT / _COMPACT (below) */
    uint32_t cache_chunks; /* compact store: encoded chunks held per lane, 0 = 16 */
    uint32_t baby_steps;   /* g of the diagonal split g x h = d_pad: 0 = 2^ceil(log2(d_pad)/2) (BSGS,
                              Sec. 4.1); d_pad = the plain diagonal method with no giant steps, which
                              Sec. 5 uses for clusters of sqrt(d) chunks or more (clusters may then have
                              up to d_pad - 1 chunks); any power of two from 2 to d_pad */
} wally_params;

/* How wally_load_clusters keeps the clusters.
 *  WALLY_STORE_NTT: every chunk's g*h plaintexts encoded, in NTT form, resident
 *    (d_pad * L * N * 8 bytes a chunk: 50 MB at N = 8192, L = 3, d_pad = 256;
 *    805 MB at N = 16384, L = 6, d_pad = 1024).
 *  WALLY_STORE_COMPACT: only the int8 embeddings are resident (d bytes a row);
 *    each wave encodes the chunks its queries name (the same kernel and the
 *    same bits as the NTT store) into a per-lane cache of cache_chunks chunks
 *    right before its multiply-accumulate.  Waves then also end where their
 *    clusters would need more than cache_chunks chunks, and the evaluation
 *    reads the per-cluster query counts back once per call (one host
 *    synchronisation of `stream`).  For databases whose encoded form exceeds
 *    device memory (1 M x 768 at N = 16384: 805 GB encoded, 768 MB as int8).
 *  WALLY_STORE_AUTO: NTT if the encoded clusters take at most 60 % of the
 *    free device memory when they are loaded, else COMPACT. */
#define WALLY_STORE_AUTO 0u
#define WALLY_STORE_NTT 1u
#define WALLY_STORE_COMPACT 2u

typedef struct {
    uint32_t n, log_n, num_q, dim, d_pad, g, h;
    uint32_t num_clusters;           /* after wally_load_clusters */
    uint64_t q[WALLY_MAX_LIMBS];
    uint64_t p_special, t, zeta_t;   /* zeta_t: the slot root (smallest x with x^N = -1 mod t) */
    uint64_t k1, kg;                 /* Galois elements of left rotation by 1 and by g */
    uint64_t ct_words;               /* 2*L*N */
    uint64_t keys_words;             /* 2*L*2*(L+1)*N */
    uint64_t total_chunks;           /* sum over clusters of their chunk counts */
    uint64_t cluster_bytes;          /* device bytes of the encoded clusters */
    uint32_t max_wave;
    uint32_t drop_c0, drop_c1;       /* low bits dropped from c0 / c1 of a compressed response */
    uint64_t compressed_bytes;       /* bytes of one compressed response ciphertext */
    uint32_t store;                  /* WALLY_STORE_NTT or _COMPACT once clusters are loaded, else the request */
    uint32_t cache_chunks;           /* compact store: chunks per lane cache */
} wally_info;

/* Derive primes, roots and NTT tables for `params` on `params->device` and
 * return a new context in *out.  Allocates only the tables (a few MB).
 * Errors: WALLY_EINVAL (unsupported sizes), WALLY_ECUDA, WALLY_ENOMEM. */
int wally_setup_params(const wally_params *params, wally_ctx **out);

/* Free the context and every device buffer it owns.  NULL is accepted. */
void wally_destroy(wally_ctx *ctx);

int wally_query_info(const wally_ctx *ctx, wally_info *out);

/* Server initialisation (Alg. "Server Initialization", Sec. 5): encode every
 * cluster into its plaintext set and keep it resident in device memory in NTT
 * form (or keep the embeddings and encode per wave: WALLY_STORE_COMPACT).  Cluster c has sizes[c] embeddings (rows of `embeddings`, host, int8
 * [sum sizes][dim], clusters back to back in id order).  Per cluster,
 * m = max(1, ceil(size/N)) chunks of g*h plaintexts; chunk k, slot
 * s = beta*d_pad + x holds embedding k*N + s, and plaintext (i, b) is diagonal
 * g*i + b rotated right by g*i within each row (BSGS pre-rotation).  Replaces
 * any previously loaded clusters.  Synchronises `stream` before returning.
 * Errors: WALLY_EINVAL (m >= g: the paper uses BSGS only while the number of
 * chunks is below sqrt(d), Sec. 5), WALLY_ENOMEM, WALLY_ECUDA. */
int wally_load_clusters(wally_ctx *ctx, uint32_t num_clusters, const uint32_t *sizes,
                        const int8_t *embeddings, void *stream);

/* Number of chunks m of a loaded cluster (= ciphertexts in its response). */
int wally_cluster_chunks(const wally_ctx *ctx, uint32_t cluster_id, uint32_t *m_out);

/* The encoded plaintexts of one cluster, back in coefficient form, residues
 * mod q_l: out (device) uint64_t [m][h][g][L][N].  For checking the encoder. */
int wally_export_cluster(wally_ctx *ctx, uint32_t cluster_id, uint64_t *out, void *stream);

/* Server computation for a batch (Alg. "Server Computation"; Sec. 5):
 *   ct'[0] = ct, ct'[j] = Rot_1(ct'[j-1]) for j < g        (baby steps)
 *   per chunk k of the query's cluster:
 *     T_i = sum_b P'_{k,i,b} * ct'[b]                      (i < h)
 *     S = T_{h-1}; S = Rot_g(S) + T_i for i = h-2 .. 0      (giant steps)
 *     out chunk k = S
 * Rot_r is the Galois automorphism X -> X^(3^r) followed by hybrid RNS key
 * switching with one-limb digits and the special prime P (Sec. 7).
 * Query q (0 <= q < n) names cluster cluster_ids[q], uses ciphertext
 * cts[src] and keys galois_keys[src] with src = input_index ? input_index[q]
 * : q, and writes its m ciphertexts to out[out_offsets[q] .. + m).
 *   cluster_ids  device uint32_t [n]
 *   cts          device uint64_t [*][2][L][N]
 *   galois_keys  device uint64_t [*][2][L][2][L+1][N]
 *   input_index  device uint32_t [n] or NULL
 *   out_offsets  device uint64_t [n]  (chunk offsets, e.g. exclusive prefix sums of m)
 *   out          device uint64_t [sum m][2][L][N], coefficient form, residues in [0, q_l)
 * Asynchronous on `stream`: queries are grouped by cluster on the device and
 * evaluated in waves of at most max_wave queries in scratch memory the
 * context owns (allocated on first use, grown when needed).  Consecutive
 * waves alternate between lanes 0 and 1 (see wally_eval_batch_lane), the odd
 * ones on a second stream of the context that forks from `stream` and joins
 * back into it before the call's work is complete on `stream`.  Queries with
 * an out-of-range cluster id produce no output and make wally_sync return
 * WALLY_EINVAL.  Calls on one context must not overlap (the scratch is
 * shared), nor with wally_eval_batch_lane on lanes 0 or 1.
 * Errors: WALLY_EINVAL, WALLY_ESTATE (no clusters), WALLY_ENOMEM, WALLY_ECUDA. */
int wally_eval_batch(wally_ctx *ctx, uint32_t n, const uint32_t *cluster_ids, const uint64_t *cts,
                     const uint64_t *galois_keys, const uint32_t *input_index, const uint64_t *out_offsets,
                     uint64_t *out, void *stream);

/* wally_eval_batch on one of WALLY_MAX_LANES independent workspaces
 * ("lanes") of the context.  Lanes share the context's tables and resident
 * clusters, so calls on different lanes may overlap on different streams
 * (continuous batching: a new wave is admitted on a free lane while others
 * are still running).  Calls on the same lane must not overlap.
 * wally_eval_batch is lane 0.  Each lane allocates its own workspace on first
 * use. */
#define WALLY_MAX_LANES 4
int wally_eval_batch_lane(wally_ctx *ctx, uint32_t lane, uint32_t n, const uint32_t *cluster_ids,
                          const uint64_t *cts, const uint64_t *galois_keys, const uint32_t *input_index,
                          const uint64_t *out_offsets, uint64_t *out, void *stream);

/* wally_eval_batch with HOST buffers (same layouts; cluster_ids, input_index,
 * out_offsets host arrays too).  Copies each wave's inputs to the device,
 * evaluates, and copies the results back; returns when `out` is filled.
 * Pinned host memory makes the copies asynchronous with the compute. */
int wally_eval_batch_host(wally_ctx *ctx, uint32_t n, const uint32_t *cluster_ids, const uint64_t *cts,
                          const uint64_t *galois_keys, const uint32_t *input_index,
                          const uint64_t *out_offsets, uint64_t *out, void *stream);

/* One rotation per ciphertext (Sec. 2 CtRotate; hybrid key switching of
 * Sec. 7): out[i] = Rot_k(cts[i]) with key keys[i] ([L][2][L+1][N], the key of
 * Galois element k).  k odd, 0 < k < 2N.  All device, coefficient form.
 * Asynchronous on `stream`. */
int wally_rotate(wally_ctx *ctx, uint32_t n, uint64_t galois_elt, const uint64_t *cts, const uint64_t *keys,
                 uint64_t *out, void *stream);

/* wally_rotate without any device allocation (the paper has no counterpart:
 * this is a service for callers, not a step of the method).  For callers
 * that must not call cudaMalloc/cudaFree at this point -- a serving thread
 * that cannot take the device-wide synchronisation those calls cause while
 * other streams run, or a process whose framework allocator already owns all
 * device memory.  Same arguments, layouts and results as wally_rotate.
 * Its scratch is one static device array of WALLY_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library keeps until exit; n is limited to
 *   WALLY_NOALLOC_SCRATCH_BYTES / (8 N (7L + 2 + 3L(L+1)))
 * ciphertexts (4 at N = 8192, L = 3); larger n returns WALLY_EINVAL.  At
 * N = 16384, L = 6 one ciphertext needs 22.3 MB, more than the array holds,
 * so every call with those parameters returns WALLY_EINVAL.  The first call
 * on a device looks up the array's device address (set-up) and keeps it for
 * the life of the process, so make it before any stream capture, and do not
 * reset the device (cudaDeviceReset) while the library is loaded: the kept
 * address would then be stale.  All calls share the array: calls whose
 * work overlaps on the GPU (other streams, other contexts on the device) race
 * and must be serialised by the caller.  Asynchronous on `stream`. */
#define WALLY_NOALLOC_SCRATCH_BYTES (16u << 20)
int wally_rotate_noalloc(wally_ctx *ctx, uint32_t n, uint64_t galois_elt, const uint64_t *cts,
                         const uint64_t *keys, uint64_t *out, void *stream);

/* Wait for `stream` and report the first device-side error recorded since
 * the previous wally_sync (and clear it). */
int wally_sync(wally_ctx *ctx, void *stream);

/* Response compression (Sec. 7 "Reducing the response size"): every score
 * ciphertext (device, [n][2][L][N], coefficient form, as wally_eval_batch
 * writes it) is switched to its last limb q' = q_{L-1} by a chain of exact
 * rescalings by q_0, ..., q_{L-2} (each replaces c by round(c / q_i), via the
 * centred residue mod q_i), then l0 = floor(log2(q'/t) - 2) low bits of c0
 * and l1 = floor(log2(q'/t) - 2 - log2(8 sqrt(2N/9))) of c1 are dropped with
 * rounding to nearest (wally_info.drop_c0 / drop_c1).  Each group of 8
 * coefficients packs into b bytes (b bits a value, little-endian bits),
 * component 0 then 1: out (device) [n][wally_info.compressed_bytes].
 * Asynchronous on `stream`. */
int wally_compress_responses(wally_ctx *ctx, uint32_t n, const uint64_t *cts, uint8_t *out, void *stream);

/* Client side: decrypt compressed responses (device [n][compressed_bytes])
 * with x = c0'' 2^l0 + c1'' 2^l1 s (mod q'), m = round(t x / q') mod t, and
 * decode the slots: scores device int64_t [n][N], centred; response i uses
 * secret[secret_index ? secret_index[i] : i]. */
int wally_decrypt_compressed(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                             const uint8_t *packed, int64_t *scores, void *stream);

/* ---------------------------------------------------------------- metadata: index PIR
 * The keyword PIR of Sec. 4.2 ("Details of keyword PIR") fetches the metadata
 * of one entry of a cluster: entries sit in two cuckoo tables (split tables:
 * one for each hash function), each table is a d1 x d2 matrix of plaintexts,
 * and the client runs an index PIR on each table (MulPIR).  The server side
 * of that index PIR built here is its query expansion and its first
 * dimension: the query ciphertext encrypts (2^c)^-1 X^row (c levels,
 * 2^c >= d1); the server expands it obliviously into 2^c ciphertexts (level
 * a: C -> C + sigma(C) and (C - sigma(C)) X^(-2^a), sigma the substitution
 * X -> X^(N/2^a + 1) with the client's key for it), so that ciphertext i
 * encrypts [i == row]; the answer is, per column j, sum_i table[i][j] *
 * ciphertext i, which decrypts to table[row][j] (wally_pir_answer, one
 * dimension: the answer holds all d2 columns).  wally_pir_answer2 adds
 * MulPIR's second dimension: the query encrypts (2^c)^-1 (X^row + X^(d1+col))
 * with 2^c >= d1 + d2, the expansion also yields the column indicators, and
 * the answer is one ciphertext, sum_j column_j x indicator_(d1+j), formed by
 * BFV ciphertext products (Sec. 2 CtCtMult: the tensor of the centred lifts,
 * scaled by t/Q and rounded; the d2 tensors are summed before the one
 * rescaling and the one relinearisation). */

/* Load the table: host uint64_t [rows][cols][N], plaintext coefficients in
 * [0, t).  rows (d1) 1..4096, cols (d2) >= 1.  The table is lifted centred
 * into the ciphertext moduli, kept in NTT form (device, rows*cols*L*N*8
 * bytes), and replaces any previous table.  Expansion levels c =
 * ceil(log2 rows).  Synchronises `stream`.
 * Errors: WALLY_EINVAL (sizes, a coefficient >= t), WALLY_ENOMEM, WALLY_ECUDA. */
int wally_pir_load(wally_ctx *ctx, uint32_t rows, uint32_t cols, const uint64_t *table, void *stream);

/* Answer n queries (all device buffers, coefficient form):
 *   queries  uint64_t [n][2][L][N]                 the clients' query ciphertexts
 *   keys     uint64_t [n][c][L][2][L+1][N]         per query, the key of N/2^a + 1 for level a < c
 *   out      uint64_t [n][cols][2][L][N]           column j of query q: table[row_q][j]
 * Asynchronous on `stream`; works on up to 64 queries at a time in scratch
 * the context owns (about 5 * 2^c ciphertexts a query at L = 3, plus its keys
 * and answer).
 * Errors: WALLY_ESTATE (no table), WALLY_EINVAL, WALLY_ENOMEM, WALLY_ECUDA. */
int wally_pir_answer(wally_ctx *ctx, uint32_t n, const uint64_t *queries, const uint64_t *keys, uint64_t *out,
                     void *stream);

/* MulPIR with both dimensions (see above): one answer ciphertext a query.
 *   queries     uint64_t [n][2][L][N]           encrypting (2^c)^-1 (X^row + X^(d1+col))
 *   keys        uint64_t [n][c][L][2][L+1][N]   c = ceil(log2(rows + cols)) substitution keys
 *   relin_keys  uint64_t [n][L][2][L+1][N]      wally_keygen_relin
 *   out         uint64_t [n][2][L][N]           decrypts to table[row][col]
 * The exact tensor is formed in an extension basis of L + K primes (K chosen
 * so that their product exceeds 2^(log2 N + 13) Q; L + K <= 7, so L <= 3 at
 * 50-bit limbs).  rows + cols <= 4096.  Asynchronous on `stream` after a
 * one-time set-up of the extension basis.  The noise of a product needs
 * log2(Q / t) well above log2(t N) + the noise of the operands: the
 * N = 8192, three 50-bit limb parameters qualify, N = 4096 with two 36-bit
 * limbs do not.
 * Errors: WALLY_ESTATE (no table), WALLY_EINVAL (sizes, L), WALLY_ENOMEM, WALLY_ECUDA. */
int wally_pir_answer2(wally_ctx *ctx, uint32_t n, const uint64_t *queries, const uint64_t *keys,
                      const uint64_t *relin_keys, uint64_t *out, void *stream);

/* Relinearisation keys (key switching from s^2 to s): key_a device
 * [n][L][L+1][N], key_e device int8 [n][L][N]; keys device [n][L][2][L+1][N]
 * with b_i = -a_i s + e_i + [i == j] P s^2 (mod q_j), b_i = -a_i s + e_i (mod P). */
int wally_keygen_relin(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint64_t *key_a, const int8_t *key_e,
                       uint64_t *keys, void *stream);

/* Sec. 4.2 "Reducing evaluation key size": (N/2^a + 1)^2 = N/2^(a-1) + 1
 * (mod 2N) while a <= floor((log2 N - 1) / 2), so with derivation enabled the
 * client sends only the keys of levels b .. c-1, b = min(c - 1,
 * floor((log2 N - 1) / 2)), and the server reaches every level a < b by
 * substituting 2^(b - a) times with the key of level b.  The keys arguments
 * of wally_pir_answer / wally_pir_answer2 then hold c - b keys a query
 * (levels b .. c-1).  Off by default; it changes the answer's bits (more
 * key switches), not what it decrypts to. */
int wally_pir_derive_keys(wally_ctx *ctx, int enable);

/* The expansion levels whose keys the client sends for the loaded table:
 * *first .. *first + *count - 1 (two_dims: for wally_pir_answer2). */
int wally_pir_key_levels(const wally_ctx *ctx, int two_dims, uint32_t *first, uint32_t *count);

/* Client side of the PIR.  Galois keys for a list of elements (at most 16):
 * galois (host) [num_keys], odd, < 2N; key_a device [n][num_keys][L][L+1][N],
 * key_e device int8 [n][num_keys][L][N]; keys device [n][num_keys][L][2][L+1][N]
 * (the same relation as wally_keygen). */
int wally_keygen_galois(wally_ctx *ctx, uint32_t n, uint32_t num_keys, const uint64_t *galois, const int8_t *secret,
                        const uint64_t *key_a, const int8_t *key_e, uint64_t *keys, void *stream);

/* Encrypt plaintext polynomials m (device uint64_t [n][N], coefficients in
 * [0, t)) as in wally_encrypt_query (no slot encoding): cts [n][2][L][N]. */
int wally_encrypt_poly(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint64_t *m, const uint64_t *enc_a,
                       const int8_t *enc_e, uint64_t *cts, void *stream);

/* Decrypt to plaintext coefficients: coeffs device int64_t [n][N] in [0, t);
 * ciphertext i uses secret[secret_index ? secret_index[i] : i].  Synchronous. */
int wally_decrypt_poly(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                       const uint64_t *cts, int64_t *coeffs, void *stream);

/* ---------------------------------------------------------------- measurement
 * Per-launch device time of the evaluation kernels, taken with CUDA events
 * recorded on the launch stream around every launch (observability; the
 * paper has no counterpart).  wally_profile_enable(ctx, 1) starts a fresh
 * collection, 0 stops it.  wally_profile_read synchronises the device, sums
 * launches and milliseconds per kernel kind into out[0 .. *count) (at most
 * cap entries) and clears the collection.  Launches captured in a CUDA graph
 * while profiling is on record their events as external nodes of the graph:
 * every replay rewrites them, and a read after replays reports the latest
 * replay (the same holds for wally_profile_waves). */
typedef struct {
    char name[16];       /* to_ntt, ks_a, ks_b, ks_c, mac, output, plan, encode (compact store) */
    uint64_t launches;
    double total_ms;
} wally_kernel_time;

int wally_profile_enable(wally_ctx *ctx, int enable);
int wally_profile_read(wally_ctx *ctx, wally_kernel_time *out, uint32_t cap, uint32_t *count);

/* Completion time of every wave of the evaluation calls (wally_eval_batch,
 * wally_eval_batch_lane, wally_eval_batch_host) made while profiling is on
 * (measurement only; the paper has no counterpart): for wave w in submission
 * order, call[w] = index of its call (0 = the first call since profiling was
 * enabled), queries[w] = the queries it evaluated, done_ms[w] = milliseconds
 * from the start of that call (an event recorded on the call's stream at its
 * entry) to the wave's outputs being written.  A query's latency inside a
 * batch is its wave's done_ms.  Synchronises the device, writes at most cap
 * entries of each non-NULL array, sets *count to the number of waves, and
 * clears the wave records (wally_profile_read does not clear them). */
int wally_profile_waves(wally_ctx *ctx, uint32_t cap, uint32_t *call, uint32_t *queries, float *done_ms,
                        uint32_t *count);

/* Throughput ceiling of the integer primitives on `device` (all SMs busy,
 * independent operations, no memory traffic): 64-bit Shoup modular
 * multiplications, NTT butterflies (the forward butterfly the transforms
 * use: one Shoup product written out in 32-bit multiply-adds plus three
 * 64-bit additions), and exact multiply-accumulates of operands below 2^56
 * into a 128-bit sum (in the kernels' form: four 32-bit multiply-adds on
 * 28-bit limbs), each in operations per second.  Used as the denominator of the integer-ALU
 * roofline.  Synchronous; allocates a few kilobytes. */
int wally_measure_int_peaks(int32_t device, double *modmul_per_s, double *butterfly_per_s, double *mac128_per_s);

/* Issue rates of the 32-bit instructions the modular arithmetic is built from
 * (observability; the paper has no counterpart), each with all SMs busy and
 * enough independent operations to keep the pipe full, in operations per
 * second: mad.lo.u32, mul.hi.u32 and mad.wide.u32 (all on the integer
 * multiplier).  sm_clock_hz: the SM clock (clock64 ticks of a CTA over the
 * event time of a launch of one CTA an SM).  bfly_ceiling_per_s: the rate at which the
 * multiplier could retire NTT butterflies if it did nothing else -- one
 * butterfly issues two mul.hi, three mad.wide and four mad.lo, so the
 * ceiling is 1 / (2/mul_hi + 3/mad_wide + 4/mad_lo).  Synchronous. */
typedef struct {
    double mad_lo_per_s;
    double mul_hi_per_s;
    double mad_wide_per_s;
    double sm_clock_hz;
    double bfly_ceiling_per_s;
} wally_pipe_rates;

int wally_measure_pipe_rates(int32_t device, wally_pipe_rates *out);

/* ---------------------------------------------------------------- launch shapes
 * The paper has no counterpart: these choose how the batch is laid onto this
 * GPU, never what is computed (every shape gives the same bits).
 *   max_wave         queries per wave (the wave workspace grows with it:
 *                    about 25 MB a query at N = 8192, L = 3)
 *   lanes            1: the waves of a wally_eval_batch call run in sequence
 *                    on the caller's stream; 2: they alternate between two
 *                    streams (lanes 0 and 1) so that one wave's kernels fill
 *                    the other's idle SMs
 *   mac_ctas_per_sm  1..3: resident CTAs per SM of the persistent
 *                    multiply-accumulate kernel (its grid)
 *   ntt_ctas_per_sm  0: as many transform-kernel CTAs per SM as shared memory
 *                    allows; k > 0: at most k (they are launched with more
 *                    shared memory than they use)
 *   ks_core          the NTT shape of the key-switch kernels: 0 = passes of
 *                    1 + 4 + 4 + 4 stages (N = 8192) over a shared-memory
 *                    polynomial, 16 coefficients a thread at a time, three
 *                    CTAs an SM; 1 = passes of 5 + 5 + 3 stages on 32
 *                    coefficients held in registers, two CTAs an SM
 *   mac_halves       0: the multiply-accumulate loads each plaintext tile
 *                    whole into one buffer; 1: it works on half tiles,
 *                    copying the next half into a second buffer while it
 *                    multiplies the current one
 * Defaults: 1024 (or the max_wave of wally_params), 2, 3, 0, 0, 0. */
typedef struct {
    uint32_t max_wave;
    uint32_t lanes;
    uint32_t mac_ctas_per_sm;
    uint32_t ntt_ctas_per_sm;
    uint32_t ks_core;
    uint32_t mac_halves;
} wally_tuning;

int wally_get_tuning(const wally_ctx *ctx, wally_tuning *out);

/* Errors: WALLY_EINVAL (max_wave 0, lanes not 1 or 2, mac_ctas_per_sm not
 * 1..3, ks_core or mac_halves not 0 or 1).  An ntt_ctas_per_sm at or above what shared memory allows anyway is
 * no cap.  Takes effect at the next call; it must not overlap running
 * evaluations of the context. */
int wally_set_tuning(wally_ctx *ctx, const wally_tuning *tuning);

/* Autotuner: evaluates the sample batch (the arguments of wally_eval_batch,
 * device buffers; `out` is overwritten) once untimed and `reps` times timed
 * with CUDA events on `stream` under each candidate shape, keeps the fastest
 * in the context and returns its index in *best.  With candidates non-NULL
 * the candidates are candidates[0 .. num_candidates).  With candidates NULL
 * (num_candidates 0) the search is staged: max_wave in {512, 1024, 2048} x
 * lanes in {1, 2} with mac 3, ntt 0, ks_core 0, mac_halves 0; then, at the
 * best of those, mac_ctas_per_sm in {2, 3} x ntt_ctas_per_sm in {0, 2}; then
 * the best so far with ks_core 1, then the best so far with mac_halves 1 (11
 * shapes in all).
 * tried (host, [WALLY_AUTOTUNE_MAX] or [num_candidates], may be NULL)
 * receives the shapes in the order timed, ms_per_query (same length, may be
 * NULL) their mean device milliseconds per query of the sample, or -1 where
 * the shape's workspace did not fit in device memory (skipped), and
 * *num_tried (may be NULL) their number.  Synchronous; frees the wave
 * workspaces between shapes.  For the timings to stand for a large batch,
 * the sample should hold several waves per lane of the largest max_wave.
 * Errors: WALLY_EINVAL, WALLY_ESTATE (no clusters), WALLY_ENOMEM (no shape
 * fits), WALLY_ECUDA. */
#define WALLY_AUTOTUNE_MAX 16
int wally_autotune(wally_ctx *ctx, const wally_tuning *candidates, uint32_t num_candidates, uint32_t reps,
                   uint32_t n, const uint32_t *cluster_ids, const uint64_t *cts, const uint64_t *galois_keys,
                   const uint32_t *input_index, const uint64_t *out_offsets, uint64_t *out,
                   wally_tuning *tried, double *ms_per_query, uint32_t *num_tried, uint32_t *best, void *stream);

/* ---------------------------------------------------------------- client side
 * Sec. 2 and Alg. "Client Query Generation".  The random numbers a client
 * draws are inputs, so that results are reproducible:
 *   secret   device int8_t [n][N]           ternary, in {-1, 0, 1}
 *   key_a    device uint64_t [n][2][L][L+1][N]  uniform, row j in [0, q_j) (j = L: P)
 *   key_e    device int8_t [n][2][L][N]     small errors
 *   enc_a    device uint64_t [n][L][N]      uniform in [0, q_l)
 *   enc_e    device int8_t [n][N]           small errors
 */

/* Galois keys for left rotations by 1 and by g (Sec. 7 "Reducing the request
 * size"): for key element k with s' = sigma_k(s), digit i:
 *   b_i = -a_i*s + e_i + [i == j] P s'  (mod q_j),   b_i = -a_i*s + e_i (mod P).
 * galois_keys: device uint64_t [n][2][L][2][L+1][N], coefficient form. */
int wally_keygen(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint64_t *key_a, const int8_t *key_e,
                 uint64_t *galois_keys, void *stream);

/* EncSemPt of the replicated query: queries device int8_t [n][dim] (a fake
 * query passes zeros).  Slot beta*d_pad + x holds q[x] for x < d, 0 above.
 * ct = (c0, c1) = (-a*s + e + Delta*m, a) with Delta = floor(Q/t) and m the
 * slot encoding of that vector, coefficients in [0, t).
 * cts: device uint64_t [n][2][L][N]. */
int wally_encrypt_query(wally_ctx *ctx, uint32_t n, const int8_t *secret, const int8_t *queries,
                        const uint64_t *enc_a, const int8_t *enc_e, uint64_t *cts, void *stream);

/* Decrypt score ciphertexts (Sec. 2: m = round(t/Q * [c0 + c1*s]_Q) mod t)
 * and decode the slots: scores device int64_t [n][N], centred into
 * (-t/2, t/2]; ciphertext i uses secret[secret_index[i]] (NULL: secret[i]).
 * The score of embedding k*N + s of the cluster is slot s of chunk k. */
int wally_decrypt_scores(wally_ctx *ctx, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                         const uint64_t *cts, int64_t *scores, void *stream);

/* Thread-local message of the last failing call on this thread. */
const char *wally_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WALLY_H */
