// kernels.hpp -- launchers of the device kernels (host side).  Every
// launcher enqueues on `st` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace wally {

// A batch of independent rotations Rot_k (automorphism + hybrid key switch,
// Sec. 2 CtRotate, Sec. 7).  Item x reads ciphertext src + x*src_stride
// (NTT form), writes dst + x*dst_stride (NTT form), adds add + x*add_stride
// when add != nullptr (the Horner step S = Rot_g(S) + T_i), and uses the key
// (NTT form, Montgomery scaled, [L][2][L+1][N]) at
// key + (key_map ? key_map[x] : x) * key_stride.  Item count: *n_dev when
// n_dev != nullptr (bounded by n_max), else n_max.  Scratch sc [n][2][L][N]
// (the automorphism of the input, NTT form), dg [n][L][N] (digits),
// u [n][2][L+1][N] (key products), dd [n][L+1][L][N] (transformed digits).
// prepared: sc and dg already hold this rotation's input (the previous
// rotation of the chain wrote them), so src is not read.  next_galois != 0:
// also prepare sc and dg for a following rotation by that element.
struct RotArgs {
    const u64 *src;
    size_t src_stride;
    u64 *dst;
    size_t dst_stride;
    const u64 *add;
    size_t add_stride;
    const u64 *key;
    size_t key_stride;
    const u32 *key_map;
    u32 n_max;
    const u32 *n_dev;
    u64 galois;
    u64 next_galois;
    bool prepared;
    u64 *sc, *dg, *u, *dd;
};

// Per-wave plan, all device arrays sized for max_wave queries (pairs: x m_max).
struct WavePlan {
    u32 *counts;          // [0] queries in the wave, [1] (query, chunk) pairs, [2] segments
    u32 *cluster;         // [W] cluster of wave position (grouped by cluster)
    const u64 **src_ct;   // [W] input ciphertext (coefficient form)
    const u64 **src_key;  // [W] input keys (coefficient form, both keys)
    u64 **dst_out;        // [W] output of chunk 0 (chunk k at + k*2LN)
    u32 *pair_pos;        // [W*m_max] wave position of pair
    u32 *pair_k;          // [W*m_max] chunk of pair
    u32 *pair_off;        // [W+1] first pair of wave position
    u32 *seg_cluster;     // [W] segments: maximal runs of one cluster
    u32 *seg_begin, *seg_end;
};

// Encoded clusters: plaintext (z = global chunk, i, b, limb l, slot position s)
// lives at ((z*L + l)*(N/ts) + s/ts)*(d_pad*ts) + (i*g + b)*ts + s%ts, in NTT
// form, Montgomery scaled; ts slots per tile (d_pad*ts*8 bytes = one tile).
struct ClusterStore {
    const u64 *ptxt;
    const u32 *chunk0;  // [K] first global chunk of cluster
    const u32 *chunks;  // [K] chunk count m
    u32 ts;
};

// Optional timing of every launch with CUDA events on the launch stream.
enum KernelKind { KK_TO_NTT = 0, KK_KS_A, KK_KS_B, KK_KS_C, KK_MAC, KK_OUTPUT, KK_PLAN, KK_ENCODE, KK_COUNT };
struct Profiler {
    virtual void begin(int kind, cudaStream_t st) = 0;
    virtual void end(int kind, cudaStream_t st) = 0;
    virtual ~Profiler() {}
};

cudaError_t set_kernel_attributes(int log_n, u32 g);

cudaError_t launch_to_ntt(const DevParams &dp, const u64 *const *src_ptrs, const u64 *src, size_t src_stride,
                          u64 *dst, size_t dst_stride, u32 polys, u32 mod_cycle, u32 n_max, const u32 *n_dev,
                          bool mont, cudaStream_t st, Profiler *pr = nullptr);
cudaError_t launch_rotate(const DevParams &dp, const RotArgs &a, cudaStream_t st, Profiler *pr = nullptr);
cudaError_t launch_mac(const DevParams &dp, const ClusterStore &cs, const WavePlan &wp, const u64 *ctp, u64 *T,
                       u32 max_wave, u32 m_max, int num_sms, cudaStream_t st, Profiler *pr = nullptr);
// Output: pair p (INTT of S + p*S_stride) -> dst_out[pair_pos[p]] + pair_k[p]*2LN.
cudaError_t launch_output(const DevParams &dp, const WavePlan &wp, const u64 *S, size_t S_stride, u32 n_max,
                          cudaStream_t st, Profiler *pr = nullptr);
// Plain coefficient <-> NTT for wally_rotate.
cudaError_t launch_from_ntt(const DevParams &dp, const u64 *src, u64 *dst, u32 polys_per_item, u32 mod_cycle,
                            u32 n_items, cudaStream_t st);

// Device-side grouping of a batch by cluster (a0) and the per-wave plan.
cudaError_t launch_group(const u32 *ids, u32 n, u32 num_clusters, u32 *counts, u32 *cstart, u32 *fill,
                         u32 *sorted_q, u32 *err, cudaStream_t st);
cudaError_t launch_gather_wave(const WavePlan &wp, const u32 *sorted_q, const u32 *ids, const u32 *cstart,
                               u32 num_clusters, u32 wave_begin, u32 wave_len, const u64 *cts, const u64 *keys,
                               const u32 *input_index, const u64 *out_offsets, u64 *out, size_t ct_words,
                               size_t keys_words, cudaStream_t st);
cudaError_t launch_wave_plan(const WavePlan &wp, const u32 *cluster_chunks, u32 wave_len_max, cudaStream_t st,
                             Profiler *pr = nullptr);

// Setup: encode clusters (Alg. "Server Initialization").
struct EncodeArgs {
    const int8_t *emb;   // [sum sizes][d]
    const u64 *row0;     // [K] first row of cluster
    const u32 *size;     // [K]
    const u32 *chunk_cluster;  // [Z]
    const u32 *chunk_k;        // [Z]
    u32 total_chunks;
    u64 *ptxt;
    u32 ts;
    u32 *chunk0_out;     // optional [K]: chunk0_out[c] = local index of chunk (c, 0)
};
size_t ntt_smem_need(int log_n);  // shared memory a transform kernel needs
cudaError_t launch_encode_clusters(const DevParams &dp, const EncodeArgs &a, cudaStream_t st, Profiler *pr = nullptr);
cudaError_t launch_export_cluster(const DevParams &dp, const ClusterStore &cs, u32 cluster, u32 m, u64 *out,
                                  cudaStream_t st);

// Client side.
cudaError_t launch_encode_queries(const DevParams &dp, const int8_t *queries, u32 n, u64 *m_out, cudaStream_t st);
cudaError_t launch_encrypt(const DevParams &dp, const int8_t *secret, const u64 *m, const u64 *enc_a,
                           const int8_t *enc_e, u32 n, u64 *cts, cudaStream_t st);
cudaError_t launch_keygen(const DevParams &dp, const int8_t *secret, const u64 *key_a, const int8_t *key_e, u32 n,
                          u64 k1, u64 kg, u64 k1_inv, u64 kg_inv, u64 *keys, cudaStream_t st);
// Response compression (switch to the last limb, drop low bits, pack).
cudaError_t launch_compress(const DevParams &dp, const u64 *cts, u32 n, uint8_t *out, u32 l0, u32 l1, u32 b0, u32 b1,
                            cudaStream_t st);
cudaError_t launch_decrypt_compressed(const DevParams &dp, const int8_t *secret, const u32 *secret_index,
                                      const uint8_t *packed, u32 n, u32 l0, u32 l1, u32 b0, u32 b1, int64_t *scores,
                                      cudaStream_t st);
cudaError_t launch_decrypt(const DevParams &dp, const int8_t *secret, const u32 *secret_index, const u64 *cts, u32 n,
                           u64 *xs, int64_t *scores, cudaStream_t st);

}  // namespace wally
