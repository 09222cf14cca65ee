// plan.hpp -- host-side wave planning of a batch (no CUDA): how the
// cluster-sorted queries of one wally_eval_batch call are cut into waves.
#pragma once
#include <cstdint>
#include <vector>

namespace wally {

// One wave: positions [begin, begin + len) of the cluster-sorted order and,
// with the compact cluster store, its nz chunks (entries z_off .. of the
// chunk list) to encode before its multiply-accumulate.
struct Wave {
    uint32_t begin, len, z_off, nz;
};

// Fixed waves of at most W positions (the NTT store).
void fixed_waves(uint32_t n, uint32_t W, std::vector<Wave> &waves);

// Compact store: cluster k (k < K, chunks[k] chunks) holds positions
// [start_k, start_k + cnt[k]) of the sorted order (clusters in id order).  A
// wave ends at W queries or where its clusters would need more than C
// encoded chunks (C >= every chunks[k]); a cluster split between waves is
// encoded in each.  zc / zk: (cluster, chunk) of every wave's chunks, a
// cluster's chunks consecutive.
void compact_waves(const uint32_t *chunks, uint32_t K, uint32_t C, const uint32_t *cnt, uint32_t W,
                   std::vector<Wave> &waves, std::vector<uint32_t> &zc, std::vector<uint32_t> &zk);

}  // namespace wally
