// plan.cpp -- host-side wave planning (see plan.hpp).
#include "plan.hpp"

#include <algorithm>

namespace wally {

void fixed_waves(uint32_t n, uint32_t W, std::vector<Wave> &waves)
{
    waves.clear();
    for (uint32_t wb = 0; wb < n; wb += W) waves.push_back(Wave{wb, std::min(W, n - wb), 0, 0});
}

void compact_waves(const uint32_t *chunks, uint32_t K, uint32_t C, const uint32_t *cnt, uint32_t W,
                   std::vector<Wave> &waves, std::vector<uint32_t> &zc, std::vector<uint32_t> &zk)
{
    waves.clear();
    zc.clear();
    zk.clear();
    uint32_t pos = 0;
    Wave cur{0, 0, 0, 0};
    for (uint32_t k = 0; k < K; k++) {
        uint32_t rem = cnt[k];
        const uint32_t m = chunks[k];
        while (rem) {
            if (cur.len == W || cur.nz + m > C) {
                waves.push_back(cur);
                cur = Wave{pos, 0, (uint32_t)zc.size(), 0};
            }
            const uint32_t take = std::min(rem, W - cur.len);
            for (uint32_t j = 0; j < m; j++) {
                zc.push_back(k);
                zk.push_back(j);
            }
            cur.nz += m;
            cur.len += take;
            rem -= take;
            pos += take;
        }
    }
    if (cur.len) waves.push_back(cur);
}

}  // namespace wally
