// The dataset-eviction policy of the library (dataset_lru.h) behind a C interface for ctypes
// (test infrastructure).
#include <cstdint>
#include <vector>

#include "dataset_lru.h"

extern "C" int lru_victims(const uint64_t *ids, const uint64_t *bytes, const uint64_t *last_use,
                           const uint8_t *resident, const uint8_t *evictable, int n, uint64_t used,
                           uint64_t need, uint64_t budget, uint64_t keep, uint64_t *out)
{
    std::vector<rs::lru::Entry> e;
    for (int i = 0; i < n; ++i) e.push_back({ids[i], bytes[i], last_use[i], resident[i] != 0, evictable[i] != 0});
    const std::vector<uint64_t> v = rs::lru::victims(e, used, need, budget, keep);
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
    return (int)v.size();
}
