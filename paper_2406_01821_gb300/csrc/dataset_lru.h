// Choice of the datasets to evict under a device-memory budget for a context's datasets, free of
// CUDA: the policy that the registry (runtime.cu) applies and that a CPU test drives directly.
//
// A context with a dataset budget keeps every dataset's data on the host as well; when registering
// or using a dataset would take the resident datasets beyond the budget, the least recently used
// resident datasets that nothing is using are evicted (their device copies freed) until it fits,
// and an evicted dataset is rebuilt on the device the next time a call names it. A dataset in use
// (a call running on it, a serving request queued or running on it), one without a host copy, or
// the one being made resident is never chosen; when not enough can be evicted the budget is
// exceeded rather than the call refused.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace rs {
namespace lru {

struct Entry {
    uint64_t id = 0;
    size_t bytes = 0;          // device bytes while resident
    uint64_t last_use = 0;     // larger is more recent
    bool resident = false;
    bool evictable = false;    // a host copy exists and nothing is using the dataset
};

// Ids to evict, least recently used first, so that used - their bytes + need <= budget; `keep` is
// never chosen. Returns as many as help (possibly fewer than needed) or none when it already fits.
inline std::vector<uint64_t> victims(std::vector<Entry> entries, size_t used, size_t need, size_t budget,
                                     uint64_t keep)
{
    std::vector<uint64_t> out;
    if (budget == 0 || used + need <= budget) return out;
    std::sort(entries.begin(), entries.end(), [](const Entry &a, const Entry &b) {
        return a.last_use != b.last_use ? a.last_use < b.last_use : a.id < b.id;
    });
    for (const Entry &e : entries) {
        if (used + need <= budget) break;
        if (!e.resident || !e.evictable || e.id == keep) continue;
        out.push_back(e.id);
        used -= std::min(used, e.bytes);
    }
    return out;
}

}  // namespace lru
}  // namespace rs
