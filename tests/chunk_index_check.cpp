// Host check of the global store's chunk index (csrc/chunk_index.h) against
// std::map: random inserts and lookups over keys with negative coordinates,
// runs of neighbouring keys (the access pattern of a shift), overwrites, and
// a full enumeration. Prints "ok" and exits 0 on success.
#include <cstdio>
#include <map>
#include <random>
#include <tuple>

#include "chunk_index.h"

using tsdf::ChunkIndex;
using tsdf::ChunkKey;

int main() {
    std::mt19937_64 rng(12345);
    ChunkIndex idx;
    std::map<std::tuple<long long, long long, long long>, uint32_t> ref;
    auto check = [&](const ChunkKey& k) {
        auto it = ref.find(std::make_tuple(k.x, k.y, k.z));
        const long long want = it == ref.end() ? -1 : (long long)it->second;
        const long long got = idx.find(k);
        if (got != want) {
            std::printf("mismatch at (%lld, %lld, %lld): %lld != %lld\n", k.x, k.y, k.z, got, want);
            return false;
        }
        return true;
    };
    uint32_t next = 0;
    std::uniform_int_distribution<long long> wide(-3000, 3000), narrow(-40, 40);
    for (int round = 0; round < 60; ++round) {
        // a run of neighbouring chunks, as a shift enumerates them (x fastest)
        const long long x0 = wide(rng), y0 = wide(rng), z0 = narrow(rng);
        for (long long z = z0; z < z0 + 2; ++z)
            for (long long y = y0; y < y0 + 24; ++y)
                for (long long x = x0; x < x0 + 24; ++x) {
                    const ChunkKey k{x, y, z};
                    if (!check(k)) return 1;
                    if ((rng() & 3) != 0) {
                        const uint32_t v = next++;
                        idx.insert(k, v);
                        ref[std::make_tuple(x, y, z)] = v;
                    }
                    // interleave a lookup far away (the entering chunk of a shift)
                    if (!check(ChunkKey{-x - 17, y + 9, z - 3})) return 1;
                }
        // scattered keys, some overwritten
        for (int i = 0; i < 500; ++i) {
            const ChunkKey k{narrow(rng), narrow(rng), narrow(rng)};
            if (!check(k)) return 1;
            const uint32_t v = next++;
            idx.insert(k, v);
            ref[std::make_tuple(k.x, k.y, k.z)] = v;
            if (!check(k)) return 1;
        }
    }
    if (idx.size() != ref.size()) {
        std::printf("size %zu != %zu\n", idx.size(), ref.size());
        return 1;
    }
    size_t seen = 0;
    bool ok = true;
    idx.for_each([&](const ChunkKey& k, uint32_t v) {
        auto it = ref.find(std::make_tuple(k.x, k.y, k.z));
        if (it == ref.end() || it->second != v) ok = false;
        ++seen;
    });
    if (!ok || seen != ref.size()) {
        std::printf("enumeration: ok=%d seen=%zu of %zu\n", (int)ok, seen, ref.size());
        return 1;
    }
    std::printf("ok %zu keys\n", ref.size());
    return 0;
}
