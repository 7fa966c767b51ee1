// Host check of the global store's slot bookkeeping (csrc/chunk_store.h): a
// window of chunks walks back and forth over a line of chunk keys, some of
// which hold data. A fake two-tier memory records which chunk each slot
// holds, standing in for the shift kernel (which claims candidate slots, in a
// random order, only for leaving chunks that hold data) and the tier-to-tier
// copies. Checked after every shift:
// every chunk that holds data and is outside the window is stored exactly
// once, reads back as itself when it re-enters, no two chunks share a slot,
// empty chunks are not kept, device-tier use never exceeds its capacity, and
// the device chunks moved out are the ones stored longest ago. Prints "ok".
#include <algorithm>
#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "chunk_store.h"

using tsdf::ChunkKey;
using tsdf::ChunkStore;

int main() {
    std::mt19937_64 rng(777);
    const long long W = 24;                      // window: chunks [o, o + W) along x
    const uint32_t kDev = 40, kHost = 4096;       // tier capacities (slots)
    ChunkStore st;
    st.add_slots(0, 0, kDev);
    st.add_slots(1, 0, kHost);
    std::vector<long long> mem[2] = {std::vector<long long>(kDev, -1), std::vector<long long>(kHost, -1)};
    std::map<long long, bool> data;              // chunk x -> holds data (fixed per chunk)
    auto has = [&](long long x) {
        auto it = data.find(x);
        if (it == data.end()) it = data.emplace(x, (rng() % 3) != 0).first;
        return it->second;
    };
    auto at = [&](uint32_t loc) -> long long& {
        return mem[ChunkStore::is_host(loc) ? 1 : 0][ChunkStore::slot_of(loc)];
    };
    std::vector<int32_t> claim;
    std::set<long long> seen;                    // chunks that have been inside the window
    for (long long x = 0; x < W; ++x) seen.insert(x);
    long long o = 0;
    uint64_t serial = 0;
    size_t spilled = 0;
    for (int step = 0; step < 4000; ++step) {
        const long long d = (long long)(rng() % 9) - 4;   // shift by -4 .. +4 chunks
        const long long no = o + d;
        if (!claim.empty() || step > 0) st.commit(claim.data());
        std::vector<long long> leave, enter;
        for (long long x = o; x < o + W; ++x)
            if (x < no || x >= no + W) leave.push_back(x);
        for (long long x = no; x < no + W; ++x)
            if (x < o || x >= o + W) enter.push_back(x);
        // room: move the oldest device chunks out until the shift fits
        uint64_t last_stamp = 0;
        while (st.free_count(0) < leave.size()) {
            ChunkKey k;
            uint32_t loc0;
            uint64_t stamp;
            if (!st.oldest_device(&k, &loc0, &stamp)) break;
            if (stamp < last_stamp) { std::printf("spill order\n"); return 1; }
            last_stamp = stamp;
            uint32_t from, to;
            if (!st.spill_oldest(&from, &to) || from != loc0) { std::printf("spill failed\n"); return 1; }
            at(to) = at(from);
            at(from) = -2;
            ++spilled;
        }
        ++serial;
        std::vector<ChunkKey> keys;
        for (long long x : leave) keys.push_back(ChunkKey{x, 0, 0});
        std::vector<uint32_t> locs;
        if (!st.candidates(keys, serial, &locs) || locs.size() != keys.size()) { std::printf("no slots\n"); return 1; }
        for (long long x : enter) {
            const long long loc = st.take(ChunkKey{x, 0, 0});
            const bool stored = loc >= 0;
            if (stored != (has(x) && seen.count(x) > 0)) {
                std::printf("chunk %lld: stored %d, holds data %d\n", x, (int)stored, (int)has(x));
                return 1;
            }
            if (stored && at((uint32_t)loc) != x) {
                std::printf("chunk %lld read back %lld\n", x, at((uint32_t)loc));
                return 1;
            }
            seen.insert(x);
        }
        st.end_shift();
        // the kernel: the leaving chunks with data claim candidates in some order
        std::vector<size_t> order;
        for (size_t i = 0; i < leave.size(); ++i)
            if (has(leave[i])) order.push_back(i);
        std::shuffle(order.begin(), order.end(), rng);
        claim.assign(leave.size(), -1);
        for (size_t c = 0; c < order.size(); ++c) {
            claim[order[c]] = (int32_t)c;
            at(locs[c]) = leave[order[c]];
        }
        o = no;
        // invariants, with this shift committed on a copy
        ChunkStore copy = st;
        copy.commit(claim.data());
        std::set<uint32_t> locset;
        size_t n = 0;
        bool ok = true;
        copy.for_each([&](const ChunkKey& k, uint32_t loc) {
            ++n;
            if (!locset.insert(loc).second) ok = false;                    // shared slot
            if (k.x >= o && k.x < o + W) ok = false;                       // inside the window
            if (!has(k.x)) ok = false;                                     // empty chunk kept
            if (at(loc) != k.x) ok = false;                                // wrong contents
        });
        size_t want = 0;
        for (auto& kv : data)
            want += (kv.second && seen.count(kv.first) && (kv.first < o || kv.first >= o + W)) ? 1 : 0;
        if (!ok || n != want || copy.used(0) > kDev || copy.used(0) + copy.used(1) != n) {
            std::printf("step %d: ok=%d stored=%zu want=%zu dev=%zu host=%zu\n", step, (int)ok, n, want,
                        copy.used(0), copy.used(1));
            return 1;
        }
    }
    if (spilled == 0) { std::printf("no spill exercised\n"); return 1; }
    std::printf("ok %zu chunks known, %zu spilled\n", data.size(), spilled);
    return 0;
}
