// Host bookkeeping of the global chunk store (used by api.cu; plain C++ with
// no CUDA dependency, so that it is also unit-tested on the host).
//
// The global map outside the window is kept as 8^3 chunks of 2 KiB in up to
// three tiers of slots: tier 0 in device memory, tier 1 in pinned host memory
// that the device reads and writes in place, and, optionally, tier 2 in a
// file (records the host writes and reads; the device never addresses them).
// This class only decides which slot holds which chunk; the owner allocates
// the memory behind the slots (it adds slots with add_slots), copies chunks
// between tiers and runs the shift.
//
// A shift hands its kernel one candidate slot per leaving chunk (candidates:
// device-tier slots first), and the kernel claims candidates in order for the
// leaving chunks that hold data: the claimed ones form a prefix of the list.
// The next call of commit() records the claimed chunks and frees the unclaimed
// candidates, so chunks without data never enter the index. Entering chunks
// are looked up and removed (take); their slots are freed by end_shift(),
// after the candidates of the same shift are out of the free lists, so that no
// slot is read and written by one kernel. Device-tier chunks are queued in the
// order they were stored, so that the oldest can be moved to the host tier
// first (oldest_device, spill_oldest); host-tier chunks are queued in the
// order they entered that tier, so that the oldest move to the file first
// (spill_oldest_host). A chunk in the file tier is read back into a host slot
// (take_slot) before the shift kernel reads it.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

#include "chunk_index.h"

namespace tsdf {

class ChunkStore {
public:
    static constexpr uint32_t kHostBit = 0x80000000u;   // location = tier bit | slot
    static constexpr uint32_t kFileBit = 0x40000000u;   // (slots stay below 2^30)
    static bool is_host(uint32_t loc) { return (loc & kHostBit) != 0; }
    static bool is_file(uint32_t loc) { return (loc & kFileBit) != 0; }
    static int tier_of(uint32_t loc) { return is_host(loc) ? 1 : (is_file(loc) ? 2 : 0); }
    static uint32_t slot_of(uint32_t loc) { return loc & ~(kHostBit | kFileBit); }
    static uint32_t loc_of(int tier, uint32_t slot) { return slot | (tier == 1 ? kHostBit : tier == 2 ? kFileBit : 0u); }

    // New free slots [first, first + n) of a tier (0 device, 1 host, 2 file).
    void add_slots(int tier, uint32_t first, uint32_t n) {
        for (uint32_t i = 0; i < n; ++i) free_[tier].push_back(first + n - 1 - i);   // lowest slot popped first
        cap_[tier] += n;
    }
    size_t capacity(int tier) const { return cap_[tier]; }
    size_t free_count(int tier) const { return free_[tier].size(); }
    // slots not free: stored chunks plus the candidates of a shift not yet committed
    size_t used(int tier) const { return cap_[tier] - free_[tier].size(); }
    size_t chunks() const { return index_.size(); }
    bool pending() const { return !cand_.empty(); }

    // location of a stored chunk, or -1
    long long find(const ChunkKey& k) { return index_.find(k); }

    // Candidate slots for a shift whose leaving chunks are `keys` (in the
    // kernel's item order): `locs` receives one location per key, device tier
    // first; false when the tiers have fewer free slots (nothing is taken).
    bool candidates(const std::vector<ChunkKey>& keys, uint64_t stamp, std::vector<uint32_t>* locs) {
        const size_t n = keys.size();
        if (free_[0].size() + free_[1].size() < n) return false;
        locs->resize(n);
        for (size_t i = 0; i < n; ++i) {
            if (!free_[0].empty()) {
                (*locs)[i] = free_[0].back();
                free_[0].pop_back();
            } else {
                (*locs)[i] = free_[1].back() | kHostBit;
                free_[1].pop_back();
            }
        }
        cand_ = *locs;
        keys_ = keys;
        stamp_ = stamp;
        return true;
    }

    // The last shift's outcome: claim[i] is the candidate index the kernel
    // claimed for leaving chunk i, or -1 when the chunk held no data. Claimed
    // chunks are recorded (device-tier ones queued by age), unclaimed
    // candidates freed. Returns the number of chunks stored.
    size_t commit(const int32_t* claim) {
        size_t stored = 0;
        for (size_t i = 0; i < keys_.size(); ++i) {
            const int32_t c = claim[i];
            if (c < 0 || (size_t)c >= cand_.size()) continue;
            const uint32_t loc = cand_[(size_t)c];
            index_.insert(keys_[i], loc);
            if (!is_host(loc)) fifo_.push_back(Entry{keys_[i], loc, stamp_});
            else fifo_host_.push_back(Entry{keys_[i], loc, stamp_});
            cand_[(size_t)c] = kClaimed;
            ++stored;
        }
        for (uint32_t loc : cand_)
            if (loc != kClaimed) release(loc);
        cand_.clear();
        keys_.clear();
        if (fifo_.size() > 64 && fifo_.size() > 2 * index_.size()) compact_fifo(&fifo_);
        if (fifo_host_.size() > 64 && fifo_host_.size() > 2 * index_.size()) compact_fifo(&fifo_host_);
        return stored;
    }

    // An entering chunk: its location (or -1 when it is not stored), removed
    // from the index; the slot is freed by end_shift().
    long long take(const ChunkKey& k) {
        const long long loc = index_.find(k);
        if (loc >= 0) {
            index_.erase(k);
            taken_.push_back((uint32_t)loc);
        }
        return loc;
    }

    // A free slot of `tier` that is freed again by end_shift() (a host slot
    // into which an entering file-tier chunk is read), or -1 when the tier
    // has no free slot.
    long long take_slot(int tier) {
        if (free_[tier].empty()) return -1;
        const uint32_t loc = loc_of(tier, free_[tier].back());
        free_[tier].pop_back();
        taken_.push_back(loc);
        return (long long)loc;
    }

    // After a shift's candidates are out: the entering chunks' slots become free.
    void end_shift() {
        for (uint32_t loc : taken_) release(loc);
        taken_.clear();
    }

    // The device-tier chunk stored longest ago (and when), without removing it;
    // false when the device tier holds none.
    bool oldest_device(ChunkKey* k, uint32_t* loc, uint64_t* stamp) {
        while (!fifo_.empty()) {
            const Entry& e = fifo_.front();
            if (index_.find(e.key) == (long long)e.loc) {
                *k = e.key;
                *loc = e.loc;
                *stamp = e.stamp;
                return true;
            }
            fifo_.pop_front();   // the chunk re-entered or moved
        }
        return false;
    }

    // Move the oldest device-tier chunk to a free host-tier slot: returns
    // false when there is none to move or no free host slot; else the two
    // locations (the caller copies the chunk before the device slot is used
    // again: the device slot is free at once).
    bool spill_oldest(uint32_t* from, uint32_t* to) {
        ChunkKey k;
        uint32_t loc;
        uint64_t stamp;
        if (free_[1].empty() || !oldest_device(&k, &loc, &stamp)) return false;
        fifo_.pop_front();
        const uint32_t h = free_[1].back() | kHostBit;
        free_[1].pop_back();
        index_.insert(k, h);
        fifo_host_.push_back(Entry{k, h, stamp});
        release(loc);
        *from = loc;
        *to = h;
        return true;
    }

    // The same from the host tier to the file tier: the oldest host-tier
    // chunk (by when it entered that tier) moves to a free file slot; false
    // when the host tier holds none or no file slot is free. The host slot is
    // free at once (the caller writes the chunk out first).
    bool spill_oldest_host(uint32_t* from, uint32_t* to) {
        if (free_[2].empty()) return false;
        while (!fifo_host_.empty()) {
            const Entry e = fifo_host_.front();
            fifo_host_.pop_front();
            if (index_.find(e.key) != (long long)e.loc) continue;   // re-entered or moved
            const uint32_t f = free_[2].back() | kFileBit;
            free_[2].pop_back();
            index_.insert(e.key, f);
            release(e.loc);
            *from = e.loc;
            *to = f;
            return true;
        }
        return false;
    }

    // Every stored chunk (after commit(): a shift's candidates are not listed).
    template <typename F>
    void for_each(F&& f) const { index_.for_each(f); }

    // A chunk written directly (loading a saved map): a free slot, device tier
    // first, recorded as stored; -1 when both memory tiers are full.
    long long insert_stored(const ChunkKey& k, uint64_t stamp) {
        uint32_t loc;
        if (!free_[0].empty()) {
            loc = free_[0].back();
            free_[0].pop_back();
            fifo_.push_back(Entry{k, loc, stamp});
        } else if (!free_[1].empty()) {
            loc = free_[1].back() | kHostBit;
            free_[1].pop_back();
            fifo_host_.push_back(Entry{k, loc, stamp});
        } else {
            return -1;
        }
        index_.insert(k, loc);
        return (long long)loc;
    }

private:
    static constexpr uint32_t kClaimed = 0xFFFFFFFFu;
    struct Entry {
        ChunkKey key;
        uint32_t loc;
        uint64_t stamp;
    };
    void release(uint32_t loc) { free_[tier_of(loc)].push_back(slot_of(loc)); }
    void compact_fifo(std::deque<Entry>* q) {
        std::deque<Entry> keep;
        for (const Entry& e : *q)
            if (index_.find(e.key) == (long long)e.loc) keep.push_back(e);
        q->swap(keep);
    }
    ChunkIndex index_;
    std::vector<uint32_t> free_[3];
    size_t cap_[3] = {0, 0, 0};
    std::vector<uint32_t> cand_;     // the last shift's candidate slots (kClaimed once recorded)
    std::vector<ChunkKey> keys_;     // the last shift's leaving chunks, in item order
    uint64_t stamp_ = 0;
    std::vector<uint32_t> taken_;
    std::deque<Entry> fifo_;         // device-tier chunks in the order they were stored (stale entries skipped)
    std::deque<Entry> fifo_host_;    // host-tier chunks in the order they entered that tier (likewise)
};

}  // namespace tsdf
