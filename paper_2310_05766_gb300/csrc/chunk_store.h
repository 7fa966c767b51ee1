// Host bookkeeping of the global chunk store (used by api.cu; plain C++ with
// no CUDA dependency, so that it is also unit-tested on the host).
//
// The global map outside the window is kept as 8^3 chunks of 2 KiB in two
// tiers of slots: tier 0 in device memory, tier 1 in pinned host memory that
// the device reads and writes in place. This class only decides which slot
// holds which chunk; the owner allocates the memory behind the slots (it adds
// slots with add_slots), copies chunks between tiers and runs the shift.
//
// A shift hands every leaving chunk a slot before the shift kernel runs
// (place), but the kernel writes only the chunks that hold data; it reports
// per candidate whether it did, and the next call of resolve() drops the
// empty ones and frees their slots. Entering chunks are looked up and removed
// (take); their slots are freed by end_shift(), after the leaving chunks of the
// same shift have their slots, so that no slot is read and written by one
// kernel. Device-tier chunks are queued in the order they were stored, so that
// the oldest can be moved to the host tier first (oldest_device).
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
    static bool is_host(uint32_t loc) { return (loc & kHostBit) != 0; }
    static uint32_t slot_of(uint32_t loc) { return loc & ~kHostBit; }

    // New free slots [first, first + n) of a tier (0 device, 1 host).
    void add_slots(int tier, uint32_t first, uint32_t n) {
        for (uint32_t i = 0; i < n; ++i) free_[tier].push_back(first + n - 1 - i);   // lowest slot popped first
        cap_[tier] += n;
    }
    size_t capacity(int tier) const { return cap_[tier]; }
    size_t free_count(int tier) const { return free_[tier].size(); }
    size_t used(int tier) const { return cap_[tier] - free_[tier].size(); }
    // chunks known to the index (stored ones, plus candidates of the last
    // shift not yet resolved)
    size_t chunks() const { return index_.size(); }
    bool pending() const { return !pend_.empty(); }

    // location of a stored chunk, or -1
    long long find(const ChunkKey& k) { return index_.find(k); }

    // The previous shift's candidates, in the order place() handed them out:
    // flags[i] != 0 when candidate i was written (it held data); the others
    // are dropped and their slots freed.
    void resolve(const uint8_t* flags) {
        for (size_t i = 0; i < pend_.size(); ++i) {
            if (flags[i]) continue;
            const Pending& p = pend_[i];
            if (index_.find(p.key) == (long long)p.loc) {
                index_.erase(p.key);
                release(p.loc);
            }
        }
        pend_.clear();
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

    // A leaving chunk: a slot for it, from the device tier while it has free
    // slots, else from the host tier; -1 when neither has one (the owner adds
    // slots first). Recorded as a candidate of this shift.
    long long place(const ChunkKey& k, uint64_t stamp) {
        uint32_t loc;
        if (!free_[0].empty()) {
            loc = free_[0].back();
            free_[0].pop_back();
            fifo_.push_back(Entry{k, loc, stamp});
        } else if (!free_[1].empty()) {
            loc = free_[1].back() | kHostBit;
            free_[1].pop_back();
        } else {
            return -1;
        }
        index_.insert(k, loc);
        pend_.push_back(Pending{k, loc});
        return (long long)loc;
    }

    // After a shift's place() calls: the entering chunks' slots become free.
    void end_shift() {
        for (uint32_t loc : taken_) release(loc);
        taken_.clear();
        if (fifo_.size() > 64 && fifo_.size() > 2 * index_.size()) compact_fifo();
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
            fifo_.pop_front();   // the chunk re-entered, was dropped, or moved
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
        release(loc);
        *from = loc;
        *to = h;
        return true;
    }

    // Every stored chunk (call after resolve(): unresolved candidates are listed too).
    template <typename F>
    void for_each(F&& f) const { index_.for_each(f); }

    // A chunk written directly (loading a saved map): a slot as place()
    // gives, not a candidate (it is known to hold data).
    long long insert_stored(const ChunkKey& k, uint64_t stamp) {
        const long long loc = place(k, stamp);
        if (loc >= 0) pend_.pop_back();
        return loc;
    }

private:
    struct Entry {
        ChunkKey key;
        uint32_t loc;
        uint64_t stamp;
    };
    struct Pending {
        ChunkKey key;
        uint32_t loc;
    };
    void release(uint32_t loc) {
        if (is_host(loc)) free_[1].push_back(slot_of(loc));
        else free_[0].push_back(loc);
    }
    void compact_fifo() {
        std::deque<Entry> keep;
        for (const Entry& e : fifo_)
            if (index_.find(e.key) == (long long)e.loc) keep.push_back(e);
        fifo_.swap(keep);
    }
    ChunkIndex index_;
    std::vector<uint32_t> free_[2];
    size_t cap_[2] = {0, 0};
    std::vector<Pending> pend_;
    std::vector<uint32_t> taken_;
    std::deque<Entry> fifo_;   // device-tier chunks in the order they were stored (stale entries skipped)
};

}  // namespace tsdf
