// Host index of the global chunk store (used by api.cu; a plain C++ header
// with no CUDA dependency, so that it is also unit-tested on the host).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace tsdf {

struct ChunkKey {
    long long x, y, z;
    bool operator==(const ChunkKey& o) const { return x == o.x && y == o.y && z == o.z; }
};

// Index of the global store: chunk key -> store location, in two levels. Chunks
// are grouped into 8 x 8 x 8 super-chunks; an open-addressing hash table
// (linear probing, grown by doubling at half load) maps a super-chunk key to
// a block of 512 slots. A shift works on a few dozen neighbouring
// super-chunks, so the blocks found recently are kept in a small direct-mapped
// cache (and the last super-chunk found absent is remembered): most lookups
// are one array access instead of a probe of the table.
class ChunkIndex {
public:
    ChunkIndex() {
        for (size_t i = 0; i < kCache; ++i) cache_blk_[i] = -1;
    }
    // slot of `k`, or -1
    long long find(const ChunkKey& k) {
        const uint32_t* b = block(super(k), false);
        if (!b) return -1;
        const uint32_t v = b[local(k)];
        return v == kNone ? -1 : (long long)v;
    }
    void insert(const ChunkKey& k, uint32_t v) {
        uint32_t* b = block(super(k), true);
        uint32_t& e = b[local(k)];
        if (e == kNone) ++count_;
        e = v;
    }
    void erase(const ChunkKey& k) {
        uint32_t* b = block(super(k), false);
        if (!b) return;
        uint32_t& e = b[local(k)];
        if (e != kNone) {
            e = kNone;
            --count_;
        }
    }
    size_t size() const { return count_; }
    template <typename F>
    void for_each(F&& f) const {
        for (size_t i = 0; i < keys_.size(); ++i) {
            if (!used_[i]) continue;
            const uint32_t* b = &slots_[(size_t)vals_[i] * 512];
            for (int j = 0; j < 512; ++j)
                if (b[j] != kNone)
                    f(ChunkKey{keys_[i].x * 8 + (j & 7), keys_[i].y * 8 + ((j >> 3) & 7), keys_[i].z * 8 + (j >> 6)},
                      b[j]);
        }
    }

private:
    static constexpr uint32_t kNone = 0xFFFFFFFFu;
    // floor division by 8 and the remainder (arithmetic shift on the signed keys)
    static ChunkKey super(const ChunkKey& k) { return ChunkKey{k.x >> 3, k.y >> 3, k.z >> 3}; }
    static int local(const ChunkKey& k) { return (int)(((k.z & 7) << 6) | ((k.y & 7) << 3) | (k.x & 7)); }
    // the 512 slots of super-chunk `s`, created (all empty) when `create`, else null if absent
    uint32_t* block(const ChunkKey& s, bool create) {
        const size_t ci = cache_slot(s);
        if (cache_blk_[ci] >= 0 && cache_key_[ci] == s) return &slots_[(size_t)cache_blk_[ci] * 512];
        if (!create && miss_valid_ && miss_key_ == s) return nullptr;   // absent, as found last time
        long long bi = -1;
        if (!keys_.empty()) {
            for (size_t i = hash(s) & mask_;; i = (i + 1) & mask_) {
                if (!used_[i]) break;
                if (keys_[i] == s) {
                    bi = vals_[i];
                    break;
                }
            }
        }
        if (bi < 0) {
            if (!create) {
                miss_key_ = s;
                miss_valid_ = true;
                return nullptr;
            }
            if (miss_valid_ && miss_key_ == s) miss_valid_ = false;
            bi = (long long)(slots_.size() / 512);
            slots_.resize(slots_.size() + 512, kNone);
            if (2 * (nblocks_ + 1) > keys_.size()) grow();
            put(s, (uint32_t)bi);
            ++nblocks_;
        }
        cache_blk_[ci] = bi;
        cache_key_[ci] = s;
        return &slots_[(size_t)bi * 512];
    }
    // direct-mapped cache of found blocks, indexed by a cheap mix of the key
    static size_t cache_slot(const ChunkKey& k) {
        return (size_t)(((unsigned long long)k.x * 0x9E3779B1ull + (unsigned long long)k.y * 0x85EBCA77ull +
                         (unsigned long long)k.z * 0xC2B2AE3Dull) >> 7) & (kCache - 1);
    }
    static size_t hash(const ChunkKey& k) {
        unsigned long long h = (unsigned long long)k.x * 0x9E3779B97F4A7C15ull;
        h ^= (unsigned long long)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
        h ^= (unsigned long long)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
        return (size_t)(h ^ (h >> 29));
    }
    void put(const ChunkKey& k, uint32_t v) {
        size_t i = hash(k) & mask_;
        while (used_[i]) i = (i + 1) & mask_;
        keys_[i] = k;
        vals_[i] = v;
        used_[i] = 1;
    }
    void grow() {
        std::vector<ChunkKey> ok;
        std::vector<uint32_t> ov;
        std::vector<unsigned char> ou;
        ok.swap(keys_);
        ov.swap(vals_);
        ou.swap(used_);
        const size_t n = ok.empty() ? 4096 : 2 * ok.size();
        keys_.assign(n, ChunkKey{0, 0, 0});
        vals_.assign(n, 0u);
        used_.assign(n, 0);
        mask_ = n - 1;
        for (size_t i = 0; i < ok.size(); ++i)
            if (ou[i]) put(ok[i], ov[i]);
    }
    std::vector<ChunkKey> keys_;          // super-chunk keys
    std::vector<uint32_t> vals_;          // their block numbers
    std::vector<unsigned char> used_;
    std::vector<uint32_t> slots_;         // 512 slots per block
    size_t mask_ = 0, count_ = 0, nblocks_ = 0;
    static constexpr size_t kCache = 256;
    long long cache_blk_[kCache] = {};    // blocks found recently (-1: none), and their keys
    ChunkKey cache_key_[kCache] = {};
    ChunkKey miss_key_ = {};              // the last super-chunk looked up and found absent
    bool miss_valid_ = false;
};

}  // namespace tsdf
