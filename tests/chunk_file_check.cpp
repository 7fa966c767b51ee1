// Host check of the global store's file tier (csrc/chunk_store.h with
// csrc/chunk_file.h): a window of chunks walks back and forth over a line of
// chunk keys, some of which hold data, with a small device tier and a host
// tier kept to `kHostCap` chunks at the start of every shift, the rest going
// to a real file through the asynchronous writer. The steps follow the
// library's shift: record the last shift's claims, move host chunks beyond
// the limit to the file, make device room (oldest device chunks to the host
// tier), reserve host slots for the candidates and for entering file-tier
// chunks, hand out candidates, take the entering chunks (file-tier ones read
// into host slots), free their slots, and let a stand-in for the kernel write
// every leaving chunk that holds data into a candidate slot. Each chunk's
// content changes every time it leaves the window, so a stale copy is caught.
// Checked: every re-entering chunk reads back its last content, the host tier
// holds at most kHostCap chunks after each trim, every stored chunk is stored
// once, and at the end every file-tier chunk reads back from the file after
// the writer has drained. Last, a write that fails (the process's file size
// limit lowered to 8 KiB) must make flush, put and get report the failure.
// Prints "ok". Usage: chunk_file_check <scratch path> <second scratch path>.
#include <algorithm>
#include <csignal>
#include <cstdio>
#include <cstring>
#include <map>
#include <random>
#include <set>
#include <vector>

#include <sys/resource.h>

#include "chunk_file.h"
#include "chunk_store.h"

using tsdf::ChunkFile;
using tsdf::ChunkKey;
using tsdf::ChunkStore;

namespace {

constexpr size_t kB = ChunkFile::kBytes;

void pattern(long long x, long long v, char* out) {
    uint64_t w[kB / 8];
    for (size_t i = 0; i < kB / 8; ++i) w[i] = ((uint64_t)x * 1000003ull + (uint64_t)v) ^ (i * 0x9E3779B97F4A7C15ull);
    std::memcpy(out, w, kB);
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    std::mt19937_64 rng(4242);
    const long long W = 24;                       // window: chunks [o, o + W) along x
    const uint32_t kDev = 32, kHostCap = 20, kHostSeg = 16, kFileSeg = 64;
    ChunkStore st;
    ChunkFile file;
    if (!file.open(argv[1], 8)) {                 // a short queue: put() also waits for the writer
        std::printf("open failed\n");
        return 1;
    }
    {
        // a path that exists is refused and left in place
        ChunkFile other;
        if (other.open(argv[1], 8) || other.is_open()) {
            std::printf("an existing path was opened\n");
            return 1;
        }
    }
    if (::access(argv[1], F_OK) != 0) {
        std::printf("the refused open removed the file\n");
        return 1;
    }
    // reads right after writes (mostly served from the queue) and rewrites of
    // one slot: each read returns the slot's latest content
    {
        char in[kB], out[kB];
        for (int i = 0; i < 2000; ++i) {
            const uint32_t slot = (uint32_t)(rng() % 16);
            pattern(-1 - (long long)slot, i, in);
            if (!file.put(slot, in) || !file.get(slot, out) || std::memcmp(in, out, kB) != 0) {
                std::printf("read after write, slot %u\n", slot);
                return 1;
            }
        }
    }
    st.add_slots(0, 0, kDev);
    std::vector<char> mem[2];
    mem[0].assign(kDev * kB, 0);
    auto grow_host = [&]() {
        const uint32_t first = (uint32_t)st.capacity(1);
        st.add_slots(1, first, kHostSeg);
        mem[1].resize((first + kHostSeg) * kB, 0);
    };
    auto at = [&](uint32_t loc) -> char* { return &mem[ChunkStore::tier_of(loc)][ChunkStore::slot_of(loc) * kB]; };
    std::map<long long, bool> data;               // chunk x -> holds data (fixed per chunk)
    std::map<long long, long long> ver;           // chunk x -> content version when it last left
    auto has = [&](long long x) {
        auto it = data.find(x);
        if (it == data.end()) it = data.emplace(x, (rng() % 3) != 0).first;
        return it->second;
    };
    std::vector<int32_t> claim;
    std::set<long long> seen;
    for (long long x = 0; x < W; ++x) seen.insert(x);
    long long o = 0;
    uint64_t serial = 0;
    size_t to_file = 0, from_file = 0;
    char buf[kB], want[kB];
    for (int step = 0; step < 3000; ++step) {
        const long long d = (long long)(rng() % 13) - 6;   // shift by -6 .. +6 chunks
        const long long no = o + d;
        if (step > 0) st.commit(claim.data());
        // host chunks beyond the limit go to the file, oldest first
        while (st.used(1) > kHostCap) {
            if (st.free_count(2) == 0) st.add_slots(2, (uint32_t)st.capacity(2), kFileSeg);
            uint32_t from, to;
            if (!st.spill_oldest_host(&from, &to)) { std::printf("host spill failed\n"); return 1; }
            if (ChunkStore::tier_of(from) != 1 || ChunkStore::tier_of(to) != 2) { std::printf("tiers\n"); return 1; }
            if (!file.put(ChunkStore::slot_of(to), at(from))) { std::printf("put failed\n"); return 1; }
            std::memset(at(from), 0x5A, kB);     // the host slot is free now: poison it
            ++to_file;
        }
        if (st.used(1) > kHostCap) { std::printf("host tier over its limit\n"); return 1; }
        std::vector<long long> leave, enter;
        for (long long x = o; x < o + W; ++x)
            if (x < no || x >= no + W) leave.push_back(x);
        for (long long x = no; x < no + W; ++x)
            if (x < o || x >= o + W) enter.push_back(x);
        // device room: the oldest device chunks move to the host tier
        while (st.free_count(0) < leave.size()) {
            if (st.free_count(1) == 0) grow_host();
            uint32_t from, to;
            if (!st.spill_oldest(&from, &to)) break;
            std::memcpy(at(to), at(from), kB);
            std::memset(at(from), 0x33, kB);
        }
        // host slots for the candidates beyond the device tier and for the
        // entering file-tier chunks
        size_t nfile = 0;
        for (long long x : enter) {
            const long long loc = st.find(ChunkKey{x, 0, 0});
            nfile += (loc >= 0 && ChunkStore::is_file((uint32_t)loc)) ? 1 : 0;
        }
        const size_t host_need = (leave.size() > st.free_count(0) ? leave.size() - st.free_count(0) : 0) + nfile;
        while (st.free_count(1) < host_need) grow_host();
        ++serial;
        std::vector<ChunkKey> keys;
        for (long long x : leave) keys.push_back(ChunkKey{x, 0, 0});
        std::vector<uint32_t> locs;
        if (!st.candidates(keys, serial, &locs)) { std::printf("no slots\n"); return 1; }
        std::set<uint32_t> cand(locs.begin(), locs.end());
        for (long long x : enter) {
            long long loc = st.take(ChunkKey{x, 0, 0});
            const bool stored = loc >= 0;
            if (stored != (has(x) && seen.count(x) > 0)) {
                std::printf("chunk %lld: stored %d, holds data %d\n", x, (int)stored, (int)has(x));
                return 1;
            }
            if (stored && ChunkStore::is_file((uint32_t)loc)) {
                const long long h = st.take_slot(1);
                if (h < 0 || cand.count((uint32_t)h)) { std::printf("page-in slot\n"); return 1; }
                if (!file.get(ChunkStore::slot_of((uint32_t)loc), at((uint32_t)h))) { std::printf("get failed\n"); return 1; }
                loc = h;
                ++from_file;
            }
            if (stored) {
                pattern(x, ver[x], want);
                if (std::memcmp(at((uint32_t)loc), want, kB) != 0) {
                    std::printf("chunk %lld (tier %d) read back wrong content\n", x, ChunkStore::tier_of((uint32_t)loc));
                    return 1;
                }
            }
            seen.insert(x);
        }
        st.end_shift();
        // the kernel: leaving chunks with data claim candidates in some order,
        // each with new content
        std::vector<size_t> order;
        for (size_t i = 0; i < leave.size(); ++i)
            if (has(leave[i])) order.push_back(i);
        std::shuffle(order.begin(), order.end(), rng);
        claim.assign(leave.size(), -1);
        for (size_t c = 0; c < order.size(); ++c) {
            const long long x = leave[order[c]];
            claim[order[c]] = (int32_t)c;
            ver[x] = (long long)step * 7 + 1;
            pattern(x, ver[x], at(locs[c]));
        }
        o = no;
        // every stored chunk once, none inside the window
        ChunkStore copy = st;
        copy.commit(claim.data());
        std::set<uint32_t> used;
        size_t n = 0;
        bool ok = true;
        copy.for_each([&](const ChunkKey& k, uint32_t loc) {
            ++n;
            if (!used.insert(loc).second) ok = false;
            if (k.x >= o && k.x < o + W) ok = false;
            if (!has(k.x)) ok = false;
        });
        size_t nwant = 0;
        for (auto& kv : data)
            nwant += (kv.second && seen.count(kv.first) && (kv.first < o || kv.first >= o + W)) ? 1 : 0;
        if (!ok || n != nwant || copy.used(0) + copy.used(1) + copy.used(2) != n || copy.used(0) > kDev) {
            std::printf("step %d: ok=%d stored=%zu want=%zu\n", step, (int)ok, n, nwant);
            return 1;
        }
    }
    // the file tier after the writer drains: every chunk reads its content
    st.commit(claim.data());
    if (!file.flush()) { std::printf("flush failed\n"); return 1; }
    size_t checked = 0;
    bool ok = true;
    st.for_each([&](const ChunkKey& k, uint32_t loc) {
        if (!ChunkStore::is_file(loc)) return;
        pattern(k.x, ver[k.x], want);
        if (!file.get(ChunkStore::slot_of(loc), buf) || std::memcmp(buf, want, kB) != 0) ok = false;
        ++checked;
    });
    if (!ok || checked == 0 || to_file == 0 || from_file == 0) {
        std::printf("final: ok=%d checked=%zu to_file=%zu from_file=%zu\n", (int)ok, checked, to_file, from_file);
        return 1;
    }
    file.close();
    // a failing write (beyond the file size limit: EFBIG instead of SIGXFSZ)
    std::signal(SIGXFSZ, SIG_IGN);
    struct rlimit lim = {8192, 8192};
    if (::setrlimit(RLIMIT_FSIZE, &lim) != 0) { std::printf("setrlimit failed\n"); return 1; }
    {
        ChunkFile bad;
        if (!bad.open(argv[2], 8)) { std::printf("open of the second path failed\n"); return 1; }
        pattern(1, 1, want);
        if (!bad.put(0, want) || !bad.flush()) { std::printf("a write within the limit failed\n"); return 1; }
        if (!bad.get(0, buf) || std::memcmp(buf, want, kB) != 0) { std::printf("read back within the limit\n"); return 1; }
        bad.put(9, want);   // offset 18 KiB: over the limit
        if (bad.flush() || !bad.failed()) { std::printf("a failed write was not reported\n"); return 1; }
        if (bad.put(1, want) || bad.get(0, buf)) { std::printf("calls after a failed write succeeded\n"); return 1; }
    }
    if (::access(argv[2], F_OK) == 0) { std::printf("the second file was not removed\n"); return 1; }
    std::printf("ok %zu to file, %zu read back, %zu in the file at the end, %llu from the queue; failed write "
                "reported\n", to_file, from_file, checked, (unsigned long long)file.pending_hits());
    return 0;
}
