// File tier of the global chunk store (used by api.cu; plain C++ and POSIX
// with no CUDA dependency, so that it is also checked on the host).
//
// The paper keeps the global map on disk: parts of the map that leave the
// local window are written out while previously mapped parts are read back
// (Introduction; the closing remarks of the Evaluation put the global map on
// an SSD). Here the chunks of the store's third tier live in one scratch file
// as 2 KiB records, the record of file slot s at byte s * 2 KiB.
//
// Writes are asynchronous: put() copies the chunk into a pending buffer and
// returns; a writer thread writes the pending chunks in the order they were
// put (so a slot written twice ends with the later chunk). get() of a slot
// whose write has not finished copies the pending chunk instead of reading
// the file. put() and get() are called from one thread (the map's); the
// writer thread only writes. A failed write or read makes every later call
// fail (failed()). The file is created by open(), which refuses a path that
// already exists (so that no other file is overwritten or later removed), and
// removed when the object is destroyed.
#pragma once

#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <fcntl.h>
#include <sys/types.h>
#include <unistd.h>

namespace tsdf {

class ChunkFile {
public:
    static constexpr size_t kBytes = 2048;

    ChunkFile() = default;
    ChunkFile(const ChunkFile&) = delete;
    ChunkFile& operator=(const ChunkFile&) = delete;
    ~ChunkFile() { close(); }

    // Creates the file (false if it exists or cannot be created) and starts
    // the writer; at most `max_pending` chunks wait to be written (put()
    // blocks beyond that).
    bool open(const char* path, size_t max_pending) {
        if (fd_ >= 0 || max_pending == 0) return false;
        fd_ = ::open(path, O_RDWR | O_CREAT | O_EXCL | O_CLOEXEC, 0600);
        if (fd_ < 0) return false;
        char* full = ::realpath(path, nullptr);   // removed by this name even if the working directory changes
        path_ = full ? full : path;
        std::free(full);
        buf_.resize(max_pending * kBytes);
        free_bufs_.clear();
        for (size_t i = max_pending; i-- > 0;) free_bufs_.push_back((uint32_t)i);
        stop_ = false;
        writer_ = std::thread([this] { write_loop(); });
        return true;
    }

    bool is_open() const { return fd_ >= 0; }

    // Queues `src` (kBytes) as the content of file slot `slot`.
    bool put(uint32_t slot, const void* src) {
        std::unique_lock<std::mutex> lk(mu_);
        room_.wait(lk, [&] { return !free_bufs_.empty() || failed_; });
        if (failed_) return false;
        const uint32_t b = free_bufs_.back();
        free_bufs_.pop_back();
        std::memcpy(&buf_[(size_t)b * kBytes], src, kBytes);
        const uint64_t seq = ++seq_;
        queue_.push_back(Job{slot, b, seq});
        latest_[slot] = Job{slot, b, seq};
        ++writes_;
        work_.notify_one();
        return true;
    }

    // Copies the content of file slot `slot` to `dst` (kBytes).
    bool get(uint32_t slot, void* dst) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (failed_) return false;
            ++reads_;
            auto it = latest_.find(slot);
            if (it != latest_.end()) {   // still waiting to be written
                std::memcpy(dst, &buf_[(size_t)it->second.buf * kBytes], kBytes);
                ++pending_hits_;
                return true;
            }
        }
        // (the slot's last write has finished: only this thread queues writes)
        size_t done = 0;
        while (done < kBytes) {
            const ssize_t r = ::pread(fd_, static_cast<char*>(dst) + done, kBytes - done,
                                      (off_t)((uint64_t)slot * kBytes + done));
            if (r <= 0) {
                std::lock_guard<std::mutex> lk(mu_);
                failed_ = true;
                room_.notify_all();
                return false;
            }
            done += (size_t)r;
        }
        return true;
    }

    // Waits until every queued chunk is written; false if a write failed.
    bool flush() {
        std::unique_lock<std::mutex> lk(mu_);
        idle_.wait(lk, [&] { return (queue_.empty() && !busy_) || failed_; });
        return !failed_;
    }

    bool failed() {
        std::lock_guard<std::mutex> lk(mu_);
        return failed_;
    }
    uint64_t writes() const { return writes_; }
    uint64_t reads() const { return reads_; }
    uint64_t pending_hits() const { return pending_hits_; }

    void close() {
        if (writer_.joinable()) {
            {
                std::lock_guard<std::mutex> lk(mu_);
                stop_ = true;
                work_.notify_all();
            }
            writer_.join();
        }
        if (fd_ >= 0) {
            ::close(fd_);
            ::unlink(path_.c_str());
            fd_ = -1;
        }
    }

private:
    struct Job {
        uint32_t slot;
        uint32_t buf;
        uint64_t seq;
    };

    bool write_one(const Job& j) {
        size_t done = 0;
        const char* src = &buf_[(size_t)j.buf * kBytes];
        while (done < kBytes) {
            const ssize_t r = ::pwrite(fd_, src + done, kBytes - done, (off_t)((uint64_t)j.slot * kBytes + done));
            if (r <= 0) return false;
            done += (size_t)r;
        }
        return true;
    }

    void write_loop() {
        std::vector<Job> batch;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            work_.wait(lk, [&] { return stop_ || !queue_.empty(); });
            if (queue_.empty()) break;   // stop requested and nothing left
            batch.assign(queue_.begin(), queue_.end());
            queue_.clear();
            busy_ = true;
            lk.unlock();
            bool ok = true;
            for (const Job& j : batch) ok = ok && write_one(j);   // in put() order
            lk.lock();
            busy_ = false;
            if (!ok) failed_ = true;
            for (const Job& j : batch) {
                auto it = latest_.find(j.slot);
                if (it != latest_.end() && it->second.seq == j.seq) latest_.erase(it);
                free_bufs_.push_back(j.buf);
            }
            room_.notify_all();
            idle_.notify_all();
        }
        busy_ = false;
        idle_.notify_all();
    }

    int fd_ = -1;
    std::string path_;
    std::vector<char> buf_;                      // pending chunks, kBytes each
    std::vector<uint32_t> free_bufs_;
    std::deque<Job> queue_;                      // not yet taken by the writer
    std::unordered_map<uint32_t, Job> latest_;   // slot -> its newest unfinished write
    uint64_t seq_ = 0;
    bool stop_ = false, busy_ = false, failed_ = false;
    uint64_t writes_ = 0, reads_ = 0, pending_hits_ = 0;
    std::mutex mu_;
    std::condition_variable work_, room_, idle_;
    std::thread writer_;
};

}  // namespace tsdf
