// host_alloc.h -- host-side logic shared by the context and the server:
// the first-fit sub-allocator over a caller's device buffer and the server's
// admission queue.  Plain C++ (no CUDA): it hands out offsets and never
// touches the memory, so it is tested on the CPU.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <deque>
#include <map>

namespace gmls {
namespace host {

// First-fit allocator over [base, base + cap).  256-byte granularity;
// neighbouring free blocks merge on release.  fail_after(n) arms a fault
// injector: the n-th allocation from now fails as if the buffer were full
// (n = 0 disarms), so that every out-of-memory path can be exercised.
class FirstFit {
 public:
  void init(void* base, size_t bytes) {
    const uintptr_t b = reinterpret_cast<uintptr_t>(base);
    const uintptr_t a = (b + 255) & ~uintptr_t(255);
    base_ = reinterpret_cast<char*>(a);
    cap_ = (bytes > (a - b)) ? ((bytes - (a - b)) & ~size_t(255)) : 0;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
    used_ = peak_ = 0;
    fail_in_ = 0;
  }
  void fail_after(int64_t n) { fail_in_ = n > 0 ? n : 0; }
  void* alloc(size_t bytes) {
    if (fail_in_ > 0 && --fail_in_ == 0) return nullptr;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        live_[off] = bytes;
        used_ += bytes;
        if (used_ > peak_) peak_ = used_;
        return base_ + off;
      }
    }
    return nullptr;
  }
  // releasing NULL or a pointer this allocator did not hand out does nothing
  void release(void* p) {
    if (!p) return;
    const size_t off = static_cast<char*>(p) - base_;
    auto it = live_.find(off);
    if (it == live_.end()) return;
    size_t sz = it->second;
    live_.erase(it);
    used_ -= sz;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + sz == nx->first) {
      sz += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        pv->second += sz;
        return;
      }
    }
    free_[off] = sz;
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t cap() const { return cap_; }
  size_t live_blocks() const { return live_.size(); }
  size_t free_blocks() const { return free_.size(); }

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  int64_t fail_in_ = 0;
  std::map<size_t, size_t> free_, live_;
};

// Tickets waiting for admission, in arrival order.  admit() walks the first
// `look` of them and asks try_admit(ticket) for each: 0 keep it waiting (not
// enough memory or slots yet), 1 admitted, 2 rejected (it can never fit);
// admitted and rejected tickets leave the queue.  A look-ahead above one lets
// small requests pass one that waits for memory.  cancel() takes a ticket out
// before it is admitted.  The caller serialises access (the server's lock).
class AdmissionQueue {
 public:
  void push(int64_t t) { q_.push_back(t); }
  bool cancel(int64_t t) {
    for (auto it = q_.begin(); it != q_.end(); ++it)
      if (*it == t) {
        q_.erase(it);
        return true;
      }
    return false;
  }
  template <typename F>
  int admit(int look, F&& try_admit) {
    int changed = 0, seen = 0;
    for (auto it = q_.begin(); it != q_.end() && seen < look;) {
      ++seen;
      const int r = try_admit(*it);
      if (r < 0) break;  // stop: no admission possible now (no free slot)
      if (r == 0) {
        ++it;
        continue;
      }
      it = q_.erase(it);
      ++changed;
    }
    return changed;
  }
  size_t size() const { return q_.size(); }
  bool empty() const { return q_.empty(); }

 private:
  std::deque<int64_t> q_;
};

}  // namespace host
}  // namespace gmls
