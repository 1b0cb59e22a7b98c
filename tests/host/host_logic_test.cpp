// Host-only checks of host_alloc.h (the context arena and the server's
// admission queue): built with the system C++ compiler by
// tests/test_host_logic.py; exits non-zero with a message on the first
// failed check.  No GPU and no CUDA headers are involved.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "host_alloc.h"

using gmls::host::AdmissionQueue;
using gmls::host::FirstFit;

static int fails = 0;
#define CHECK(c)                                                     \
  do {                                                               \
    if (!(c)) {                                                      \
      std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
      ++fails;                                                       \
    }                                                                \
  } while (0)

static void test_first_fit() {
  std::vector<char> buf(1 << 20);
  FirstFit a;
  a.init(buf.data() + 3, buf.size() - 3);  // unaligned base: rounded up to 256 bytes
  CHECK(reinterpret_cast<uintptr_t>(a.alloc(1)) % 256 == 0);
  a.init(buf.data(), buf.size());
  const size_t cap = a.cap();
  void* p = a.alloc(1000);  // rounds to 1024
  void* q = a.alloc(256);
  void* r = a.alloc(0);  // one granule
  CHECK(p && q && r);
  CHECK(a.used() == 1024 + 256 + 256);
  CHECK(static_cast<char*>(q) - static_cast<char*>(p) == 1024);
  a.release(q);
  CHECK(a.used() == 1024 + 256);
  void* q2 = a.alloc(200);  // first fit reuses the hole
  CHECK(q2 == q);
  a.release(p);
  a.release(q2);
  a.release(r);
  a.release(nullptr);  // no-op
  a.release(buf.data() + 5);  // not handed out: no-op
  CHECK(a.used() == 0 && a.live_blocks() == 0);
  CHECK(a.free_blocks() == 1);  // neighbours merged back into one block
  CHECK(a.alloc(cap) != nullptr);  // the whole buffer is one block again
  CHECK(a.alloc(256) == nullptr);  // full
  CHECK(a.peak() == cap);
}

static void test_fault_injection() {
  std::vector<char> buf(1 << 16);
  FirstFit a;
  a.init(buf.data(), buf.size());
  a.fail_after(3);
  void* x1 = a.alloc(256);
  void* x2 = a.alloc(256);
  void* x3 = a.alloc(256);  // the third allocation fails as if full
  void* x4 = a.alloc(256);  // disarmed after firing
  CHECK(x1 && x2 && !x3 && x4);
  // a caller that unwinds on the failure leaves nothing behind
  a.release(x1);
  a.release(x2);
  a.release(x4);
  CHECK(a.used() == 0 && a.live_blocks() == 0 && a.free_blocks() == 1);
  a.fail_after(1);
  CHECK(a.alloc(256) == nullptr);
  a.fail_after(0);  // disarmed
  CHECK(a.alloc(256) != nullptr);
  // every position of a multi-allocation call: fail the n-th, unwind, no leak
  for (int n = 1; n <= 6; ++n) {
    a.init(buf.data(), buf.size());
    a.fail_after(n);
    std::vector<void*> got;
    bool oom = false;
    for (int i = 0; i < 5; ++i) {
      void* p = a.alloc(512);
      if (!p) {
        oom = true;
        break;
      }
      got.push_back(p);
    }
    CHECK(oom == (n <= 5));
    for (void* p : got) a.release(p);
    CHECK(a.used() == 0 && a.free_blocks() == 1);
  }
}

static void test_admission_queue() {
  // a server arena of 10 units: requests of 4, 8, 2, 20 and 3 units;
  // admission of the first that fit (look-ahead 8), rejection of one that never can
  std::vector<char> buf(10 * 256);
  FirstFit mem;
  mem.init(buf.data(), buf.size());
  const size_t need[] = {0, 4, 8, 2, 20, 3};
  AdmissionQueue q;
  for (int t = 1; t <= 5; ++t) q.push(t);
  std::vector<int> admitted, rejected;
  std::vector<void*> slice(6, nullptr);
  auto try_admit = [&](int64_t t) -> int {
    if (need[t] * 256 > buf.size()) {
      rejected.push_back((int)t);
      return 2;
    }
    void* p = mem.alloc(need[t] * 256);
    if (!p) return 0;
    slice[t] = p;
    admitted.push_back((int)t);
    return 1;
  };
  CHECK(q.admit(8, try_admit) == 4);  // 1 (4 units), 3 (2 units) and 5 (3 units) fit; 4 rejected; 2 waits
  CHECK((admitted == std::vector<int>{1, 3, 5}));
  CHECK((rejected == std::vector<int>{4}));
  CHECK(q.size() == 1);
  CHECK(q.admit(8, try_admit) == 0);  // 2 still waits for memory
  mem.release(slice[1]);
  mem.release(slice[5]);
  CHECK(q.admit(8, try_admit) == 0);  // 7 units free but in two holes of 4: still waits
  mem.release(slice[3]);
  CHECK(q.admit(8, try_admit) == 1 && admitted.back() == 2);  // holes merged: admitted
  CHECK(q.empty());
  // cancellation: only while waiting
  q.push(7);
  q.push(8);
  CHECK(q.cancel(7));
  CHECK(!q.cancel(7));  // already gone
  CHECK(q.size() == 1);
  // a full slot table stops the walk (-1) without removing anything
  CHECK(q.admit(8, [](int64_t) { return -1; }) == 0 && q.size() == 1);
  // look-ahead bound: only the first `look` tickets are examined
  for (int t = 10; t < 20; ++t) q.push(t);
  int seen = 0;
  q.admit(3, [&](int64_t) {
    ++seen;
    return 0;
  });
  CHECK(seen == 3);
}

int main() {
  test_first_fit();
  test_fault_injection();
  test_admission_queue();
  if (fails) return 1;
  std::printf("host logic ok\n");
  return 0;
}
