// serve.cu -- continuous-batching stencil server (host runtime over libgmls).
//
// Requests (a point cloud and what to compute on it) arrive at any time from
// client threads.  A scheduler thread admits them as in-flight slots and arena
// memory become free -- requests that arrive while others run on the GPU are
// admitted at once if they fit -- and issues each admitted request's pipeline
// (cloud upload and cell list, neighbour lists, stencils) on one of several
// CUDA streams, so the work of concurrent requests overlaps on the device.
// Completion is detected with events; results stay resident on the device
// until the client copies them out and releases the request.
//
// Each request gets its own gmls context over a slice of the server's arena
// (first-fit, sized from an estimate of the request's memory), so a request's
// result depends only on its own inputs: it is bit-for-bit the same whether it
// ran alone or among others (the kernel variant for a shape is fixed: server
// contexts do not autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gmls.h"
#include "basis_tables.cuh"
#include "host_alloc.h"

namespace gmls {
void set_global_error(const std::string& msg);
int device_sm_count();
bool dfx_path_available(int dim, int deg, int kmax, int L);
size_t dfx_scratch_bytes(int dim, int deg, int64_t n_tgt, int sms);
}

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { PENDING = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

struct Request {
  int64_t ticket = 0;
  gmls_request req;
  std::vector<double> xyz;  // copy of the caller's coordinates
  Clock::time_point arrival, done_at;
  ReqState state = PENDING;
  gmls_status error = GMLS_OK;
  std::string message;
  char* slice = nullptr;
  size_t slice_bytes = 0;
  gmls_ctx* ctx = nullptr;
  int stream = -1;
  cudaEvent_t done_ev = nullptr;
  int64_t cloud = 0, nbrs = 0, stencil = 0;
};

// bytes a request may need inside its own context (estimate with margin)
size_t estimate_bytes(const gmls_request& r) {
  const int64_t n = r.n, k = r.k, d = r.dim;
  const int nc = r.basis == GMLS_BASIS_SCALAR ? 1 : (int)d;
  size_t cloud = (size_t)n * (d * (8 + 8 + 4) + 4 + 4 + 2 * 4 * 3) + 64 * 1024;
  size_t nbrs = (size_t)n * (k * 4 * 2 + 8 + 8 + 4 + 1 + 16) + 64 * 1024;
  size_t weights = 0;
  for (int f = 0; f < r.n_functionals; ++f) {
    const int fn = r.functionals[f];
    const int rows = (fn == GMLS_F_LAPLACIAN || fn == GMLS_F_DIV) ? 1 : (int)d;
    const int comp = (fn == GMLS_F_GRAD || fn == GMLS_F_LAPLACIAN) ? 1 : (int)d;
    weights += (size_t)n * k * rows * comp * 8;
  }
  size_t stencils = weights + (size_t)n * (4 * 8 + 2 + 4 + 16);
  // global tiles of shapes too big for shared memory: at most (SMs x 4) groups
  const int nb = gmls_gen::basis_size(r.basis, (int)d, r.degree);
  const size_t rows = (size_t)k * nc;
  size_t tiles = 0;
  if ((size_t)nb * rows * 12 > 100 * 1024) tiles = (size_t)gmls::device_sm_count() * 4 * ((size_t)nb * rows * 12 + 4096);
  // per-warp slots of the factored divergence-free kernel (during its launch)
  if (r.basis == GMLS_BASIS_DIVFREE && gmls::dfx_path_available((int)d, r.degree, (int)k, (int)d))
    tiles += gmls::dfx_scratch_bytes((int)d, r.degree, n, gmls::device_sm_count()) + 4096;
  const size_t total = cloud + nbrs + stencils + tiles;
  return total + total / 8 + (16u << 20);
}

}  // namespace

struct gmls_server {
  int device = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  gmls::host::FirstFit slices;  // first-fit slices of the server arena
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_load;
  int max_inflight = 8;
  std::mutex mu;
  std::condition_variable cv;
  gmls::host::AdmissionQueue pending;
  std::map<int64_t, Request> reqs;
  int64_t next_ticket = 1;
  int inflight = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> lat_ms;
  int64_t targets_done = 0;
  Clock::time_point first_arrival, last_done;
  bool have_first = false;
  std::string err;
};

static void issue(gmls_server* s, Request& r) {
  // runs on the scheduler thread with s->mu held
  const gmls_request& q = r.req;
  gmls_status rc = gmls_create(&r.ctx, s->device, s->streams[r.stream], r.slice, r.slice_bytes);
  if (rc == GMLS_OK) rc = gmls_set_option(r.ctx, GMLS_OPT_AUTOTUNE, 0);
  if (rc == GMLS_OK) rc = gmls_cloud(r.ctx, q.dim, q.n, r.xyz.data(), nullptr, nullptr, &r.cloud);
  if (rc == GMLS_OK) {
    gmls_nbr_params np;
    std::memset(&np, 0, sizeof(np));
    np.mode = GMLS_NBR_KNN;
    np.k = q.k;
    np.eps_factor = q.eps_factor;
    np.cap = q.k;
    rc = gmls_neighbors(r.ctx, r.cloud, &np, &r.nbrs);
  }
  if (rc == GMLS_OK) {
    gmls_stencil_params sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.basis = q.basis;
    sp.degree = q.degree;
    sp.weight = GMLS_WEIGHT_POLY;
    sp.weight_power = 4;
    sp.precision = q.precision;
    sp.n_functionals = q.n_functionals;
    for (int f = 0; f < q.n_functionals; ++f) sp.functionals[f] = q.functionals[f];
    rc = gmls_stencils(r.ctx, r.nbrs, &sp, &r.stencil);
  }
  if (rc == GMLS_OK && cudaEventRecord(r.done_ev, s->streams[r.stream]) != cudaSuccess) rc = GMLS_ECUDA;
  if (rc != GMLS_OK) {
    r.state = FAILED;
    r.error = rc;
    r.message = r.ctx ? gmls_last_error(r.ctx) : gmls_last_error(nullptr);
    r.done_at = Clock::now();
    return;
  }
  r.state = RUNNING;
}

static void finish(gmls_server* s, Request& r, ReqState st) {
  r.state = st;
  r.done_at = Clock::now();
  s->inflight--;
  s->stream_load[r.stream]--;
  if (st == DONE) {
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.done_at - r.arrival).count());
    s->targets_done += r.req.n;
    s->last_done = r.done_at;
  }
}

static void scheduler(gmls_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    bool progress = false;
    // completions
    for (auto& kv : s->reqs) {
      Request& r = kv.second;
      if (r.state != RUNNING) continue;
      cudaError_t e = cudaEventQuery(r.done_ev);
      if (e == cudaSuccess) {
        finish(s, r, DONE);
        progress = true;
      } else if (e != cudaErrorNotReady) {
        r.error = GMLS_ECUDA;
        r.message = cudaGetErrorString(e);
        finish(s, r, FAILED);
        progress = true;
      }
    }
    // admissions: first pending requests that fit (a look-ahead of 8 lets
    // small requests pass one that waits for memory)
    const int admitted = s->pending.admit(8, [&](int64_t t) -> int {
      if (s->inflight >= s->max_inflight) return -1;
      Request& r = s->reqs.at(t);
      r.slice_bytes = estimate_bytes(r.req);
      r.slice = static_cast<char*>(s->slices.alloc(r.slice_bytes));
      if (!r.slice) {
        if (r.slice_bytes > s->arena_bytes) {  // can never fit
          r.state = FAILED;
          r.error = GMLS_ENOMEM;
          r.message = "request needs more memory than the server arena";
          r.done_at = Clock::now();
          return 2;
        }
        return 0;
      }
      int best = 0;
      for (int i = 1; i < (int)s->streams.size(); ++i)
        if (s->stream_load[i] < s->stream_load[best]) best = i;
      r.stream = best;
      s->stream_load[best]++;
      s->inflight++;
      issue(s, r);
      if (r.state == FAILED) {
        s->inflight--;
        s->stream_load[best]--;
      }
      return 1;
    });
    progress |= admitted > 0;
    if (!progress) s->cv.wait_for(lock, std::chrono::microseconds(50));
  }
}

extern "C" {

gmls_status gmls_server_create(gmls_server** out, int device, void* arena, size_t arena_bytes, int32_t n_streams,
                               int32_t max_inflight) {
  if (!out || !arena || arena_bytes < (64u << 20) || n_streams < 1 || n_streams > 16 || max_inflight < 1) {
    gmls::set_global_error("gmls_server_create: need out, arena >= 64 MiB, 1..16 streams, max_inflight >= 1");
    return GMLS_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    gmls::set_global_error("gmls_server_create: no such device");
    cudaGetLastError();
    return GMLS_ECUDA;
  }
  gmls_server* s = new gmls_server();
  s->device = device;
  uintptr_t b = reinterpret_cast<uintptr_t>(arena), a = (b + 255) & ~uintptr_t(255);
  s->arena = reinterpret_cast<char*>(a);
  s->arena_bytes = (arena_bytes - (a - b)) & ~size_t(255);
  s->slices.init(s->arena, s->arena_bytes);
  s->max_inflight = max_inflight;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      gmls::set_global_error("gmls_server_create: cannot create streams");
      return GMLS_ECUDA;
    }
    s->streams.push_back(st);
    s->stream_load.push_back(0);
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return GMLS_OK;
}

gmls_status gmls_server_submit(gmls_server* s, const gmls_request* q, int64_t* ticket) {
  if (!s || !q || !ticket || !q->xyz || (q->dim != 2 && q->dim != 3) || q->n < 1 || q->k < 1 || q->k > q->n ||
      q->n_functionals < 1 || q->n_functionals > 5 || gmls_gen::basis_size(q->basis, q->dim, q->degree) <= 0)
    return GMLS_EINVAL;
  Request r;
  r.req = *q;
  r.xyz.assign(q->xyz, q->xyz + (size_t)q->dim * q->n);
  r.req.xyz = nullptr;
  r.arrival = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming) != cudaSuccess) return GMLS_ECUDA;
    r.ticket = s->next_ticket++;
    if (!s->have_first) {
      s->first_arrival = r.arrival;
      s->have_first = true;
    }
    *ticket = r.ticket;
    s->pending.push(r.ticket);
    s->reqs.emplace(r.ticket, std::move(r));
  }
  s->cv.notify_one();
  return GMLS_OK;
}

gmls_status gmls_server_wait(gmls_server* s, int64_t ticket, int32_t timeout_ms, int32_t* done) {
  if (!s || !done) return GMLS_EINVAL;
  const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  for (;;) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      auto it = s->reqs.find(ticket);
      if (it == s->reqs.end()) return GMLS_ENOTFOUND;
      const ReqState st = it->second.state;
      if (st == DONE || st == FAILED || st == CANCELLED) {
        *done = 1;
        return st == DONE ? GMLS_OK : st == CANCELLED ? GMLS_ECANCELED : it->second.error;
      }
    }
    if (Clock::now() >= until) {
      *done = 0;
      return GMLS_OK;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

gmls_status gmls_server_result(gmls_server* s, int64_t ticket, int32_t what, int32_t functional, void* dst,
                               size_t bytes, size_t* needed) {
  if (!s) return GMLS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GMLS_ENOTFOUND;
  Request& r = it->second;
  if (r.state != DONE) return r.state == FAILED ? r.error : r.state == CANCELLED ? GMLS_ECANCELED : GMLS_EBUSY;
  const int64_t id = (what == GMLS_X_NBR_INDEX || what == GMLS_X_NBR_EPS || what == GMLS_X_NBR_OFFSETS ||
                      what == GMLS_X_NBR_STATUS)
                         ? r.nbrs
                         : r.stencil;
  size_t need = 0;
  gmls_status rc = gmls_export_size(r.ctx, id, what, functional, &need);
  if (rc != GMLS_OK) return rc;
  if (needed) *needed = need;
  if (!dst) return GMLS_OK;
  return gmls_export(r.ctx, id, what, functional, dst, bytes);
}

gmls_status gmls_server_cancel(gmls_server* s, int64_t ticket) {
  if (!s) return GMLS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GMLS_ENOTFOUND;
    Request& r = it->second;
    if (r.state != PENDING || !s->pending.cancel(ticket)) return GMLS_EBUSY;  // admitted or finished
    r.state = CANCELLED;
    r.error = GMLS_ECANCELED;
    r.done_at = Clock::now();
  }
  s->cv.notify_one();
  return GMLS_OK;
}

gmls_status gmls_server_release(gmls_server* s, int64_t ticket) {
  if (!s) return GMLS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GMLS_ENOTFOUND;
  Request& r = it->second;
  if (r.state == PENDING || r.state == RUNNING) return GMLS_EBUSY;
  if (r.ctx) gmls_destroy(r.ctx);
  if (r.slice) s->slices.release(r.slice);
  if (r.done_ev) cudaEventDestroy(r.done_ev);
  s->reqs.erase(it);
  s->cv.notify_one();
  return GMLS_OK;
}

gmls_status gmls_server_stats(gmls_server* s, gmls_serve_stats* out) {
  if (!s || !out) return GMLS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  std::vector<double> l = s->lat_ms;
  std::sort(l.begin(), l.end());
  out->completed = (int64_t)l.size();
  out->targets = s->targets_done;
  out->pending = (int64_t)s->pending.size();
  out->inflight = s->inflight;
  if (!l.empty()) {
    auto pct = [&](double p) {
      const double pos = p * (l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    out->p50_ms = pct(0.5);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = sum / l.size();
    out->elapsed_s = std::chrono::duration<double>(s->last_done - s->first_arrival).count();
    out->targets_per_s = out->elapsed_s > 0 ? s->targets_done / out->elapsed_s : 0.0;
  }
  return GMLS_OK;
}

gmls_status gmls_server_destroy(gmls_server* s) {
  if (!s) return GMLS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_one();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (auto& kv : s->reqs) {
    if (kv.second.ctx) gmls_destroy(kv.second.ctx);
    if (kv.second.done_ev) cudaEventDestroy(kv.second.done_ev);
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return GMLS_OK;
}

}  // extern "C"
