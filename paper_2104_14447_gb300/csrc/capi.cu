// capi.cu -- the C ABI of libgmls (declared in include/gmls.h): context,
// arena allocator, handles, argument checking and launch orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "basis_tables.cuh"
#include "gmls_internal.cuh"
#include "host_alloc.h"

using namespace gmls;

namespace {

// First-fit allocator over the caller's device buffer (host_alloc.h).  Frees
// are stream ordered with the context's single stream, so a block can be
// reused by later work on that stream as soon as it is released.
using Arena = gmls::host::FirstFit;

enum Kind { K_CLOUD = 1, K_NBRS = 2, K_STENCIL = 3, K_GRAPH = 4 };

struct CloudObj {
  int dim = 0;
  int64_t n = 0;
  double* x = nullptr;
  double* normals = nullptr;
  uint8_t* bflag = nullptr;
  double* xs = nullptr;
  float* xsf = nullptr;  // fl32 of xs
  int32_t* sorted = nullptr;
  int32_t* cell_start = nullptr;
  GridParams* grid = nullptr;
  int64_t ncell = 0;
  int refs = 0;
};

struct NbrObj {
  int64_t cloud = 0;
  int dim = 0;
  int64_t n_tgt = 0;
  int32_t* tgt = nullptr;
  int64_t* off = nullptr;
  int32_t* idx = nullptr;
  double* eps = nullptr;
  uint8_t* status = nullptr;
  int mode = 0, k = 0, cap = 0;
  bool variable = false;  // per-target list lengths (offsets from a scan)
  bool all_targets = false;  // targets are every point of the cloud, in order
  int64_t idx_cap = 0;  // allocated index entries
  int16_t* order = nullptr;  // id order of the lists, computed on first use (CSR, Stokes system)
  int64_t parent = 0;        // the longer fixed-k list this one is a prefix of (0: none)
  int refs = 0;
};

struct StencilObj {
  int64_t nbrs = 0;
  int basis = 0, dim = 0, L = 0;
  int nout = 0;
  int fn[5], rows[5], ncomp[5];
  int src[5] = {0, 0, 0, 0, 0};  // first solve row of each functional (its beta column)
  int neumann = 0;
  double* w[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* beta = nullptr;
  uint8_t* status = nullptr;
  uint8_t* iters = nullptr;
  int32_t* fb_items = nullptr;
  int32_t* fb_count = nullptr;
};

struct Obj {
  Kind kind;
  CloudObj c;
  NbrObj nb;
  StencilObj s;
  cudaGraphExec_t exec = nullptr;
};

std::string g_create_error;

}  // namespace

namespace gmls {
// last error of a call made without a context (see gmls_last_error(NULL))
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gmls

struct TuneKey {
  int basis, dim, degree, precision, ld, L, neumann, bucketed;
  bool operator<(const TuneKey& o) const {
    const int a[8] = {basis, dim, degree, precision, ld, L, neumann, bucketed};
    const int b[8] = {o.basis, o.dim, o.degree, o.precision, o.ld, o.L, o.neumann, o.bucketed};
    for (int i = 0; i < 8; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
struct TuneRecord {
  TuneKey key;
  int variant;  // -1 / -2 / -4 register kernel (32 / 16 / 8 lanes per target), -3 factored, else warps per target
  float ms;
};

struct gmls_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Arena arena;
  std::unordered_map<int64_t, Obj> objs;
  int64_t next_id = 1;
  int64_t launches = 0;
  bool force_generic = false;  // testing: use the generic tile kernel for every shape
  int force_variant = 0;       // testing: this kernel variant for uniform shapes (0: off)
  bool poison = false;         // testing: fill stencil outputs with all-ones bytes first
  bool order_key64 = false;    // testing: sort neighbour-list id orders on 64-bit keys
  bool autotune = true;
  std::map<TuneKey, int> tune;        // chosen variant per shape
  std::vector<TuneRecord> tune_log;   // every timing the autotuner took
  std::string err;
  Launch launch() { return Launch{stream, &launches}; }
};

static gmls_status fail(gmls_ctx* c, gmls_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static gmls_status cuda_fail(gmls_ctx* c, cudaError_t e, const char* where) {
  // the launch helpers report an arena sub-allocation that failed as
  // cudaErrorMemoryAllocation (the library itself never calls cudaMalloc)
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, GMLS_ENOMEM, std::string(where) + ": arena exhausted");
  }
  return fail(c, GMLS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                            \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

template <typename T>
static T* arena_alloc(gmls_ctx* ctx, size_t count) {
  return static_cast<T*>(ctx->arena.alloc(count * sizeof(T)));
}

// copy host-or-device src into arena memory dst
static cudaError_t copy_in(gmls_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream);
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}


// ------------------------------------------------------------- launch planning
// Variant code of the shared-memory kernel: warps per target G (1, 2 or 4)
// plus 8 x the tile placement (kPlaceShared / kPlaceSplit / kPlaceGlobal).
static int vcode(int G, int place) { return G + 8 * place; }
static int v_warps(int v) { return v & 7; }
static int v_place(int v) { return v >> 3; }

static bool variant_fits(int v, int ld, int nmax, bool fp32) {
  const int G = v_warps(v), place = v_place(v);
  if (!(G == 1 || G == 2 || G == 4) || place < kPlaceShared || place > kPlaceGlobal) return false;
  if (place == kPlaceSplit && !fp32) return false;  // the FP64 path has no second tile
  return (size_t)(4 / G) * tile_bytes(ld, nmax, fp32, place) <= 227 * 1024;
}

// Heuristic variant for a tile of ld rows: a warp per target up to 64 rows,
// two up to 192, four beyond; more when the tiles would not fit twice in
// shared memory.  Tiles too big for shared memory move their float-float copy
// (FP32 path), else both tiles, to an L2-resident global slot.
static int heuristic_variant(int ld, int nmax, bool fp32) {
  int g = ld <= 64 ? 1 : (ld <= 192 ? 2 : 4);
  while (g < 4 && (size_t)(4 / g) * tile_bytes(ld, nmax, fp32) > 110 * 1024) g *= 2;
  if (variant_fits(vcode(g, kPlaceShared), ld, nmax, fp32)) return vcode(g, kPlaceShared);
  if (variant_fits(vcode(4, kPlaceSplit), ld, nmax, fp32)) return vcode(4, kPlaceSplit);
  return variant_fits(vcode(4, kPlaceGlobal), ld, nmax, fp32) ? vcode(4, kPlaceGlobal) : 0;
}

// Autotuner candidates of the shared-memory kernel: 1, 2 or 4 warps per
// target with the tiles in shared memory, and, where that leaves at most one
// block per SM, the split and global placements too.
static std::vector<int> generic_candidates(int ld, int nmax, bool fp32) {
  std::vector<int> c;
  for (int G = 1; G <= 4; G *= 2) {
    if (variant_fits(vcode(G, kPlaceShared), ld, nmax, fp32)) c.push_back(vcode(G, kPlaceShared));
    if ((size_t)(4 / G) * tile_bytes(ld, nmax, fp32) <= 110 * 1024) continue;
    for (int place : {kPlaceSplit, kPlaceGlobal})
      if (variant_fits(vcode(G, place), ld, nmax, fp32)) c.push_back(vcode(G, place));
  }
  return c;
}

static size_t plan_smem(const BatchPlan& pl, bool fp32) {
  size_t m = 0;
  for (int b = 0; b < (pl.single ? 1 : pl.nb); ++b)
    if (pl.G[b] > 0) m = std::max(m, (size_t)(4 / pl.G[b]) * tile_bytes(pl.ld[b], pl.nmax[b], fp32, pl.gtile[b]));
  return m;
}

// global tile slots for the buckets whose placement needs them:
// [blocks][groups][slot]
static bool plan_gscratch(gmls_ctx* ctx, BatchPlan& pl, bool fp32, int grid, void** owned) {
  size_t slot = 0;
  int groups = 1;
  for (int b = 0; b < (pl.single ? 1 : pl.nb); ++b) {
    if (pl.G[b] <= 0 || pl.gtile[b] == kPlaceShared) continue;
    const size_t gb = global_tile_bytes(pl.ld[b], pl.nmax[b], fp32, pl.gtile[b]);
    if (!gb) continue;
    slot = std::max(slot, gb);
    groups = std::max(groups, 4 / pl.G[b]);
  }
  *owned = nullptr;
  pl.gscratch = nullptr;
  pl.gslot_bytes = 0;
  if (!slot) return true;
  pl.gslot_bytes = (slot + 255) & ~size_t(255);
  *owned = ctx->arena.alloc((size_t)grid * groups * pl.gslot_bytes);
  pl.gscratch = static_cast<unsigned char*>(*owned);
  return *owned != nullptr;
}

static bool capturing(gmls_ctx* ctx) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Holds the stream for a fixed number of SM clock cycles (bounded: it waits
// on nothing), so that the host can queue the launches the autotuner times
// behind it and their events measure GPU time only, not the host's
// launch-preparation time between them.
__global__ void tune_delay_kernel(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}

// time a launch on the context stream (ms), for the autotuner: one warm-up,
// then the faster of two timed runs queued behind a short delay kernel
template <typename F>
static float time_launch(gmls_ctx* ctx, F&& launch) {
  cudaEvent_t ev[3];
  for (auto& e : ev) cudaEventCreate(&e);
  launch();  // warm
  tune_delay_kernel<<<1, 1, 0, ctx->stream>>>(2000000LL);  // about 1 ms at 2 GHz
  cudaEventRecord(ev[0], ctx->stream);
  launch();
  cudaEventRecord(ev[1], ctx->stream);
  launch();
  cudaEventRecord(ev[2], ctx->stream);
  cudaEventSynchronize(ev[2]);
  float ms = 1e30f;
  if (cudaGetLastError() == cudaSuccess) {
    float t0 = 1e30f, t1 = 1e30f;
    cudaEventElapsedTime(&t0, ev[0], ev[1]);
    cudaEventElapsedTime(&t1, ev[1], ev[2]);
    ms = std::min(t0, t1);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return ms;
}

static cudaError_t launch_single(gmls_ctx* ctx, const StencilJob& j, int variant, int ld, int nmax, bool fp32,
                                 int32_t* counter, int sms) {
  BatchPlan pl;
  std::memset(&pl, 0, sizeof(pl));
  pl.single = 1;
  pl.nb = 1;
  pl.G[0] = v_warps(variant);
  pl.ld[0] = ld;
  pl.nmax[0] = nmax;
  pl.task_counter = counter;
  pl.gtile[0] = v_place(variant);
  const size_t smem = plan_smem(pl, fp32);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  const int grid = sms * stencil_blocks_per_sm(fp32, smem);
  void* owned = nullptr;
  if (!plan_gscratch(ctx, pl, fp32, grid, &owned)) return cudaErrorMemoryAllocation;
  Launch L = ctx->launch();
  e = launch_stencils(L, j, pl, fp32, smem, grid);
  ctx->arena.release(owned);  // stream ordered: later work on this stream runs after the kernel
  return e;
}

// Uniform neighbour counts and degree: one shape.  Candidates: the register
// kernel with a warp (variant -1), a half warp (variant -2) or 8 lanes
// (variant -4; not for Neumann rows, which it has no instantiation for) per
// target, when this shape is instantiated, and the shared-memory kernel with 1, 2 or 4
// warps per target and its tile placements (generic_candidates); the
// autotuner times each once on up to 8192 targets and the choice is cached
// per shape.
static gmls_status launch_uniform(gmls_ctx* ctx, const StencilJob& j, const gmls_stencil_params* p, bool refine,
                                  int ld, int nmax, int sms, int32_t* counter) {
  const int dim = j.dim;
  int mr32 = 0, mr16 = 0, mr8 = 0, mr_pref = 0;
  const bool fast_allowed = refine && (p->weight_power % 2 == 0) && !ctx->force_generic;
  const bool ok32 = fast_allowed && fast_path_available(p->basis, dim, p->degree, ld, j.L, 32, &mr32);
  const bool ok16 = fast_allowed && fast_path_available(p->basis, dim, p->degree, ld, j.L, 16, &mr16);
  const bool ok8 = fast_allowed && !p->neumann && fast_path_available(p->basis, dim, p->degree, ld, j.L, 8, &mr8);
  const int hw_pref = fast_allowed ? fast_path_preferred(p->basis, dim, p->degree, ld, j.L, &mr_pref) : 0;
  // factored divergence-free kernel (variant -3): lists of at least Q and at
  // most its capacity of neighbours
  const int kmax = ld / j.nc;
  const bool okdfx = fast_allowed && p->basis == GMLS_BASIS_DIVFREE &&
                     kmax >= gmls_gen::basis_size(GMLS_BASIS_SCALAR, dim, p->degree) &&
                     dfx_path_available(dim, p->degree, kmax, j.L);
  auto launch_fast = [&](const StencilJob& jj, int variant) {
    if (variant == -3) {
      DfxShape sh;
      cudaError_t e = dfx_launch_shape(jj, sms, &sh);
      if (e != cudaSuccess) return e;
      // per-warp slots for the resident grid; on a small arena a smaller grid
      // (the warps loop over the targets, so any grid is correct)
      const size_t per_block = sh.grid > 0 ? sh.scratch / (size_t)sh.grid : sh.scratch;
      void* scr = ctx->arena.alloc(sh.scratch);
      while (!scr && sh.grid > 1) {
        sh.grid = (sh.grid + 1) / 2;
        sh.scratch = per_block * (size_t)sh.grid;
        scr = ctx->arena.alloc(sh.scratch);
      }
      if (!scr) return cudaErrorMemoryAllocation;
      StencilJob jd = jj;
      jd.dscratch = static_cast<unsigned char*>(scr);
      e = launch_stencils_dfx(ctx->launch(), jd, sh);
      ctx->arena.release(scr);  // stream ordered: later work on this stream runs after the kernel
      return e;
    }
    if (variant == -4) return launch_stencils_fast(ctx->launch(), jj, mr8, 8, sms);
    return variant == -2 ? launch_stencils_fast(ctx->launch(), jj, mr16, 16, sms)
                         : launch_stencils_fast(ctx->launch(), jj, mr32, 32, sms);
  };
  const TuneKey key{p->basis, dim, p->degree, p->precision, ld, j.L, p->neumann, 0};
  int choice = 0;  // -1 / -2 / -4 register kernel (32 / 16 / 8 lanes per target), -3 factored div-free, else a vcode
  auto it = ctx->tune.find(key);
  if (ctx->force_variant != 0) {
    const int v = ctx->force_variant;
    const bool ok = (v == -1 && ok32) || (v == -2 && ok16) || (v == -3 && okdfx) || (v == -4 && ok8) ||
                    (v > 0 && variant_fits(v, ld, nmax, refine));
    if (!ok) return fail(ctx, GMLS_EINVAL, "gmls_stencils: the forced kernel variant is not available for this shape");
    choice = v;
  } else if (ctx->force_generic) {
    choice = heuristic_variant(ld, nmax, refine);
  } else if (it != ctx->tune.end()) {
    choice = it->second;
  } else if (ctx->autotune && !capturing(ctx)) {
    // the timed sample: up to 8192 targets in 8 runs of 1024 consecutive
    // ones spread evenly over the list (the first ones may all be of one
    // kind -- e.g. a cube face of boundary targets that the register kernel
    // hands off without work -- and isolated targets would time the kernels
    // without the cache reuse of neighbouring targets)
    StencilJob js = j;
    constexpr int64_t kTuneTargets = 8192;
    int32_t* sample = nullptr;
    if (!j.items && j.n_tgt > kTuneTargets) {
      sample = arena_alloc<int32_t>(ctx, kTuneTargets + 1);
      if (sample) {
        std::vector<int32_t> h(kTuneTargets + 1);
        constexpr int64_t kRuns = 8, kRun = kTuneTargets / kRuns;
        for (int64_t r = 0; r < kRuns; ++r) {
          const int64_t start = r * (j.n_tgt - kRun) / (kRuns - 1);
          for (int64_t i = 0; i < kRun; ++i) h[r * kRun + i] = (int32_t)(start + i);
        }
        h[kTuneTargets] = (int32_t)kTuneTargets;
        CK(cudaMemcpyAsync(sample, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, ctx->stream),
           "gmls_stencils tuning sample");
        js.items = sample;
        js.n_items = sample + kTuneTargets;
      }
    }
    if (!js.items) js.n_tgt = std::min<int64_t>(j.n_tgt, kTuneTargets);
    float best = 1e30f;
    std::vector<int> cands;
    if (ok32) cands.push_back(-1);
    if (ok16) cands.push_back(-2);
    if (ok8) cands.push_back(-4);
    if (okdfx) cands.push_back(-3);
    for (int v : generic_candidates(ld, nmax, refine)) cands.push_back(v);
    for (int c : cands) {
      float ms = time_launch(ctx, [&]() {
        if (refine) cudaMemsetAsync(j.fb_count, 0, 3 * sizeof(int32_t), ctx->stream);
        if (c < 0)
          launch_fast(js, c);
        else
          launch_single(ctx, js, c, ld, nmax, refine, counter, sms);
      });
      ctx->tune_log.push_back({key, c, ms});
      if (ms < best) {
        best = ms;
        choice = c;
      }
    }
    ctx->arena.release(sample);  // the timed launches have finished (time_launch waits for them)
    if (choice == 0) return fail(ctx, GMLS_EINVAL, "gmls_stencils: no kernel variant fits this shape");
    ctx->tune[key] = choice;
  } else {
    choice = okdfx ? -3 : hw_pref == 16 ? -2 : hw_pref == 32 ? -1 : heuristic_variant(ld, nmax, refine);
  }
  if (choice == 0) return fail(ctx, GMLS_EINVAL, "gmls_stencils: tile does not fit in shared memory for this shape");
  if (refine) CK(cudaMemsetAsync(j.fb_count, 0, 3 * sizeof(int32_t), ctx->stream), "gmls_stencils memset");
  if (choice < 0) {
    // Neumann targets: the register kernel's Neumann instantiation for this
    // shape when there is one (a second launch over the list the first one
    // fills), else the shared-memory kernel
    const int mr = choice == -2 ? mr16 : choice == -4 ? mr8 : mr32, hw = choice == -2 ? 16 : choice == -4 ? 8 : 32;
    const bool neu_fast = choice != -3 && j.neu_items && fast_neu_available(dim, p->degree, mr, j.L, hw);
    StencilJob jf = j;
    if (!neu_fast) jf.neu_items = jf.neu_count = nullptr;
    CK(launch_fast(jf, choice), "gmls_stencils fast launch");
    if (neu_fast) {
      StencilJob jn = jf;
      jn.items = jf.neu_items;
      jn.n_items = jf.neu_count;
      jn.neu_items = jn.neu_count = nullptr;
      CK(launch_stencils_fast(ctx->launch(), jn, mr, hw, sms, true), "gmls_stencils Neumann launch");
    }
    // targets the register kernels handed off (tile misfits; Neumann rows
    // without a Neumann instantiation; the factored kernel's well-conditioned
    // targets that one refinement pass left short of the tolerance): the
    // shared-memory FP32 kernel, whose failures join the FP64 redo list
    StencilJob jg = j;
    jg.items = j.gen_items;
    jg.n_items = j.gen_count;
    // (with uniform neighbour counts only Neumann rows or a tile with fewer
    // rows than basis functions are handed off)
    const int vg = heuristic_variant(ld, nmax, true);
    if (vg && (p->neumann || ld < nmax || choice == -3))
      CK(launch_single(ctx, jg, vg, ld, nmax, true, counter, sms), "gmls_stencils hand-off launch");
  } else
    CK(launch_single(ctx, j, choice, ld, nmax, refine, counter, sms), "gmls_stencils launch");
  return GMLS_OK;
}

// Uneven shapes (per-target degree or radius neighbour lists): bucket the
// targets on the device by (degree, row class) and run ONE persistent launch
// over all buckets; warps per target per bucket from the autotuner cache (or
// timed now, which reads the bucket sizes back once), else the heuristic.
static gmls_status launch_bucketed(gmls_ctx* ctx, const StencilJob& j, const gmls_stencil_params* p, bool refine,
                                   int ld_max, int sms, int32_t* counter) {
  static const int kClasses[] = {32, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024};
  const int dim = j.dim;
  BucketJob b;
  std::memset(&b, 0, sizeof(b));
  b.n_tgt = j.n_tgt;
  b.off = j.off;
  b.degree_pt = j.degree_pt;
  b.degree = j.degree;
  b.nc = j.nc;
  for (int c : kClasses) {
    b.class_rows[b.n_classes++] = c;
    if (c >= ld_max) break;
  }
  b.nb = 4 * b.n_classes + 1;
  BatchPlan pl;
  std::memset(&pl, 0, sizeof(pl));
  pl.single = 0;
  pl.nb = b.nb;
  for (int m = 1; m <= 4; ++m)
    for (int rc = 0; rc < b.n_classes; ++rc) {
      const int bi = (m - 1) * b.n_classes + rc;
      pl.ld[bi] = b.class_rows[rc];
      pl.nmax[bi] = gmls_gen::basis_size(p->basis, dim, m);
      const TuneKey key{p->basis, dim, m, p->precision, pl.ld[bi], j.L, p->neumann, 1};
      auto it = ctx->tune.find(key);
      const int v = (it != ctx->tune.end()) ? it->second : heuristic_variant(pl.ld[bi], pl.nmax[bi], refine);
      pl.G[bi] = v_warps(v);
      pl.gtile[bi] = v_place(v);
    }
  pl.ld[b.nb - 1] = 32;  // targets larger than every class: reported as unsupported
  pl.nmax[b.nb - 1] = 1;
  pl.G[b.nb - 1] = 1;
  for (int bi = 0; bi < b.nb; ++bi) {
    if (pl.G[bi] == 0) {  // no variant fits: send these targets to the unsupported bucket
      pl.G[bi] = 1;
      pl.gtile[bi] = kPlaceShared;
      pl.ld[bi] = 32;
      pl.nmax[bi] = 1;
    }
    b.gpb[bi] = 4 / pl.G[bi];
  }
  b.counts = arena_alloc<int32_t>(ctx, b.nb);
  b.fill = arena_alloc<int32_t>(ctx, b.nb);
  b.bucket_of = arena_alloc<int32_t>(ctx, std::max<int64_t>(j.n_tgt, 1));
  b.bucket_start = arena_alloc<int32_t>(ctx, b.nb + 1);
  b.task_start = arena_alloc<int32_t>(ctx, b.nb + 1);
  b.items = arena_alloc<int32_t>(ctx, std::max<int64_t>(j.n_tgt, 1));
  int32_t* nsample = arena_alloc<int32_t>(ctx, 1);
  auto release = [&]() {
    for (void* q : {(void*)b.counts, (void*)b.fill, (void*)b.bucket_of, (void*)b.bucket_start, (void*)b.task_start,
                    (void*)b.items, (void*)nsample})
      ctx->arena.release(q);
  };
  if (!b.counts || !b.fill || !b.bucket_of || !b.bucket_start || !b.task_start || !b.items || !nsample) {
    release();
    return fail(ctx, GMLS_ENOMEM, "gmls_stencils: arena exhausted (bucketing)");
  }
  Launch L = ctx->launch();
  cudaError_t e = launch_bucketing(L, b);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(ctx, e, "gmls_stencils bucketing");
  }
  // autotune buckets that have no cached choice (reads the bucket sizes once)
  bool need = false;
  for (int m = 1; m <= 4 && !need; ++m)
    for (int rc = 0; rc < b.n_classes; ++rc) {
      const TuneKey key{p->basis, dim, m, p->precision, b.class_rows[rc], j.L, p->neumann, 1};
      if (!ctx->tune.count(key)) need = true;
    }
  if (need && ctx->autotune && !ctx->force_generic && !capturing(ctx)) {
    // The launch gives every bucket the shared memory of its largest one: a
    // variant that lifts it past the most the kernel's full count of blocks
    // per SM allows would slow every other bucket down (a tiny bucket's
    // choice once cost the 3D uneven batch 80 -> 111 ms).  So a bucket takes
    // the fastest variant within that footprint when it is within 1.25 x of
    // its fastest overall.
    const int bmax = stencil_blocks_per_sm(refine, 0);
    size_t fit = 0;
    for (size_t lo = 0, hi = 227 * 1024; lo <= hi;) {
      const size_t mid = (lo + hi) / 2;
      if (stencil_blocks_per_sm(refine, mid) >= bmax) {
        fit = mid;
        lo = mid + 1;
      } else {
        if (mid == 0) break;
        hi = mid - 1;
      }
    }
    std::vector<int32_t> cnt(b.nb), start(b.nb + 1);
    cudaMemcpyAsync(cnt.data(), b.counts, sizeof(int32_t) * b.nb, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(start.data(), b.bucket_start, sizeof(int32_t) * (b.nb + 1), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (int m = 1; m <= 4; ++m)
      for (int rc = 0; rc < b.n_classes; ++rc) {
        const int bi = (m - 1) * b.n_classes + rc;
        const TuneKey key{p->basis, dim, m, p->precision, b.class_rows[rc], j.L, p->neumann, 1};
        if (ctx->tune.count(key)) continue;
        if (cnt[bi] == 0) {  // nothing to time: keep the heuristic (later calls skip this pass)
          ctx->tune[key] = heuristic_variant(b.class_rows[rc], gmls_gen::basis_size(p->basis, dim, m), refine);
          continue;
        }
        const int32_t ns = std::min<int32_t>(cnt[bi], 4096);
        cudaMemcpyAsync(nsample, &ns, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
        StencilJob js = j;
        js.items = b.items + start[bi];
        js.n_items = nsample;
        float best = 1e30f, best_fit = 1e30f;
        int choice = 0, choice_fit = 0;
        for (int v : generic_candidates(pl.ld[bi], pl.nmax[bi], refine)) {
          float ms = time_launch(ctx, [&]() {
            if (refine) cudaMemsetAsync(j.fb_count, 0, 3 * sizeof(int32_t), ctx->stream);
            launch_single(ctx, js, v, pl.ld[bi], pl.nmax[bi], refine, counter, sms);
          });
          ctx->tune_log.push_back({key, v, ms});
          if (ms < best) {
            best = ms;
            choice = v;
          }
          const size_t sv = (size_t)(4 / v_warps(v)) * tile_bytes(pl.ld[bi], pl.nmax[bi], refine, v_place(v));
          if (sv <= fit && ms < best_fit) {
            best_fit = ms;
            choice_fit = v;
          }
        }
        if (choice_fit && best_fit <= 1.25f * best) choice = choice_fit;
        if (choice) {
          ctx->tune[key] = choice;
          pl.G[bi] = v_warps(choice);
          pl.gtile[bi] = v_place(choice);
          b.gpb[bi] = 4 / pl.G[bi];
        }
      }
    // block tasks depend on the chosen G: recompute the plan
    e = launch_bucketing(L, b);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(ctx, e, "gmls_stencils bucketing");
    }
  }
  pl.items = b.items;
  pl.bucket_start = b.bucket_start;
  pl.task_start = b.task_start;
  pl.task_counter = counter;
  const size_t smem = plan_smem(pl, refine);
  const int grid = sms * stencil_blocks_per_sm(refine, smem);
  void* owned = nullptr;
  if (!plan_gscratch(ctx, pl, refine, grid, &owned)) {
    release();
    return fail(ctx, GMLS_ENOMEM, "gmls_stencils: arena exhausted (global tiles)");
  }
  if (refine) CK(cudaMemsetAsync(j.fb_count, 0, 3 * sizeof(int32_t), ctx->stream), "gmls_stencils memset");
  e = cudaMemsetAsync(counter, 0, sizeof(int32_t), ctx->stream);
  if (e == cudaSuccess) e = launch_stencils(L, j, pl, refine, smem, grid);
  ctx->arena.release(owned);
  release();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmls_stencils bucketed launch");
  return GMLS_OK;
}

static gmls_status plan_and_launch(gmls_ctx* ctx, const StencilJob& j0, const gmls_stencil_params* p, NbrObj& nb,
                                   StencilObj& s, bool refine, int ld, int nmax, int sms) {
  StencilJob j = j0;
  int32_t* counter = arena_alloc<int32_t>(ctx, 2);
  if (!counter) return fail(ctx, GMLS_ENOMEM, "gmls_stencils: arena exhausted");
  const bool uniform = !p->degree_per_target && !nb.variable;
  gmls_status rc = uniform ? launch_uniform(ctx, j, p, refine, ld, nmax, sms, counter)
                           : launch_bucketed(ctx, j, p, refine, ld, sms, counter);
  if (rc == GMLS_OK && refine) {
    // FP64 redo of the targets the FP32 path handed back
    StencilJob jf = j;
    jf.items = s.fb_items;
    jf.n_items = s.fb_count;
    jf.fallback_run = 1;
    const int gf = heuristic_variant(ld, nmax, false);
    if (gf) {
      cudaError_t e = launch_single(ctx, jf, gf, ld, nmax, false, counter + 1, sms);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "gmls_stencils FP64 redo");
    }
  }
  ctx->arena.release(counter);
  return rc;
}

extern "C" {

const char* gmls_version(void) { return "gmls-gb300 0.1 (sm_103a)"; }

const char* gmls_last_error(gmls_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

gmls_status gmls_create(gmls_ctx** out, int device, void* cuda_stream, void* arena, size_t arena_bytes) {
  if (!out || !arena || arena_bytes < (1u << 20)) {
    g_create_error = "gmls_create: out and arena must be non-NULL and arena_bytes >= 1 MiB";
    return GMLS_EINVAL;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    g_create_error = std::string("gmls_create: no such CUDA device (") + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return GMLS_ECUDA;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    g_create_error = std::string("gmls_create: ") + cudaGetErrorString(e);
    return GMLS_ECUDA;
  }
  gmls_ctx* c = new gmls_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->arena.init(arena, arena_bytes);
  *out = c;
  return GMLS_OK;
}

gmls_status gmls_destroy(gmls_ctx* ctx) {
  if (!ctx) return GMLS_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return GMLS_OK;
}

gmls_status gmls_set_stream(gmls_ctx* ctx, void* cuda_stream) {
  if (!ctx) return GMLS_EINVAL;
  cudaSetDevice(ctx->device);
  // released arena blocks may still be read by work on the old stream
  CK(cudaStreamSynchronize(ctx->stream), "gmls_set_stream");
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return GMLS_OK;
}

gmls_status gmls_sync(gmls_ctx* ctx) {
  if (!ctx) return GMLS_EINVAL;
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream), "gmls_sync");
  CK(cudaGetLastError(), "gmls_sync");
  return GMLS_OK;
}

gmls_status gmls_arena_usage(gmls_ctx* ctx, size_t* used, size_t* peak, size_t* capacity) {
  if (!ctx) return GMLS_EINVAL;
  if (used) *used = ctx->arena.used();
  if (peak) *peak = ctx->arena.peak();
  if (capacity) *capacity = ctx->arena.cap();
  return GMLS_OK;
}

gmls_status gmls_set_option(gmls_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return GMLS_EINVAL;
  switch (option) {
    case GMLS_OPT_FORCE_GENERIC: ctx->force_generic = value != 0; return GMLS_OK;
    case GMLS_OPT_FAIL_ALLOC:
      if (value < 0) return fail(ctx, GMLS_EINVAL, "gmls_set_option: GMLS_OPT_FAIL_ALLOC needs n >= 0");
      ctx->arena.fail_after(value);
      return GMLS_OK;
    case GMLS_OPT_AUTOTUNE: ctx->autotune = value != 0; return GMLS_OK;
    case GMLS_OPT_FORCE_VARIANT:
      if (value != 0 && value != -1 && value != -2 && value != -3 && value != -4 &&
          !(value > 0 && value < 24 && (v_warps((int)value) == 1 || v_warps((int)value) == 2 ||
                                        v_warps((int)value) == 4)))
        return fail(ctx, GMLS_EINVAL, "gmls_set_option: variant must be 0, -1 .. -4 or G + 8 * P (G 1, 2, 4; P 0, 1, 2)");
      ctx->force_variant = (int)value;
      return GMLS_OK;
    case GMLS_OPT_POISON:
      ctx->poison = value != 0;
      return GMLS_OK;
    case GMLS_OPT_ORDER_KEY64:
      ctx->order_key64 = value != 0;
      return GMLS_OK;
    case GMLS_OPT_CLEAR_TUNING:
      ctx->tune.clear();
      ctx->tune_log.clear();
      return GMLS_OK;
    default: return fail(ctx, GMLS_EINVAL, "gmls_set_option: unknown option");
  }
}

gmls_status gmls_tune_info(gmls_ctx* ctx, int32_t index, int32_t* fields, float* ms) {
  if (!ctx || !fields) return GMLS_EINVAL;
  if (index < 0 || index >= (int32_t)ctx->tune_log.size()) return fail(ctx, GMLS_ENOTFOUND, "gmls_tune_info: no such record");
  const TuneRecord& r = ctx->tune_log[index];
  const int32_t v[9] = {r.key.basis, r.key.dim, r.key.degree, r.key.precision, r.key.ld, r.key.L, r.key.neumann,
                        r.key.bucketed, r.variant};
  for (int i = 0; i < 9; ++i) fields[i] = v[i];
  if (ms) *ms = r.ms;
  return GMLS_OK;
}

gmls_status gmls_capture_begin(gmls_ctx* ctx) {
  if (!ctx) return GMLS_EINVAL;
  CK(cudaSetDevice(ctx->device), "gmls_capture_begin");
  if (!ctx->stream) return fail(ctx, GMLS_EINVAL, "gmls_capture_begin: the legacy default stream cannot be captured");
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed), "gmls_capture_begin");
  return GMLS_OK;
}

gmls_status gmls_capture_end(gmls_ctx* ctx, int64_t* graph_id) {
  if (!ctx || !graph_id) return GMLS_EINVAL;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamEndCapture(ctx->stream, &graph), "gmls_capture_end");
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmls_capture_end instantiate");
  Obj o;
  o.kind = K_GRAPH;
  o.exec = exec;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *graph_id = id;
  return GMLS_OK;
}

gmls_status gmls_graph_launch(gmls_ctx* ctx, int64_t graph_id) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(graph_id);
  if (it == ctx->objs.end() || it->second.kind != K_GRAPH) return fail(ctx, GMLS_ENOTFOUND, "gmls_graph_launch: no such graph");
  CK(cudaSetDevice(ctx->device), "gmls_graph_launch");
  CK(cudaGraphLaunch(it->second.exec, ctx->stream), "gmls_graph_launch");
  ctx->launches += 1;
  return GMLS_OK;
}

gmls_status gmls_launch_count(gmls_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return GMLS_EINVAL;
  *launches = ctx->launches;
  return GMLS_OK;
}

gmls_status gmls_cloud(gmls_ctx* ctx, int dim, int64_t n, const double* xyz, const double* normals,
                       const uint8_t* bflags, int64_t* cloud_id) {
  if (!ctx) return GMLS_EINVAL;
  if (!cloud_id || !xyz || (dim != 2 && dim != 3) || n < 1 || n > INT32_MAX)
    return fail(ctx, GMLS_EINVAL, "gmls_cloud: need dim in {2,3}, 1 <= n < 2^31, xyz and cloud_id non-NULL");
  CK(cudaSetDevice(ctx->device), "gmls_cloud");
  Obj o;
  o.kind = K_CLOUD;
  CloudObj& c = o.c;
  c.dim = dim;
  c.n = n;
  // cells per axis: about two particles per cell over the bounding box
  int32_t nc_axis[3] = {1, 1, 1};
  double per_axis = std::pow(std::max(1.0, n / 2.0), 1.0 / dim);
  for (int a = 0; a < dim; ++a) nc_axis[a] = std::max(1, std::min(1 << 20, (int)std::ceil(per_axis)));
  int64_t ncell = 1;
  for (int a = 0; a < dim; ++a) ncell *= nc_axis[a];
  c.ncell = ncell;
  const int n_part = (int)std::min<int64_t>(256, (n + 255) / 256);
  const int64_t scan_elems = scan_scratch_elems(ncell);
  c.x = arena_alloc<double>(ctx, (size_t)dim * n);
  c.xs = arena_alloc<double>(ctx, (size_t)dim * n);
  c.xsf = arena_alloc<float>(ctx, (size_t)dim * n);
  c.sorted = arena_alloc<int32_t>(ctx, n);
  c.cell_start = arena_alloc<int32_t>(ctx, ncell + 1);
  c.grid = arena_alloc<GridParams>(ctx, 1);
  if (normals) c.normals = arena_alloc<double>(ctx, (size_t)dim * n);
  if (bflags) c.bflag = arena_alloc<uint8_t>(ctx, n);
  double* part = arena_alloc<double>(ctx, (size_t)n_part * 6);
  int32_t* cell_of = arena_alloc<int32_t>(ctx, n);
  int32_t* counts = arena_alloc<int32_t>(ctx, ncell);
  int32_t* fill = arena_alloc<int32_t>(ctx, ncell);
  int32_t* scan_tmp = arena_alloc<int32_t>(ctx, scan_elems);
  void* all[] = {c.x, c.xs, c.xsf, c.sorted, c.cell_start, c.grid, part, cell_of, counts, fill, scan_tmp};
  bool oom = false;
  for (void* p : all) oom |= (p == nullptr);
  oom |= (normals && !c.normals) || (bflags && !c.bflag);
  if (oom) {
    for (void* p : all) ctx->arena.release(p);
    ctx->arena.release(c.normals);
    ctx->arena.release(c.bflag);
    return fail(ctx, GMLS_ENOMEM, "gmls_cloud: arena exhausted");
  }
  Launch L = ctx->launch();
  CK(copy_in(ctx, c.x, xyz, sizeof(double) * dim * n), "gmls_cloud copy");
  if (normals) CK(copy_in(ctx, c.normals, normals, sizeof(double) * dim * n), "gmls_cloud copy normals");
  if (bflags) CK(copy_in(ctx, c.bflag, bflags, n), "gmls_cloud copy flags");
  CK(cudaMemsetAsync(counts, 0, sizeof(int32_t) * ncell, ctx->stream), "gmls_cloud memset");
  CK(cudaMemsetAsync(fill, 0, sizeof(int32_t) * ncell, ctx->stream), "gmls_cloud memset");
  CK(launch_bbox_and_grid(L, dim, n, c.x, nc_axis, c.grid, part, n_part), "gmls_cloud bbox");
  CK(launch_cell_count(L, dim, n, c.x, c.grid, cell_of, counts), "gmls_cloud count");
  CK(launch_scan_i32(L, counts, c.cell_start, ncell, scan_tmp, scan_elems), "gmls_cloud scan");
  CK(launch_cell_scatter(L, dim, n, c.x, c.grid, cell_of, c.cell_start, fill, c.sorted, c.xs, c.xsf), "gmls_cloud scatter");
  ctx->arena.release(part);
  ctx->arena.release(cell_of);
  ctx->arena.release(counts);
  ctx->arena.release(fill);
  ctx->arena.release(scan_tmp);
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *cloud_id = id;
  return GMLS_OK;
}

gmls_status gmls_neighbors(gmls_ctx* ctx, int64_t cloud_id, const gmls_nbr_params* p, int64_t* nbrs_id) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(cloud_id);
  if (it == ctx->objs.end() || it->second.kind != K_CLOUD) return fail(ctx, GMLS_ENOTFOUND, "gmls_neighbors: no such cloud");
  if (!p || !nbrs_id) return fail(ctx, GMLS_EINVAL, "gmls_neighbors: NULL params");
  CloudObj& c = it->second.c;
  if ((p->mode != GMLS_NBR_KNN && p->mode != GMLS_NBR_RADIUS) || p->k < 1 || p->k > kMaxK || !(p->eps_factor > 0.0) ||
      p->reserved != 0)
    return fail(ctx, GMLS_EINVAL, "gmls_neighbors: need mode KNN/RADIUS, 1 <= k <= 1024, eps_factor > 0");
  if (p->mode == GMLS_NBR_RADIUS && (p->cap < p->k || p->cap > kMaxK))
    return fail(ctx, GMLS_EINVAL, "gmls_neighbors: radius mode needs k <= cap <= 1024");
  const bool variable = p->mode == GMLS_NBR_RADIUS || p->k_per_target;
  if (p->mode == GMLS_NBR_KNN && p->k > c.n)
    return fail(ctx, GMLS_EINVAL, "gmls_neighbors: k exceeds the number of particles");
  const int64_t nt = p->targets ? p->n_targets : c.n;
  if (nt < 0 || nt > INT32_MAX) return fail(ctx, GMLS_EINVAL, "gmls_neighbors: bad n_targets");
  CK(cudaSetDevice(ctx->device), "gmls_neighbors");
  Obj o;
  o.kind = K_NBRS;
  NbrObj& nb = o.nb;
  nb.cloud = cloud_id;
  nb.dim = c.dim;
  nb.n_tgt = nt;
  nb.mode = p->mode;
  nb.k = p->k;
  nb.cap = p->mode == GMLS_NBR_RADIUS ? p->cap : p->k;
  nb.variable = variable;
  nb.all_targets = p->targets == nullptr;
  nb.idx_cap = nt * (int64_t)nb.cap;
  nb.tgt = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
  nb.off = arena_alloc<int64_t>(ctx, nt + 1);
  nb.idx = arena_alloc<int32_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
  nb.eps = arena_alloc<double>(ctx, std::max<int64_t>(nt, 1));
  nb.status = arena_alloc<uint8_t>(ctx, std::max<int64_t>(nt, 1));
  double* hs = p->halfspace ? arena_alloc<double>(ctx, (size_t)nt * c.dim) : nullptr;
  int32_t* kpt = p->k_per_target ? arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1)) : nullptr;
  int32_t* padded = nullptr;
  int32_t* cnt = nullptr;
  int64_t* scan_tmp = nullptr;
  int64_t scan_elems = 0;
  if (variable) {
    padded = arena_alloc<int32_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
    cnt = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
    scan_elems = scan_scratch_elems(nt);
    scan_tmp = arena_alloc<int64_t>(ctx, scan_elems);
  }
  bool oom = !nb.tgt || !nb.off || !nb.idx || !nb.eps || !nb.status || (p->halfspace && !hs) ||
             (p->k_per_target && !kpt) || (variable && (!padded || !cnt || !scan_tmp));
  if (oom) {
    for (void* q : {(void*)nb.tgt, (void*)nb.off, (void*)nb.idx, (void*)nb.eps, (void*)nb.status, (void*)hs,
                    (void*)kpt, (void*)padded, (void*)cnt, (void*)scan_tmp})
      ctx->arena.release(q);
    return fail(ctx, GMLS_ENOMEM, "gmls_neighbors: arena exhausted");
  }
  Launch L = ctx->launch();
  if (p->targets)
    CK(copy_in(ctx, nb.tgt, p->targets, sizeof(int32_t) * nt), "gmls_neighbors copy targets");
  else
    CK(launch_fill_identity(L, nb.tgt, nt), "gmls_neighbors identity");
  if (hs) CK(copy_in(ctx, hs, p->halfspace, sizeof(double) * nt * c.dim), "gmls_neighbors copy halfspace");
  if (kpt) CK(copy_in(ctx, kpt, p->k_per_target, sizeof(int32_t) * nt), "gmls_neighbors copy k");
  NbrQuery q;
  q.cloud = CloudDev{c.dim, c.n, c.x, c.xs, c.sorted, c.cell_start, c.grid, c.ncell, c.xsf};
  q.n_tgt = nt;
  q.tgt = nb.tgt;
  q.halfspace = hs;
  q.mode = p->mode;
  q.k = p->k;
  q.k_pt = kpt;
  q.cap = nb.cap;
  q.eps_factor = p->eps_factor;
  q.out_idx = variable ? padded : nb.idx;
  q.out_cnt = cnt;
  q.out_eps = nb.eps;
  q.out_status = nb.status;
  CK(launch_nbr_query(L, q), "gmls_neighbors query");
  if (!variable) {
    CK(launch_fill_offsets_fixed(L, nb.off, nt, p->k), "gmls_neighbors offsets");
  } else {
    CK(launch_scan_i64_from_i32(L, cnt, nb.off, nt, scan_tmp, scan_elems), "gmls_neighbors scan");
    CK(launch_compact_padded(L, padded, nb.cap, cnt, nb.off, nb.idx, nt), "gmls_neighbors compact");
  }
  ctx->arena.release(hs);
  ctx->arena.release(kpt);
  ctx->arena.release(padded);
  ctx->arena.release(cnt);
  ctx->arena.release(scan_tmp);
  c.refs++;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *nbrs_id = id;
  return GMLS_OK;
}

gmls_status gmls_neighbors_prefix(gmls_ctx* ctx, int64_t nbrs_id, int32_t k, double eps_factor, int64_t* out_id) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(nbrs_id);
  if (it == ctx->objs.end() || it->second.kind != K_NBRS)
    return fail(ctx, GMLS_ENOTFOUND, "gmls_neighbors_prefix: no such neighbour handle");
  if (!out_id) return fail(ctx, GMLS_EINVAL, "gmls_neighbors_prefix: NULL output");
  NbrObj& src = it->second.nb;
  if (src.variable || src.mode != GMLS_NBR_KNN || k < 1 || k > src.k || !(eps_factor > 0.0))
    return fail(ctx, GMLS_EINVAL, "gmls_neighbors_prefix: needs a fixed-k nearest-neighbour handle and 1 <= k <= its k");
  CloudObj& c = ctx->objs.at(src.cloud).c;
  CK(cudaSetDevice(ctx->device), "gmls_neighbors_prefix");
  Obj o;
  o.kind = K_NBRS;
  NbrObj& nb = o.nb;
  nb.cloud = src.cloud;
  nb.dim = src.dim;
  nb.n_tgt = src.n_tgt;
  nb.all_targets = src.all_targets;
  nb.mode = GMLS_NBR_KNN;
  nb.k = k;
  nb.cap = k;
  nb.idx_cap = src.n_tgt * (int64_t)k;
  nb.parent = nbrs_id;
  const int64_t nt = src.n_tgt;
  nb.tgt = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
  nb.off = arena_alloc<int64_t>(ctx, nt + 1);
  nb.idx = arena_alloc<int32_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
  nb.eps = arena_alloc<double>(ctx, std::max<int64_t>(nt, 1));
  nb.status = arena_alloc<uint8_t>(ctx, std::max<int64_t>(nt, 1));
  if (!nb.tgt || !nb.off || !nb.idx || !nb.eps || !nb.status) {
    for (void* q : {(void*)nb.tgt, (void*)nb.off, (void*)nb.idx, (void*)nb.eps, (void*)nb.status}) ctx->arena.release(q);
    return fail(ctx, GMLS_ENOMEM, "gmls_neighbors_prefix: arena exhausted");
  }
  Launch L = ctx->launch();
  CK(cudaMemcpyAsync(nb.tgt, src.tgt, sizeof(int32_t) * nt, cudaMemcpyDeviceToDevice, ctx->stream),
     "gmls_neighbors_prefix copy");
  CK(launch_fill_offsets_fixed(L, nb.off, nt, k), "gmls_neighbors_prefix offsets");
  CK(launch_nbr_prefix(L, c.dim, c.n, c.x, src.tgt, nt, src.idx, src.k, k, eps_factor, nb.idx, nb.eps, nb.status),
     "gmls_neighbors_prefix");
  c.refs++;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *out_id = id;
  return GMLS_OK;
}

// rows / components of one functional's output
static bool functional_shape(int basis, int dim, int fn, int* rows, int* ncomp) {
  switch (fn) {
    case GMLS_F_GRAD:
      if (basis != GMLS_BASIS_SCALAR && basis != GMLS_BASIS_STAGGERED) return false;
      *rows = dim, *ncomp = 1;
      return true;
    case GMLS_F_LAPLACIAN:
      if (basis != GMLS_BASIS_SCALAR && basis != GMLS_BASIS_STAGGERED) return false;
      *rows = 1, *ncomp = 1;
      return true;
    case GMLS_F_DIV:
      if (basis == GMLS_BASIS_STAGGERED) return false;
      *rows = 1, *ncomp = dim;
      return true;
    case GMLS_F_VEC_LAPLACIAN:
    case GMLS_F_CURLCURL:
      if (basis != GMLS_BASIS_DIVFREE) return false;
      *rows = dim, *ncomp = dim;
      return true;
    default:
      return false;
  }
}

gmls_status gmls_stencils(gmls_ctx* ctx, int64_t nbrs_id, const gmls_stencil_params* p, int64_t* stencil_id) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(nbrs_id);
  if (it == ctx->objs.end() || it->second.kind != K_NBRS) return fail(ctx, GMLS_ENOTFOUND, "gmls_stencils: no such neighbour handle");
  if (!p || !stencil_id) return fail(ctx, GMLS_EINVAL, "gmls_stencils: NULL params");
  NbrObj& nb = it->second.nb;
  CloudObj& c = ctx->objs.at(nb.cloud).c;
  const int dim = nb.dim;
  if (p->basis != GMLS_BASIS_SCALAR && p->basis != GMLS_BASIS_DIVFREE && p->basis != GMLS_BASIS_STAGGERED)
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: unknown basis");
  if (p->weight != GMLS_WEIGHT_POLY || p->weight_power < 1)
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: weight must be GMLS_WEIGHT_POLY with power >= 1");
  if (p->precision != GMLS_FP64 && p->precision != GMLS_FP32_REFINE)
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: unknown precision");
  if (!p->degree_per_target && (p->degree < 1 || p->degree > 4))
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: degree must be 1..4");
  if (p->n_functionals < 1 || p->n_functionals > 5) return fail(ctx, GMLS_EINVAL, "gmls_stencils: 1..5 functionals");
  if (p->neumann && p->basis != GMLS_BASIS_SCALAR)
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: the Neumann constraint needs the scalar basis");
  if (p->neumann && (!c.normals || !c.bflag))
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: Neumann targets need cloud normals and boundary flags");
  CK(cudaSetDevice(ctx->device), "gmls_stencils");

  Obj o;
  o.kind = K_STENCIL;
  StencilObj& s = o.s;
  s.nbrs = nbrs_id;
  s.basis = p->basis;
  s.dim = dim;
  StencilJob j;
  std::memset(&j, 0, sizeof(j));
  // solve rows
  bool need_grad = false, need_lap = false, need_vlap = false;
  for (int f = 0; f < p->n_functionals; ++f) {
    const int fn = p->functionals[f];
    int rows, ncomp;
    if (!functional_shape(p->basis, dim, fn, &rows, &ncomp))
      return fail(ctx, GMLS_EINVAL, "gmls_stencils: functional not defined for this basis");
    for (int g = 0; g < f; ++g)
      if (p->functionals[g] == fn) return fail(ctx, GMLS_EINVAL, "gmls_stencils: repeated functional");
    s.fn[f] = fn;
    s.rows[f] = rows;
    s.ncomp[f] = ncomp;
    if (fn == GMLS_F_GRAD || (fn == GMLS_F_DIV && p->basis == GMLS_BASIS_SCALAR)) need_grad = true;
    if (fn == GMLS_F_LAPLACIAN) need_lap = true;
    if (fn == GMLS_F_VEC_LAPLACIAN || fn == GMLS_F_CURLCURL) need_vlap = true;
  }
  s.nout = p->n_functionals;
  int L = 0, grad0 = -1, lap0 = -1, vlap0 = -1;
  if (need_grad) {
    grad0 = L;
    for (int r = 0; r < dim; ++r, ++L) j.lam_fn[L] = 0, j.lam_row[L] = r, j.lam_order[L] = 1;
  }
  if (need_lap) {
    lap0 = L;
    j.lam_fn[L] = 1, j.lam_row[L] = 0, j.lam_order[L] = 2;
    ++L;
  }
  if (need_vlap) {
    vlap0 = L;
    for (int r = 0; r < dim; ++r, ++L) j.lam_fn[L] = 2, j.lam_row[L] = r, j.lam_order[L] = 2;
  }
  if (L > kMaxSolveRows) return fail(ctx, GMLS_EINVAL, "gmls_stencils: too many solve rows");
  s.L = L;
  const int nc = (p->basis == GMLS_BASIS_DIVFREE) ? dim : 1;
  int max_deg = p->degree;
  if (p->degree_per_target) max_deg = 4;
  const int nmax = gmls_gen::basis_size(p->basis, dim, max_deg);
  if (nmax <= 0) return fail(ctx, GMLS_EINVAL, "gmls_stencils: unsupported (dim, degree, basis)");
  const int kmax = nb.cap;
  const int ld = kmax * nc;
  const int64_t nt = nb.n_tgt;

  // allocations
  bool oom = false;
  for (int f = 0; f < s.nout; ++f) {
    s.w[f] = arena_alloc<double>(ctx, std::max<int64_t>(nb.idx_cap * s.rows[f] * s.ncomp[f], 1));
    oom |= !s.w[f];
  }
  s.beta = arena_alloc<double>(ctx, std::max<int64_t>(nt * std::max(L, 1), 1));
  s.status = arena_alloc<uint8_t>(ctx, std::max<int64_t>(nt, 1));
  s.iters = arena_alloc<uint8_t>(ctx, std::max<int64_t>(nt, 1));
  int8_t* deg = p->degree_per_target ? arena_alloc<int8_t>(ctx, std::max<int64_t>(nt, 1)) : nullptr;
  const bool refine = p->precision == GMLS_FP32_REFINE;
  if (refine) {
    // the FP64 redo list, the register kernel's hand-off to the shared-memory
    // kernel, and (Neumann targets) its list for the Neumann instantiation
    s.fb_items = arena_alloc<int32_t>(ctx, (p->neumann ? 3 : 2) * std::max<int64_t>(nt, 1));
    s.fb_count = arena_alloc<int32_t>(ctx, 3);
  }
  oom |= !s.beta || !s.status || !s.iters || (p->degree_per_target && !deg) || (refine && (!s.fb_items || !s.fb_count));
  auto release_all = [&]() {
    for (int f = 0; f < 5; ++f) ctx->arena.release(s.w[f]);
    ctx->arena.release(s.beta);
    ctx->arena.release(s.status);
    ctx->arena.release(s.iters);
    ctx->arena.release(deg);
    ctx->arena.release(s.fb_items);
    ctx->arena.release(s.fb_count);
  };
  if (oom) {
    release_all();
    return fail(ctx, GMLS_ENOMEM, "gmls_stencils: arena exhausted");
  }
  if (deg) CK(copy_in(ctx, deg, p->degree_per_target, nt), "gmls_stencils copy degrees");
  if (ctx->poison) {  // testing: every entry must be written by the kernels
    for (int f = 0; f < s.nout; ++f)
      CK(cudaMemsetAsync(s.w[f], 0xFF, sizeof(double) * std::max<int64_t>(nb.idx_cap * s.rows[f] * s.ncomp[f], 1),
                         ctx->stream), "gmls_stencils poison");
    CK(cudaMemsetAsync(s.beta, 0xFF, sizeof(double) * std::max<int64_t>(nt * std::max(L, 1), 1), ctx->stream),
       "gmls_stencils poison");
    CK(cudaMemsetAsync(s.status, 0xFF, std::max<int64_t>(nt, 1), ctx->stream), "gmls_stencils poison");
    CK(cudaMemsetAsync(s.iters, 0xFF, std::max<int64_t>(nt, 1), ctx->stream), "gmls_stencils poison");
  }

  j.dim = dim;
  j.n = c.n;
  j.x = c.x;
  j.normals = c.normals;
  j.bflag = c.bflag;
  j.n_tgt = nt;
  j.tgt = nb.tgt;
  j.off = nb.off;
  j.idx = nb.idx;
  j.eps = nb.eps;
  j.nbr_status = nb.status;
  j.items = nullptr;
  j.n_items = nullptr;
  j.kind = p->basis;
  j.degree = p->degree;
  j.degree_pt = deg;
  j.nc = nc;
  j.wpow = (double)p->weight_power;
  j.wpow_half = p->weight_power / 2;
  j.neumann = p->neumann;
  j.L = L;
  j.nout = s.nout;
  for (int f = 0; f < s.nout; ++f) {
    j.out_fn[f] = s.fn[f];
    j.out_rows[f] = s.rows[f];
    j.out_ncomp[f] = s.ncomp[f];
    j.out_w[f] = s.w[f];
    j.out_sign[f] = 1;
    switch (s.fn[f]) {
      case GMLS_F_GRAD: j.out_src[f] = grad0; break;
      case GMLS_F_LAPLACIAN: j.out_src[f] = lap0; break;
      case GMLS_F_DIV: j.out_src[f] = (p->basis == GMLS_BASIS_SCALAR) ? grad0 : -1; break;
      case GMLS_F_VEC_LAPLACIAN: j.out_src[f] = vlap0; break;
      case GMLS_F_CURLCURL: j.out_src[f] = vlap0, j.out_sign[f] = -1; break;
    }
  }
  for (int f = 0; f < s.nout; ++f) s.src[f] = j.out_src[f];
  s.neumann = p->neumann;
  j.beta = s.beta;
  j.status = s.status;
  j.iters = s.iters;
  j.max_refine = p->max_refine > 0 ? p->max_refine : 3;
  j.tol = p->refine_tol > 0.0 ? p->refine_tol : 1e-10;
  j.fb_items = s.fb_items;
  j.fb_count = s.fb_count;
  j.gen_items = refine ? s.fb_items + std::max<int64_t>(nt, 1) : nullptr;
  j.gen_count = refine ? s.fb_count + 1 : nullptr;
  j.neu_items = refine && p->neumann ? s.fb_items + 2 * std::max<int64_t>(nt, 1) : nullptr;
  j.neu_count = refine && p->neumann ? s.fb_count + 2 : nullptr;
  j.ld = ld;
  j.nmax = nmax;

  const int dev_sms = device_sm_count();
  gmls_status rc = GMLS_OK;
  if (nt > 0) {
    rc = plan_and_launch(ctx, j, p, nb, s, refine, ld, nmax, dev_sms);
    if (rc != GMLS_OK) {
      ctx->arena.release(deg);
      release_all();
      return rc;
    }
  }
  ctx->arena.release(deg);
  nb.refs++;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *stencil_id = id;
  return GMLS_OK;
}

// the lists' id order (lists never change after creation: computed once)
static gmls_status ensure_order(gmls_ctx* ctx, NbrObj& nb, const char* who) {
  if (nb.order) return GMLS_OK;
  // a prefix list takes its order from the longer list's (computed here if
  // missing): the positions below k, in that order, are its id order
  NbrObj* par = nullptr;
  if (nb.parent) {
    auto pit = ctx->objs.find(nb.parent);
    if (pit != ctx->objs.end() && pit->second.kind == K_NBRS && !pit->second.nb.variable &&
        pit->second.nb.n_tgt == nb.n_tgt && pit->second.nb.k >= nb.k)
      par = &pit->second.nb;
  }
  if (par) {
    gmls_status r = ensure_order(ctx, *par, who);
    if (r) return r;
  }
  nb.order = arena_alloc<int16_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
  if (!nb.order) return fail(ctx, GMLS_ENOMEM, std::string(who) + ": arena exhausted (neighbour id order)");
  int kcap = 1;
  while (kcap < nb.cap) kcap <<= 1;
  auto cit = ctx->objs.find(nb.cloud);
  const int64_t n_points = (!ctx->order_key64 && cit != ctx->objs.end() && cit->second.kind == K_CLOUD)
                               ? cit->second.c.n
                               : INT64_MAX;  // INT64_MAX: 64-bit keys
  cudaError_t e = par ? launch_nbr_order_prefix(ctx->launch(), nb.n_tgt, par->order, par->k, nb.k, nb.order)
                      : launch_nbr_order(ctx->launch(), nb.n_tgt, nb.off, nb.idx, kcap, nb.order, n_points);
  if (e != cudaSuccess) {
    ctx->arena.release(nb.order);
    nb.order = nullptr;
    return cuda_fail(ctx, e, who);
  }
  return GMLS_OK;
}

static int find_out(const StencilObj& s, int fn) {
  for (int f = 0; f < s.nout; ++f)
    if (s.fn[f] == fn) return f;
  return -1;
}

// total neighbour entries (reads the device offset when the lists are variable)
static gmls_status nbr_total(gmls_ctx* ctx, const NbrObj& nb, int64_t* total) {
  if (!nb.variable) {
    *total = nb.n_tgt * (int64_t)nb.k;
    return GMLS_OK;
  }
  if (capturing(ctx))
    return fail(ctx, GMLS_EBUSY, "the nonzero count of radius-mode lists is not readable during stream capture");
  int64_t v = 0;
  CK(cudaMemcpyAsync(&v, nb.off + nb.n_tgt, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream), "offset read");
  CK(cudaStreamSynchronize(ctx->stream), "offset read");
  *total = v;
  return GMLS_OK;
}

gmls_status gmls_stencil_info(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* n_targets,
                              int32_t* rows, int32_t* ncomp, int64_t* n_values) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(stencil_id);
  if (it == ctx->objs.end() || it->second.kind != K_STENCIL) return fail(ctx, GMLS_ENOTFOUND, "gmls_stencil_info: no such stencil handle");
  StencilObj& s = it->second.s;
  int f = find_out(s, functional);
  if (f < 0) return fail(ctx, GMLS_EINVAL, "gmls_stencil_info: functional not computed");
  NbrObj& nb = ctx->objs.at(s.nbrs).nb;
  if (n_targets) *n_targets = nb.n_tgt;
  if (rows) *rows = s.rows[f];
  if (ncomp) *ncomp = s.ncomp[f];
  if (n_values) {
    int64_t tot;
    gmls_status r = nbr_total(ctx, nb, &tot);
    if (r) return r;
    *n_values = tot * s.rows[f] * s.ncomp[f];
  }
  return GMLS_OK;
}

gmls_status gmls_csr_size(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* n_rows, int64_t* n_cols,
                          int64_t* nnz) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(stencil_id);
  if (it == ctx->objs.end() || it->second.kind != K_STENCIL) return fail(ctx, GMLS_ENOTFOUND, "gmls_csr_size: no such stencil handle");
  StencilObj& s = it->second.s;
  int f = find_out(s, functional);
  if (f < 0) return fail(ctx, GMLS_EINVAL, "gmls_csr_size: functional not computed");
  NbrObj& nb = ctx->objs.at(s.nbrs).nb;
  CloudObj& c = ctx->objs.at(nb.cloud).c;
  int64_t tot;
  gmls_status r = nbr_total(ctx, nb, &tot);
  if (r) return r;
  if (n_rows) *n_rows = nb.n_tgt * s.rows[f];
  if (n_cols) *n_cols = c.n * s.ncomp[f];
  if (nnz) *nnz = tot * s.rows[f] * s.ncomp[f];
  return GMLS_OK;
}

gmls_status gmls_assemble_csr_at(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t nnz_offset,
                                 int64_t* row_ptr, int32_t* col, double* val) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(stencil_id);
  if (it == ctx->objs.end() || it->second.kind != K_STENCIL) return fail(ctx, GMLS_ENOTFOUND, "gmls_assemble_csr: no such stencil handle");
  if (nnz_offset < 0) return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr_at: negative nnz_offset");
  StencilObj& s = it->second.s;
  int f = find_out(s, functional);
  if (f < 0) return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: functional not computed");
  NbrObj& nb = ctx->objs.at(s.nbrs).nb;
  // col and val may be NULL for a handle without targets (nothing is written there)
  if (!row_ptr || (nb.n_tgt > 0 && (!col || !val))) return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: NULL output");
  if (is_host_ptr(row_ptr) || (col && is_host_ptr(col)) || (val && is_host_ptr(val)))
    return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: outputs must be device buffers");
  CK(cudaSetDevice(ctx->device), "gmls_assemble_csr");
  gmls_status r = ensure_order(ctx, nb, "gmls_assemble_csr");
  if (r) return r;
  CsrJob j{nb.order, nb.n_tgt, nb.off, nb.idx, s.w[f], s.rows[f], s.ncomp[f], row_ptr, col, val, nnz_offset};
  CK(launch_csr(ctx->launch(), j), "gmls_assemble_csr");
  return GMLS_OK;
}

gmls_status gmls_assemble_csr(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* row_ptr, int32_t* col,
                              double* val) {
  return gmls_assemble_csr_at(ctx, stencil_id, functional, 0, row_ptr, col, val);
}

// ------------------------------------------------------------ Stokes system
// Validate the two stencil handles of a Stokes system and fill the job's
// inputs; *n_rows = n d + n + 1.
static gmls_status stokes_job(gmls_ctx* ctx, const gmls_stokes_params* p, StokesJob* j, int64_t* n_rows,
                              const char* who) {
  if (!ctx || !p) return GMLS_EINVAL;
  auto iv = ctx->objs.find(p->velocity), ip = ctx->objs.find(p->pressure);
  if (iv == ctx->objs.end() || iv->second.kind != K_STENCIL || ip == ctx->objs.end() ||
      ip->second.kind != K_STENCIL)
    return fail(ctx, GMLS_ENOTFOUND, std::string(who) + ": no such stencil handle");
  const StencilObj& sv = iv->second.s;
  const StencilObj& sp = ip->second.s;
  const int fcc = find_out(sv, GMLS_F_CURLCURL), fg = find_out(sp, GMLS_F_GRAD), fl = find_out(sp, GMLS_F_LAPLACIAN);
  if (sv.basis != GMLS_BASIS_DIVFREE || fcc < 0)
    return fail(ctx, GMLS_EINVAL, std::string(who) + ": velocity handle needs the divergence-free basis with curl curl");
  if (sp.basis != GMLS_BASIS_SCALAR || fg < 0 || fl < 0 || !sp.neumann)
    return fail(ctx, GMLS_EINVAL,
                std::string(who) + ": pressure handle needs the scalar basis with gradient and Laplacian, neumann = 1");
  NbrObj& nv = ctx->objs.at(sv.nbrs).nb;
  NbrObj& np = ctx->objs.at(sp.nbrs).nb;
  if (nv.cloud != np.cloud || !nv.all_targets || !np.all_targets)
    return fail(ctx, GMLS_EINVAL, std::string(who) + ": both stencils must cover every point of one cloud, in order");
  const CloudObj& c = ctx->objs.at(nv.cloud).c;
  if (!c.bflag || !c.normals)
    return fail(ctx, GMLS_EINVAL, std::string(who) + ": the cloud needs boundary flags and normals");
  if ((int64_t)c.n * (c.dim + 1) + 1 >= INT32_MAX)
    return fail(ctx, GMLS_EINVAL, std::string(who) + ": too many unknowns for 32-bit column indices");
  if (!(p->nu >= 0.0)) return fail(ctx, GMLS_EINVAL, std::string(who) + ": nu must be >= 0");
  const StencilObj* ss = nullptr;
  const NbrObj* ns = nullptr;
  int fs = -1;
  if (p->pressure_interior != 0) {
    auto is = ctx->objs.find(p->pressure_interior);
    if (is == ctx->objs.end() || is->second.kind != K_STENCIL)
      return fail(ctx, GMLS_ENOTFOUND, std::string(who) + ": no such stencil handle (pressure_interior)");
    ss = &is->second.s;
    fs = find_out(*ss, GMLS_F_LAPLACIAN);
    if (ss->basis != GMLS_BASIS_STAGGERED || fs < 0)
      return fail(ctx, GMLS_EINVAL, std::string(who) + ": pressure_interior needs the staggered basis with the Laplacian");
    ns = &ctx->objs.at(ss->nbrs).nb;
    if (ns->cloud != nv.cloud || !ns->all_targets)
      return fail(ctx, GMLS_EINVAL,
                  std::string(who) + ": the staggered stencils must cover every point of the same cloud, in order");
  }
  std::memset(j, 0, sizeof(*j));
  j->dim = c.dim;
  j->n = c.n;
  j->nu = p->nu;
  j->off_v = nv.off;
  j->idx_v = nv.idx;
  j->w_cc = sv.w[fcc];
  j->off_p = np.off;
  j->idx_p = np.idx;
  j->w_grad = sp.w[fg];
  j->w_lap = sp.w[fl];
  j->beta = sp.beta;
  j->beta_stride = std::max(sp.L, 1);
  j->beta_col = sp.src[fl];
  j->bflag = c.bflag;
  j->normals = c.normals;
  if (ss) {
    j->off_s = ns->off;
    j->idx_s = ns->idx;
    j->w_stag = ss->w[fs];
  }
  *n_rows = c.n * c.dim + c.n + 1;
  return GMLS_OK;
}

// row lengths and their exclusive scan into row_ptr (n_rows + 1 entries)
static gmls_status stokes_rows(gmls_ctx* ctx, StokesJob& j, int64_t n_rows, int64_t* row_ptr, const char* who) {
  j.row_len = arena_alloc<int32_t>(ctx, n_rows);
  const int64_t se = scan_scratch_elems(n_rows);
  int64_t* scratch = arena_alloc<int64_t>(ctx, se);
  if (!j.row_len || !scratch) {
    ctx->arena.release(j.row_len);
    ctx->arena.release(scratch);
    return fail(ctx, GMLS_ENOMEM, std::string(who) + ": arena exhausted");
  }
  j.row_ptr = row_ptr;
  Launch L = ctx->launch();
  cudaError_t e = launch_stokes_rowlen(L, j);
  if (e == cudaSuccess) e = launch_scan_i64_from_i32(L, j.row_len, row_ptr, n_rows, scratch, se);
  ctx->arena.release(j.row_len);  // stream ordered: later work on this stream runs after these kernels
  ctx->arena.release(scratch);
  j.row_len = nullptr;
  if (e != cudaSuccess) return cuda_fail(ctx, e, who);
  return GMLS_OK;
}

gmls_status gmls_stokes_size(gmls_ctx* ctx, const gmls_stokes_params* p, int64_t* n_rows, int64_t* nnz) {
  StokesJob j;
  int64_t nr = 0;
  gmls_status r = stokes_job(ctx, p, &j, &nr, "gmls_stokes_size");
  if (r) return r;
  if (!n_rows || !nnz) return fail(ctx, GMLS_EINVAL, "gmls_stokes_size: NULL output");
  if (capturing(ctx)) return fail(ctx, GMLS_EBUSY, "gmls_stokes_size reads the device and cannot run during capture");
  CK(cudaSetDevice(ctx->device), "gmls_stokes_size");
  int64_t* rp = arena_alloc<int64_t>(ctx, nr + 1);
  if (!rp) return fail(ctx, GMLS_ENOMEM, "gmls_stokes_size: arena exhausted");
  r = stokes_rows(ctx, j, nr, rp, "gmls_stokes_size");
  if (r) {
    ctx->arena.release(rp);
    return r;
  }
  int64_t total = 0;
  cudaError_t e = cudaMemcpyAsync(&total, rp + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  ctx->arena.release(rp);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmls_stokes_size");
  *n_rows = nr;
  *nnz = total;
  return GMLS_OK;
}

gmls_status gmls_stokes_assemble(gmls_ctx* ctx, const gmls_stokes_params* p, int64_t* row_ptr, int32_t* col,
                                 double* val) {
  StokesJob j;
  int64_t nr = 0;
  gmls_status r = stokes_job(ctx, p, &j, &nr, "gmls_stokes_assemble");
  if (r) return r;
  if (!row_ptr || !col || !val) return fail(ctx, GMLS_EINVAL, "gmls_stokes_assemble: NULL output");
  if (is_host_ptr(row_ptr) || is_host_ptr(col) || is_host_ptr(val))
    return fail(ctx, GMLS_EINVAL, "gmls_stokes_assemble: outputs must be device buffers");
  CK(cudaSetDevice(ctx->device), "gmls_stokes_assemble");
  {
    const StencilObj& sv = ctx->objs.at(p->velocity).s;
    const StencilObj& sp = ctx->objs.at(p->pressure).s;
    NbrObj& nv = ctx->objs.at(sv.nbrs).nb;
    NbrObj& np = ctx->objs.at(sp.nbrs).nb;
    if ((r = ensure_order(ctx, nv, "gmls_stokes_assemble")) || (r = ensure_order(ctx, np, "gmls_stokes_assemble")))
      return r;
    j.order_v = nv.order;
    j.order_p = np.order;
    if (p->pressure_interior != 0) {
      NbrObj& ns = ctx->objs.at(ctx->objs.at(p->pressure_interior).s.nbrs).nb;
      if ((r = ensure_order(ctx, ns, "gmls_stokes_assemble"))) return r;
      j.order_s = ns.order;
    }
  }
  r = stokes_rows(ctx, j, nr, row_ptr, "gmls_stokes_assemble");
  if (r) return r;
  j.col = col;
  j.val = val;
  CK(launch_stokes_fill(ctx->launch(), j), "gmls_stokes_assemble fill");
  return GMLS_OK;
}

gmls_status gmls_stokes_rhs(gmls_ctx* ctx, const gmls_stokes_params* p, const double* f, const double* w,
                            const double* div_f, double* b) {
  StokesJob j;
  int64_t nr = 0;
  gmls_status r = stokes_job(ctx, p, &j, &nr, "gmls_stokes_rhs");
  if (r) return r;
  if (!f || !w || !div_f || !b) return fail(ctx, GMLS_EINVAL, "gmls_stokes_rhs: NULL pointer");
  if (is_host_ptr(f) || is_host_ptr(w) || is_host_ptr(div_f) || is_host_ptr(b))
    return fail(ctx, GMLS_EINVAL, "gmls_stokes_rhs: arrays must be device buffers");
  CK(cudaSetDevice(ctx->device), "gmls_stokes_rhs");
  CK(launch_stokes_rhs(ctx->launch(), j, f, w, div_f, b), "gmls_stokes_rhs");
  return GMLS_OK;
}

gmls_status gmls_csr_spmv(gmls_ctx* ctx, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                          const double* val, const double* x, double* y) {
  if (!ctx) return GMLS_EINVAL;
  if (n_rows < 0 || !row_ptr || !col || !val || !x || !y) return fail(ctx, GMLS_EINVAL, "gmls_csr_spmv: bad argument");
  if (is_host_ptr(row_ptr) || is_host_ptr(col) || is_host_ptr(val) || is_host_ptr(x) || is_host_ptr(y))
    return fail(ctx, GMLS_EINVAL, "gmls_csr_spmv: arrays must be device buffers");
  CK(cudaSetDevice(ctx->device), "gmls_csr_spmv");
  int32_t* long_rows = arena_alloc<int32_t>(ctx, std::max<int64_t>(n_rows, 1));
  int32_t* n_long = arena_alloc<int32_t>(ctx, 1);
  double* partial = arena_alloc<double>(ctx, csr_spmv_partial_elems());
  if (!long_rows || !n_long || !partial) {
    ctx->arena.release(long_rows);
    ctx->arena.release(n_long);
    ctx->arena.release(partial);
    return fail(ctx, GMLS_ENOMEM, "gmls_csr_spmv: arena exhausted");
  }
  cudaError_t e = launch_csr_spmv(ctx->launch(), n_rows, row_ptr, col, val, x, y, long_rows, n_long, partial);
  ctx->arena.release(long_rows);  // stream ordered
  ctx->arena.release(n_long);
  ctx->arena.release(partial);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmls_csr_spmv");
  return GMLS_OK;
}

// ------------------------------------------------------------------- GMRES
// Restarted GMRES(m) with right Jacobi preconditioning, A D^-1 y = b,
// x = D^-1 y (D = diag A, 1 where that is zero).  Arnoldi with classical
// Gram-Schmidt applied twice; the Hessenberg column and the new norm come to
// the host once per iteration, where Givens rotations update the residual
// estimate.  The true residual is recomputed at every restart and at the end.
gmls_status gmls_gmres(gmls_ctx* ctx, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* b, double* x, const gmls_gmres_params* p, int32_t* iters, double* rel_residual) {
  if (!ctx) return GMLS_EINVAL;
  if (!p || n < 1 || !row_ptr || !col || !val || !b || !x || p->restart < 1 || p->restart > 256 || p->max_iter < 0 ||
      !(p->rtol > 0.0) || (p->row_scaling != 0 && p->row_scaling != 1) || p->reserved != 0)
    return fail(ctx, GMLS_EINVAL,
                "gmls_gmres: bad argument (restart 1..256, max_iter >= 0, rtol > 0, row_scaling 0 or 1, reserved 0)");
  if (is_host_ptr(row_ptr) || is_host_ptr(col) || is_host_ptr(val) || is_host_ptr(b) || is_host_ptr(x))
    return fail(ctx, GMLS_EINVAL, "gmls_gmres: arrays must be device buffers");
  if (capturing(ctx)) return fail(ctx, GMLS_EBUSY, "gmls_gmres reads the device every iteration: not during capture");
  CK(cudaSetDevice(ctx->device), "gmls_gmres");
  const int m = p->restart;
  double* V = arena_alloc<double>(ctx, (size_t)(m + 1) * n);
  double* z = arena_alloc<double>(ctx, n);
  double* dinv = arena_alloc<double>(ctx, n);
  double* part = arena_alloc<double>(ctx, krylov_partial_elems(m + 2));
  double* hdev = arena_alloc<double>(ctx, 2 * (m + 2));
  int32_t* long_rows = arena_alloc<int32_t>(ctx, n);
  int32_t* n_long = arena_alloc<int32_t>(ctx, 1);
  double* sp_part = arena_alloc<double>(ctx, csr_spmv_partial_elems());
  const bool rs = p->row_scaling != 0;
  double* rinv = rs ? arena_alloc<double>(ctx, n) : nullptr;
  void* all[] = {V, z, dinv, part, hdev, long_rows, n_long, sp_part, rinv};
  auto release = [&]() {
    for (void* q : all) ctx->arena.release(q);
  };
  const int n_need = rs ? 9 : 8;  // rinv (the last entry) only with row scaling
  for (int i = 0; i < n_need; ++i)
    if (!all[i]) {
      release();
      return fail(ctx, GMLS_ENOMEM, "gmls_gmres: arena exhausted (the basis needs (restart + 1) n doubles)");
    }
  Launch L = ctx->launch();
  cudaError_t e = cudaSuccess;
  auto spmv = [&](const double* in, double* out) {
    if (e == cudaSuccess) e = launch_csr_spmv(L, n, row_ptr, col, val, in, out, long_rows, n_long, sp_part);
  };
  auto dot_host = [&](const double* a, const double* c, double* out_host) {
    if (e == cudaSuccess) e = krylov_dots(L, n, 1, a, c, part, hdev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, hdev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  };
  // with row scaling R (rinv): GMRES on R A D y = R b, x = D y, and the
  // residual norms are those of R (b - A x)
  double bb = 0.0;
  if (rs) {
    if (e == cudaSuccess) e = krylov_row_equilibration(L, n, row_ptr, col, val, rinv, dinv);
    if (e == cudaSuccess) e = krylov_scale(L, n, rinv, b, z);
    dot_host(z, z, &bb);
  } else {
    if (e == cudaSuccess) e = krylov_inverse_diagonal(L, n, row_ptr, col, val, dinv);
    dot_host(b, b, &bb);
  }
  const double bnorm = std::sqrt(bb);
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), hc(2 * (m + 2), 0.0);
  int total = 0;
  double rel = 0.0;
  while (e == cudaSuccess) {
    // r = b - A x into V_0
    spmv(x, V);
    if (e == cudaSuccess) e = krylov_residual(L, n, b, V);
    if (rs && e == cudaSuccess) e = krylov_scale_in_place(L, n, rinv, V);
    double rr = 0.0;
    dot_host(V, V, &rr);
    const double beta = std::sqrt(rr);
    rel = bnorm > 0.0 ? beta / bnorm : beta;
    if (e != cudaSuccess || rel <= p->rtol || total >= p->max_iter || !(beta > 0.0)) break;
    if (e == cudaSuccess) e = krylov_scaled_copy(L, n, V, 1.0 / beta, V);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && total < p->max_iter && e == cudaSuccess; ++j) {
      double* vj = V + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      if (e == cudaSuccess) e = krylov_scale(L, n, dinv, vj, z);
      spmv(z, w);
      if (rs && e == cudaSuccess) e = krylov_scale_in_place(L, n, rinv, w);
      // CGS2: h = V^T w, w -= V h, twice; then |w|
      if (e == cudaSuccess) e = krylov_dots(L, n, j + 1, V, w, part, hdev);
      if (e == cudaSuccess) e = krylov_axpy(L, n, j + 1, V, hdev, w);
      if (e == cudaSuccess) e = krylov_dots(L, n, j + 1, V, w, part, hdev + (m + 2));
      if (e == cudaSuccess) e = krylov_axpy(L, n, j + 1, V, hdev + (m + 2), w);
      if (e == cudaSuccess) e = krylov_dots(L, n, 1, w, w, part, hdev + (m + 2) + (j + 1));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hc.data(), hdev, sizeof(double) * 2 * (m + 2), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) break;
      std::vector<double> h(j + 2);
      for (int i = 0; i <= j; ++i) h[i] = hc[i] + hc[(m + 2) + i];
      const double hn = std::sqrt(std::max(hc[(m + 2) + (j + 1)], 0.0));
      h[j + 1] = hn;
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double r = std::hypot(h[j], h[j + 1]);
      cs[j] = r > 0.0 ? h[j] / r : 1.0;
      sn[j] = r > 0.0 ? h[j + 1] / r : 0.0;
      h[j] = r;
      h[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
      ++total;
      jdone = j + 1;
      if (hn > 0.0 && e == cudaSuccess) e = krylov_scaled_copy(L, n, w, 1.0 / hn, w);
      if (std::fabs(g[j + 1]) <= p->rtol * bnorm || !(hn > 0.0)) break;
    }
    if (e != cudaSuccess || jdone == 0) break;
    // y = H^-1 g (upper triangular), x += D^-1 V y
    std::vector<double> y(jdone);
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < jdone; ++c) s -= H[(size_t)i * m + c] * y[c];
      y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hdev, y.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = krylov_update(L, n, jdone, V, hdev, dinv, x);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // y (host) stays valid until the copy ran
  }
  release();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmls_gmres");
  if (iters) *iters = total;
  if (rel_residual) *rel_residual = rel;
  return GMLS_OK;
}

static gmls_status export_src(gmls_ctx* ctx, int64_t id, int32_t what, int32_t functional, const void** src,
                              size_t* bytes) {
  auto it = ctx->objs.find(id);
  if (it == ctx->objs.end()) return fail(ctx, GMLS_ENOTFOUND, "gmls_export: no such handle");
  Obj& o = it->second;
  if (o.kind == K_NBRS) {
    NbrObj& nb = o.nb;
    switch (what) {
      case GMLS_X_NBR_OFFSETS: *src = nb.off; *bytes = sizeof(int64_t) * (nb.n_tgt + 1); return GMLS_OK;
      case GMLS_X_NBR_INDEX: {
        int64_t tot;
        gmls_status r = nbr_total(ctx, nb, &tot);
        if (r) return r;
        *src = nb.idx;
        *bytes = sizeof(int32_t) * tot;
        return GMLS_OK;
      }
      case GMLS_X_NBR_EPS: *src = nb.eps; *bytes = sizeof(double) * nb.n_tgt; return GMLS_OK;
      case GMLS_X_NBR_STATUS: *src = nb.status; *bytes = nb.n_tgt; return GMLS_OK;
      default: break;
    }
  } else if (o.kind == K_STENCIL) {
    StencilObj& s = o.s;
    NbrObj& nb = ctx->objs.at(s.nbrs).nb;
    switch (what) {
      case GMLS_X_WEIGHTS: {
        int f = find_out(s, functional);
        if (f < 0) return fail(ctx, GMLS_EINVAL, "gmls_export: functional not computed");
        int64_t tot;
        gmls_status r = nbr_total(ctx, nb, &tot);
        if (r) return r;
        *src = s.w[f];
        *bytes = sizeof(double) * tot * s.rows[f] * s.ncomp[f];
        return GMLS_OK;
      }
      case GMLS_X_BETA: *src = s.beta; *bytes = sizeof(double) * nb.n_tgt * std::max(s.L, 1); return GMLS_OK;
      case GMLS_X_STATUS: *src = s.status; *bytes = nb.n_tgt; return GMLS_OK;
      case GMLS_X_ITERS: *src = s.iters; *bytes = nb.n_tgt; return GMLS_OK;
      default: break;
    }
  }
  return fail(ctx, GMLS_EINVAL, "gmls_export: nothing of that kind in this handle");
}

gmls_status gmls_export_size(gmls_ctx* ctx, int64_t id, int32_t what, int32_t functional, size_t* bytes) {
  if (!ctx || !bytes) return GMLS_EINVAL;
  const void* src;
  return export_src(ctx, id, what, functional, &src, bytes);
}

gmls_status gmls_export(gmls_ctx* ctx, int64_t id, int32_t what, int32_t functional, void* dst, size_t bytes) {
  if (!ctx || !dst) return GMLS_EINVAL;
  CK(cudaSetDevice(ctx->device), "gmls_export");
  const void* src;
  size_t need;
  gmls_status r = export_src(ctx, id, what, functional, &src, &need);
  if (r) return r;
  if (bytes < need) return fail(ctx, GMLS_EINVAL, "gmls_export: destination too small");
  if (need == 0) return GMLS_OK;
  CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, ctx->stream), "gmls_export");
  if (is_host_ptr(dst)) CK(cudaStreamSynchronize(ctx->stream), "gmls_export");
  return GMLS_OK;
}

gmls_status gmls_release(gmls_ctx* ctx, int64_t id) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(id);
  if (it == ctx->objs.end()) return fail(ctx, GMLS_ENOTFOUND, "gmls_release: no such handle");
  Obj& o = it->second;
  Arena& a = ctx->arena;
  if (o.kind == K_GRAPH) {
    cudaGraphExecDestroy(o.exec);
  } else if (o.kind == K_CLOUD) {
    if (o.c.refs) return fail(ctx, GMLS_EBUSY, "gmls_release: cloud has live neighbour handles");
    for (void* p : {(void*)o.c.x, (void*)o.c.normals, (void*)o.c.bflag,
                    (void*)o.c.xs, (void*)o.c.xsf, (void*)o.c.sorted, (void*)o.c.cell_start, (void*)o.c.grid})
      a.release(p);
  } else if (o.kind == K_NBRS) {
    if (o.nb.refs) return fail(ctx, GMLS_EBUSY, "gmls_release: neighbours have live stencil handles");
    for (void* p : {(void*)o.nb.tgt, (void*)o.nb.off, (void*)o.nb.idx, (void*)o.nb.eps, (void*)o.nb.status,
                    (void*)o.nb.order})
      a.release(p);
    auto ci = ctx->objs.find(o.nb.cloud);
    if (ci != ctx->objs.end()) ci->second.c.refs--;
  } else {
    for (int f = 0; f < 5; ++f) a.release(o.s.w[f]);
    for (void* p : {(void*)o.s.beta, (void*)o.s.status, (void*)o.s.iters, (void*)o.s.fb_items, (void*)o.s.fb_count})
      a.release(p);
    auto ni = ctx->objs.find(o.s.nbrs);
    if (ni != ctx->objs.end()) ni->second.nb.refs--;
  }
  ctx->objs.erase(it);
  return GMLS_OK;
}

}  // extern "C"
