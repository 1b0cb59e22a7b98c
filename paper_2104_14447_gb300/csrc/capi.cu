// capi.cu -- the C ABI of libgmls (declared in include/gmls.h): context,
// arena allocator, handles, argument checking and launch orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "basis_tables.cuh"
#include "gmls_internal.cuh"

using namespace gmls;

namespace {

// First-fit allocator over the caller's device buffer.  256-byte granularity;
// neighbouring free blocks are merged on release.  Frees are stream ordered
// with the context's single stream, so a block can be reused by later work on
// that stream as soon as it is released.
class Arena {
 public:
  void init(void* base, size_t bytes) {
    uintptr_t b = reinterpret_cast<uintptr_t>(base);
    uintptr_t a = (b + 255) & ~uintptr_t(255);
    base_ = reinterpret_cast<char*>(a);
    cap_ = (bytes > (a - b)) ? ((bytes - (a - b)) & ~size_t(255)) : 0;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
    used_ = peak_ = 0;
  }
  void* alloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        size_t off = it->first, sz = it->second;
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
  void release(void* p) {
    if (!p) return;
    size_t off = static_cast<char*>(p) - base_;
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

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_, live_;
};

enum Kind { K_CLOUD = 1, K_NBRS = 2, K_STENCIL = 3 };

struct CloudObj {
  int dim = 0;
  int64_t n = 0;
  double* x = nullptr;
  float* xh = nullptr;  // float-float split of x
  float* xl = nullptr;
  double* normals = nullptr;
  uint8_t* bflag = nullptr;
  double* xs = nullptr;
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
  int64_t idx_cap = 0;  // allocated index entries
  int refs = 0;
};

struct StencilObj {
  int64_t nbrs = 0;
  int basis = 0, dim = 0, L = 0;
  int nout = 0;
  int fn[5], rows[5], ncomp[5];
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
};

std::string g_create_error;

}  // namespace

namespace gmls {
// last error of a call made without a context (see gmls_last_error(NULL))
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gmls

struct gmls_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Arena arena;
  std::unordered_map<int64_t, Obj> objs;
  int64_t next_id = 1;
  int64_t launches = 0;
  bool force_generic = false;  // testing: use the generic tile kernel for every shape
  std::string err;
  Launch launch() { return Launch{stream, &launches}; }
};

static gmls_status fail(gmls_ctx* c, gmls_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static gmls_status cuda_fail(gmls_ctx* c, cudaError_t e, const char* where) {
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
    default: return fail(ctx, GMLS_EINVAL, "gmls_set_option: unknown option");
  }
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
  c.xh = arena_alloc<float>(ctx, (size_t)dim * n);
  c.xl = arena_alloc<float>(ctx, (size_t)dim * n);
  c.xs = arena_alloc<double>(ctx, (size_t)dim * n);
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
  void* all[] = {c.x, c.xh, c.xl, c.xs, c.sorted, c.cell_start, c.grid, part, cell_of, counts, fill, scan_tmp};
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
  CK(launch_split_ff(L, c.x, c.xh, c.xl, (int64_t)dim * n), "gmls_cloud split");
  CK(launch_bbox_and_grid(L, dim, n, c.x, nc_axis, c.grid, part, n_part), "gmls_cloud bbox");
  CK(launch_cell_count(L, dim, n, c.x, c.grid, cell_of, counts), "gmls_cloud count");
  CK(launch_scan_i32(L, counts, c.cell_start, ncell, scan_tmp, scan_elems), "gmls_cloud scan");
  CK(launch_cell_scatter(L, dim, n, c.x, cell_of, c.cell_start, fill, c.sorted, c.xs), "gmls_cloud scatter");
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
  nb.idx_cap = nt * (int64_t)nb.cap;
  nb.tgt = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
  nb.off = arena_alloc<int64_t>(ctx, nt + 1);
  nb.idx = arena_alloc<int32_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
  nb.eps = arena_alloc<double>(ctx, std::max<int64_t>(nt, 1));
  nb.status = arena_alloc<uint8_t>(ctx, std::max<int64_t>(nt, 1));
  double* hs = p->halfspace ? arena_alloc<double>(ctx, (size_t)nt * c.dim) : nullptr;
  int32_t* padded = nullptr;
  int32_t* cnt = nullptr;
  int64_t* scan_tmp = nullptr;
  int64_t scan_elems = 0;
  if (p->mode == GMLS_NBR_RADIUS) {
    padded = arena_alloc<int32_t>(ctx, std::max<int64_t>(nb.idx_cap, 1));
    cnt = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
    scan_elems = scan_scratch_elems(nt);
    scan_tmp = arena_alloc<int64_t>(ctx, scan_elems);
  }
  bool oom = !nb.tgt || !nb.off || !nb.idx || !nb.eps || !nb.status || (p->halfspace && !hs) ||
             (p->mode == GMLS_NBR_RADIUS && (!padded || !cnt || !scan_tmp));
  if (oom) {
    for (void* q : {(void*)nb.tgt, (void*)nb.off, (void*)nb.idx, (void*)nb.eps, (void*)nb.status, (void*)hs,
                    (void*)padded, (void*)cnt, (void*)scan_tmp})
      ctx->arena.release(q);
    return fail(ctx, GMLS_ENOMEM, "gmls_neighbors: arena exhausted");
  }
  Launch L = ctx->launch();
  if (p->targets)
    CK(copy_in(ctx, nb.tgt, p->targets, sizeof(int32_t) * nt), "gmls_neighbors copy targets");
  else
    CK(launch_fill_identity(L, nb.tgt, nt), "gmls_neighbors identity");
  if (hs) CK(copy_in(ctx, hs, p->halfspace, sizeof(double) * nt * c.dim), "gmls_neighbors copy halfspace");
  NbrQuery q;
  q.cloud = CloudDev{c.dim, c.n, c.x, c.xs, c.sorted, c.cell_start, c.grid, c.ncell};
  q.n_tgt = nt;
  q.tgt = nb.tgt;
  q.halfspace = hs;
  q.mode = p->mode;
  q.k = p->k;
  q.cap = nb.cap;
  q.eps_factor = p->eps_factor;
  q.out_idx = (p->mode == GMLS_NBR_RADIUS) ? padded : nb.idx;
  q.out_cnt = cnt;
  q.out_eps = nb.eps;
  q.out_status = nb.status;
  CK(launch_nbr_query(L, q), "gmls_neighbors query");
  if (p->mode == GMLS_NBR_KNN) {
    CK(launch_fill_offsets_fixed(L, nb.off, nt, p->k), "gmls_neighbors offsets");
  } else {
    CK(launch_scan_i64_from_i32(L, cnt, nb.off, nt, scan_tmp, scan_elems), "gmls_neighbors scan");
    CK(launch_compact_padded(L, padded, nb.cap, cnt, nb.off, nb.idx, nt), "gmls_neighbors compact");
  }
  ctx->arena.release(hs);
  ctx->arena.release(padded);
  ctx->arena.release(cnt);
  ctx->arena.release(scan_tmp);
  c.refs++;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *nbrs_id = id;
  return GMLS_OK;
}

// rows / components of one functional's output
static bool functional_shape(int basis, int dim, int fn, int* rows, int* ncomp) {
  switch (fn) {
    case GMLS_F_GRAD:
      if (basis != GMLS_BASIS_SCALAR) return false;
      *rows = dim, *ncomp = 1;
      return true;
    case GMLS_F_LAPLACIAN:
      if (basis != GMLS_BASIS_SCALAR) return false;
      *rows = 1, *ncomp = 1;
      return true;
    case GMLS_F_DIV:
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
  if (p->basis != GMLS_BASIS_SCALAR && p->basis != GMLS_BASIS_DIVFREE)
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
  const int nc = (p->basis == GMLS_BASIS_SCALAR) ? 1 : dim;
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
    s.fb_items = arena_alloc<int32_t>(ctx, std::max<int64_t>(nt, 1));
    s.fb_count = arena_alloc<int32_t>(ctx, 1);
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

  j.dim = dim;
  j.n = c.n;
  j.x = c.x;
  j.xh = c.xh;
  j.xl = c.xl;
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
  j.beta = s.beta;
  j.status = s.status;
  j.iters = s.iters;
  j.max_refine = p->max_refine > 0 ? p->max_refine : 3;
  j.tol = p->refine_tol > 0.0 ? p->refine_tol : 1e-12;
  j.fb_items = s.fb_items;
  j.fb_count = s.fb_count;
  j.ld = ld;
  j.nmax = nmax;

  // warps per target: the smallest of 1, 2, 4 that fits and keeps lanes busy
  auto pick_g = [&](bool fp32) -> int {
    int g0 = ld <= 64 ? 1 : (ld <= 192 ? 2 : 4);
    for (int g = g0; g <= 4; g *= 2) {
      j.warps_per_target = g;
      if (stencil_smem_bytes(j, fp32) <= 227 * 1024) return g;
    }
    return 0;
  };
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  Launch Lc = ctx->launch();
  const int g_main = pick_g(refine);
  if (!g_main) {
    release_all();
    return fail(ctx, GMLS_EINVAL, "gmls_stencils: tile does not fit in shared memory for this (k, basis, degree)");
  }
  j.warps_per_target = g_main;
  auto grid_for = [&](bool fp32, int64_t items) -> int {
    const size_t smem = stencil_smem_bytes(j, fp32);
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(16, (228 * 1024) / (smem + 1024)));
    int64_t groups = (int64_t)(128 / (32 * j.warps_per_target));
    int64_t want = (items + groups - 1) / groups;
    int64_t cap = (int64_t)dev_sms * per_sm;
    return (int)std::max<int64_t>(1, std::min(want, cap));
  };
  if (refine) CK(cudaMemsetAsync(s.fb_count, 0, sizeof(int32_t), ctx->stream), "gmls_stencils memset");
  // the warp-per-target float-float kernel when this shape is instantiated
  int mr = 0;
  const bool fast = refine && !p->degree_per_target && (p->weight_power % 2 == 0) && !ctx->force_generic &&
                    fast_path_available(p->basis, dim, p->degree, ld, &mr);
  if (nt > 0) {
    if (fast)
      CK(launch_stencils_fast(Lc, j, mr, dev_sms), "gmls_stencils fast launch");
    else
      CK(launch_stencils(Lc, j, refine, grid_for(refine, nt)), "gmls_stencils launch");
    if (refine) {
      StencilJob jf = j;
      jf.items = s.fb_items;
      jf.n_items = s.fb_count;
      jf.fallback_run = 1;
      int gf = 0;
      for (int g = (ld <= 64 ? 1 : (ld <= 192 ? 2 : 4)); g <= 4; g *= 2) {
        jf.warps_per_target = g;
        if (stencil_smem_bytes(jf, false) <= 227 * 1024) {
          gf = g;
          break;
        }
      }
      if (gf) {
        jf.warps_per_target = gf;
        CK(launch_stencils(Lc, jf, false, dev_sms * 2), "gmls_stencils fallback launch");
      }
    }
  }
  ctx->arena.release(deg);
  nb.refs++;
  int64_t id = ctx->next_id++;
  ctx->objs.emplace(id, std::move(o));
  *stencil_id = id;
  return GMLS_OK;
}

static int find_out(const StencilObj& s, int fn) {
  for (int f = 0; f < s.nout; ++f)
    if (s.fn[f] == fn) return f;
  return -1;
}

// total neighbour entries (reads the device offset when the lists are variable)
static gmls_status nbr_total(gmls_ctx* ctx, const NbrObj& nb, int64_t* total) {
  if (nb.mode == GMLS_NBR_KNN) {
    *total = nb.n_tgt * (int64_t)nb.k;
    return GMLS_OK;
  }
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

gmls_status gmls_assemble_csr(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* row_ptr, int32_t* col,
                              double* val) {
  if (!ctx) return GMLS_EINVAL;
  auto it = ctx->objs.find(stencil_id);
  if (it == ctx->objs.end() || it->second.kind != K_STENCIL) return fail(ctx, GMLS_ENOTFOUND, "gmls_assemble_csr: no such stencil handle");
  if (!row_ptr || !col || !val) return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: NULL output");
  StencilObj& s = it->second.s;
  int f = find_out(s, functional);
  if (f < 0) return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: functional not computed");
  if (is_host_ptr(row_ptr) || is_host_ptr(col) || is_host_ptr(val))
    return fail(ctx, GMLS_EINVAL, "gmls_assemble_csr: outputs must be device buffers");
  NbrObj& nb = ctx->objs.at(s.nbrs).nb;
  CK(cudaSetDevice(ctx->device), "gmls_assemble_csr");
  CsrJob j{nb.n_tgt, nb.off, nb.idx, s.w[f], s.rows[f], s.ncomp[f], row_ptr, col, val};
  CK(launch_csr(ctx->launch(), j), "gmls_assemble_csr");
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
  if (o.kind == K_CLOUD) {
    if (o.c.refs) return fail(ctx, GMLS_EBUSY, "gmls_release: cloud has live neighbour handles");
    for (void* p : {(void*)o.c.x, (void*)o.c.xh, (void*)o.c.xl, (void*)o.c.normals, (void*)o.c.bflag,
                    (void*)o.c.xs, (void*)o.c.sorted, (void*)o.c.cell_start, (void*)o.c.grid})
      a.release(p);
  } else if (o.kind == K_NBRS) {
    if (o.nb.refs) return fail(ctx, GMLS_EBUSY, "gmls_release: neighbours have live stencil handles");
    for (void* p : {(void*)o.nb.tgt, (void*)o.nb.off, (void*)o.nb.idx, (void*)o.nb.eps, (void*)o.nb.status}) a.release(p);
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
