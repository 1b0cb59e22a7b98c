// nbr.cu -- cell-list build and exact neighbour queries on the device.
//
// The paper gathers, for each target x_T, the particles within the support
// radius eps (Sec. 2.1, the set N_T under Eq. optimization-discretized-4) with
// a kd-tree; here a uniform cell list on the GPU replaces the tree.  Queries
// are exact: squared distances are FP64 with every operation rounded
// separately, and lists are ordered by (d^2, particle id), so the result is
// identical on every run and machine.
#include <cuda_runtime.h>

#include <atomic>

#include "gmls_internal.cuh"

namespace gmls {

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (dev < 0 || dev >= 64) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// grid-stride launches: at most 32 blocks per SM
static inline unsigned blocks_for(int64_t n, int per_block, int per_sm = 32) {
  int64_t b = (n + per_block - 1) / per_block;
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------- bounding box
__global__ void bbox_partial_kernel(int dim, int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double smin[3][8], smax[3][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < dim; ++c) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      double v = x[c * n + i];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      smin[c][warp] = lo;
      smax[c][warp] = hi;
    }
  }
  __syncthreads();
  if (threadIdx.x < dim) {
    int c = threadIdx.x;
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, smin[c][w]);
      hi = fmax(hi, smax[c][w]);
    }
    part[(blockIdx.x * 3 + c) * 2 + 0] = lo;
    part[(blockIdx.x * 3 + c) * 2 + 1] = hi;
  }
}

__global__ void grid_finalize_kernel(int dim, int nparts, const double* __restrict__ part, int nc0, int nc1, int nc2,
                                     GridParams* __restrict__ g) {
  // one warp: the lanes reduce the block partials (min / max are exact, so
  // the order does not matter), lane 0 writes the grid
  const int lane = threadIdx.x & 31;
  double lo3[3], hi3[3];
  for (int c = 0; c < kMaxDim; ++c) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    if (c < dim)
      for (int p = lane; p < nparts; p += 32) {
        lo = fmin(lo, part[(p * 3 + c) * 2 + 0]);
        hi = fmax(hi, part[(p * 3 + c) * 2 + 1]);
      }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    lo3[c] = lo;
    hi3[c] = hi;
  }
  if (lane != 0) return;
  int ncs[3] = {nc0, nc1, nc2};
  double vol = 1.0;
  for (int c = 0; c < kMaxDim; ++c) {
    if (c >= dim) {
      g->lo[c] = 0.0;
      g->org[c] = 0.0;
      g->h[c] = 1.0;
      g->inv_h[c] = 0.0;
      g->nc[c] = 1;
      continue;
    }
    const double lo = lo3[c], hi = hi3[c];
    g->org[c] = 0.5 * lo + 0.5 * hi;
    double ext = hi - lo;
    int nc = ncs[c];
    if (!(ext > 0.0)) {  // flat axis: one cell, every point maps to it
      nc = 1;
      g->lo[c] = lo;
      g->h[c] = 1.0;
      g->inv_h[c] = 0.0;
      g->nc[c] = 1;
      continue;
    }
    g->lo[c] = lo;
    g->h[c] = ext / nc;
    g->inv_h[c] = nc / ext;
    g->nc[c] = nc;
    vol *= ext;
  }
  g->volume = vol;
}

cudaError_t launch_bbox_and_grid(const Launch& L, int dim, int64_t n, const double* x, const int32_t nc_axis[3],
                                 GridParams* grid, double* part, int n_partials) {
  bbox_partial_kernel<<<n_partials, 256, 0, L.stream>>>(dim, n, x, part);
  grid_finalize_kernel<<<1, 32, 0, L.stream>>>(dim, n_partials, part, nc_axis[0], nc_axis[1], nc_axis[2], grid);
  *L.counter += 2;
  return cudaGetLastError();
}

__device__ __forceinline__ int32_t cell_coord(const GridParams& g, int c, double v) {
  double f = floor((v - g.lo[c]) * g.inv_h[c]);
  int32_t q = (f < 0.0) ? 0 : (f >= (double)g.nc[c] ? g.nc[c] - 1 : (int32_t)f);
  return q;
}

__global__ void cell_count_kernel(int dim, int64_t n, const double* __restrict__ x, const GridParams* __restrict__ gp,
                                  int32_t* __restrict__ cell_of, int32_t* __restrict__ counts) {
  const GridParams g = *gp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t cell = 0;
    for (int c = dim - 1; c >= 0; --c) cell = cell * g.nc[c] + cell_coord(g, c, x[c * n + i]);
    cell_of[i] = cell;
    atomicAdd(&counts[cell], 1);
  }
}

cudaError_t launch_cell_count(const Launch& L, int dim, int64_t n, const double* x, const GridParams* grid,
                              int32_t* cell_of, int32_t* counts) {
  cell_count_kernel<<<blocks_for(n, 256), 256, 0, L.stream>>>(dim, n, x, grid, cell_of, counts);
  *L.counter += 1;
  return cudaGetLastError();
}

// xsf holds the FP32 rounding of the coordinates relative to the bounding-box
// centre, so that the pre-filter's rounding bound scales with the cloud's
// extent, not with its distance from the coordinate origin
__global__ void cell_scatter_kernel(int dim, int64_t n, const double* __restrict__ x, const GridParams* __restrict__ gp,
                                    const int32_t* __restrict__ cell_of, const int32_t* __restrict__ cell_start,
                                    int32_t* __restrict__ fill, int32_t* __restrict__ sorted, double* __restrict__ xs,
                                    float* __restrict__ xsf) {
  double org[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < dim; ++c) org[c] = gp->org[c];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t cell = cell_of[i];
    int32_t pos = cell_start[cell] + atomicAdd(&fill[cell], 1);
    sorted[pos] = (int32_t)i;
    for (int c = 0; c < dim; ++c) {
      const double v = x[c * n + i];
      xs[c * n + pos] = v;
      xsf[c * n + pos] = __double2float_rn(__dsub_rn(v, org[c]));
    }
  }
}

cudaError_t launch_cell_scatter(const Launch& L, int dim, int64_t n, const double* x, const GridParams* grid,
                                const int32_t* cell_of, const int32_t* cell_start, int32_t* fill, int32_t* sorted,
                                double* xs, float* xsf) {
  cell_scatter_kernel<<<blocks_for(n, 256), 256, 0, L.stream>>>(dim, n, x, grid, cell_of, cell_start, fill, sorted,
                                                                xs, xsf);
  *L.counter += 1;
  return cudaGetLastError();
}


// ----------------------------------------------------------------------- scan
// Exclusive scan in three passes: tile sums, a one-block scan of the tile
// sums, then each tile rescanned with its offset.  out has n + 1 entries;
// out[n] is the total.
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kScanThreads * kScanPerThread;

int64_t scan_scratch_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <typename TO>
__device__ __forceinline__ TO block_exclusive_scan(TO v, TO* warp_sums, TO* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TO incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    TO t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    TO s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : TO(0);
    TO si = s;
    for (int o = 1; o < 32; o <<= 1) {
      TO t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  TO r = warp_sums[warp] + incl - v;
  __syncthreads();
  return r;
}

template <typename TI, typename TO>
__global__ void scan_tile_sums_kernel(const TI* __restrict__ in, int64_t n, TO* __restrict__ sums) {
  __shared__ TO ws[32];
  __shared__ TO tot;
  int64_t base = blockIdx.x * (int64_t)kScanTile;
  TO s = 0;
  for (int i = 0; i < kScanPerThread; ++i) {
    int64_t p = base + (int64_t)threadIdx.x * kScanPerThread + i;
    if (p < n) s += (TO)in[p];
  }
  block_exclusive_scan<TO>(s, ws, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename TO>
__global__ void scan_sums_kernel(TO* __restrict__ sums, int64_t nt) {
  __shared__ TO ws[32];
  __shared__ TO tot;
  TO carry = 0;
  for (int64_t base = 0; base < nt; base += blockDim.x) {
    int64_t p = base + threadIdx.x;
    TO v = (p < nt) ? sums[p] : TO(0);
    TO ex = block_exclusive_scan<TO>(v, ws, &tot);
    if (p < nt) sums[p] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nt] = carry;
}

template <typename TI, typename TO>
__global__ void scan_apply_kernel(const TI* __restrict__ in, int64_t n, const TO* __restrict__ sums, TO* __restrict__ out,
                                  int64_t nt) {
  __shared__ TO ws[32];
  __shared__ TO tot;
  int64_t base = blockIdx.x * (int64_t)kScanTile;
  TI v[kScanPerThread];
  TO s = 0;
  for (int i = 0; i < kScanPerThread; ++i) {
    int64_t p = base + (int64_t)threadIdx.x * kScanPerThread + i;
    v[i] = (p < n) ? in[p] : TI(0);
    s += (TO)v[i];
  }
  TO ex = block_exclusive_scan<TO>(s, ws, &tot) + sums[blockIdx.x];
  for (int i = 0; i < kScanPerThread; ++i) {
    int64_t p = base + (int64_t)threadIdx.x * kScanPerThread + i;
    if (p < n) out[p] = ex;
    ex += (TO)v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nt];
}

template <typename TI, typename TO>
static cudaError_t scan_impl(const Launch& L, const TI* in, TO* out, int64_t n, TO* scratch, int64_t scratch_elems) {
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt + 1 > scratch_elems) return cudaErrorInvalidValue;
  if (nt == 0) {
    cudaMemsetAsync(out, 0, sizeof(TO), L.stream);
    return cudaGetLastError();
  }
  scan_tile_sums_kernel<TI, TO><<<(unsigned)nt, kScanThreads, 0, L.stream>>>(in, n, scratch);
  scan_sums_kernel<TO><<<1, 1024, 0, L.stream>>>(scratch, nt);
  scan_apply_kernel<TI, TO><<<(unsigned)nt, kScanThreads, 0, L.stream>>>(in, n, scratch, out, nt);
  *L.counter += 3;
  return cudaGetLastError();
}

cudaError_t launch_scan_i32(const Launch& L, const int32_t* in, int32_t* out, int64_t n, int32_t* scratch,
                            int64_t scratch_elems) {
  return scan_impl<int32_t, int32_t>(L, in, out, n, scratch, scratch_elems);
}
cudaError_t launch_scan_i64_from_i32(const Launch& L, const int32_t* in, int64_t* out, int64_t n, int64_t* scratch,
                                     int64_t scratch_elems) {
  return scan_impl<int32_t, int64_t>(L, in, out, n, scratch, scratch_elems);
}

// ------------------------------------------------------------- neighbour query
constexpr int kQueryWarps = 4;

// Per-warp candidate buffer in shared memory: cap entries of (d2, id) plus the
// row table of the current cell rows.  cap is a power of two chosen per launch
// (about twice k for k-nearest queries), so small k keeps many warps resident.
struct WarpBuf {
  double* d2;
  int32_t* id;
  int32_t* row_begin;
  int32_t* row_end;  // inclusive scan of row lengths
  int cap;
};

__host__ __device__ inline size_t warpbuf_bytes(int cap) { return (size_t)cap * 12 + 256; }

__device__ inline WarpBuf warpbuf_at(unsigned char* base, int cap) {
  WarpBuf w;
  w.d2 = reinterpret_cast<double*>(base);
  w.id = reinterpret_cast<int32_t*>(base + (size_t)cap * 8);
  w.row_begin = reinterpret_cast<int32_t*>(base + (size_t)cap * 12);
  w.row_end = w.row_begin + 32;
  w.cap = cap;
  return w;
}

// Query-side grid constants in FP32, derived once per warp from the FP64 grid.
// FP32 view of the grid in coordinates relative to the bounding-box centre
// (the frame of the pre-filter copies xsf)
struct QueryGeo {
  float lo[3], inv_h[3];
  int32_t nc[3];
  float A;   // >= max |coordinate - centre| over the grid box
  float e2;  // 2 * 2^-23 * A: twice the bound on |fl32(x_j) - fl32(x_T) - (x_j - x_T)|
};

__device__ inline QueryGeo make_query_geo(const GridParams& g, int dim) {
  QueryGeo q;
  double a = 0.0;
  for (int c = 0; c < 3; ++c) {
    q.lo[c] = 0.0f;
    q.inv_h[c] = 0.0f;
    q.nc[c] = 1;
  }
  for (int c = 0; c < dim; ++c) {
    q.lo[c] = __double2float_rn(g.lo[c] - g.org[c]);
    q.inv_h[c] = __double2float_rn(g.inv_h[c]);
    q.nc[c] = g.nc[c];
    a = fmax(a, fmax(fabs(g.lo[c] - g.org[c]), fabs(g.lo[c] + g.h[c] * g.nc[c] - g.org[c])));
  }
  q.A = __double2float_ru(a) * (1.0f + 0x1p-20f);
  q.e2 = q.A * 0x1p-22f;
  return q;
}

// Cells [lo, hi] on axis c that can hold a point with |x_c - x_T,c| <= Rbox.
// The FP32 cell coordinates get a margin far above their rounding error (and
// that of the FP64 cell assignment), so the box is never too small.
__device__ __forceinline__ void cell_range(const QueryGeo& q, int c, float xt, float Rbox, int& lo, int& hi) {
  const float m = fmaf((q.A + Rbox) * q.inv_h[c], 0x1p-19f, 0x1p-19f);
  const float u = (xt - Rbox - q.lo[c]) * q.inv_h[c] - m;
  const float v = (xt + Rbox - q.lo[c]) * q.inv_h[c] + m;
  const float top = (float)(q.nc[c] - 1);
  lo = (u > 0.0f) ? (u < top ? (int)floorf(u) : q.nc[c] - 1) : 0;
  hi = (v < top) ? (v > 0.0f ? (int)floorf(v) : 0) : q.nc[c] - 1;
}

// Row table of the cell rows [r0, r0 + 32) of the box: per lane the first
// cell-order position of its row and the inclusive scan of row lengths.
// Returns the number of positions in these rows.
__device__ __forceinline__ int32_t load_rows(const CloudDev& cl, const GridParams& g, const int* lo, const int* hi,
                                             int ny, int nrows, int r0, WarpBuf& wb) {
  const int lane = threadIdx.x & 31;
  const int r = r0 + lane;
  int32_t b = 0, len = 0;
  if (r < nrows) {
    int cy = lo[1] + r % ny, cz = lo[2] + r / ny;
    int32_t row_cell = (cz * g.nc[1] + cy) * g.nc[0];
    b = cl.cell_start[row_cell + lo[0]];
    len = cl.cell_start[row_cell + hi[0] + 1] - b;
  }
  int32_t incl = len;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  wb.row_begin[lane] = b;
  wb.row_end[lane] = incl;
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
}

// cell-order position of entry p of the loaded rows
__device__ __forceinline__ int64_t row_position(const WarpBuf& wb, int32_t p) {
  int lo_r = 0, hi_r = 31;
  while (lo_r < hi_r) {
    int mid = (lo_r + hi_r) >> 1;
    if (wb.row_end[mid] > p) hi_r = mid; else lo_r = mid + 1;
  }
  const int32_t start = lo_r ? wb.row_end[lo_r - 1] : 0;
  return wb.row_begin[lo_r] + (p - start);
}

// the cell box covers every cell of the grid
template <int D>
__device__ __forceinline__ bool box_is_whole_grid(const GridParams& g, const int* lo, const int* hi) {
  for (int c = 0; c < D; ++c)
    if (lo[c] != 0 || hi[c] != g.nc[c] - 1) return false;
  return true;
}

// Every particle with exact FP64 d2 < R2 (and on the kept side of the
// half-space) from the cells of the box, computing d2 for every particle in
// the box.  Returns the number that passed (may exceed wb.cap: overflow).
template <int D>
__device__ int gather_exact(const CloudDev& cl, const GridParams& g, const int* lo, const int* hi, const double* xT,
                            double R2, bool use_hs, const double* nrm, WarpBuf& wb) {
  const int lane = threadIdx.x & 31;
  constexpr int dim = D;
  const int ny = hi[1] - lo[1] + 1;
  const int nrows = ny * (hi[2] - lo[2] + 1);
  int count = 0;
  if (box_is_whole_grid<D>(g, lo, hi)) {
    for (int64_t p0 = 0; p0 < cl.n; p0 += 32) {
      const int64_t pos = p0 + lane;
      bool pass = false;
      int32_t j = 0;
      double d2 = 0.0;
      if (pos < cl.n) {
        double dx[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; ++c) dx[c] = __dsub_rn(cl.xs[c * cl.n + pos], xT[c]);
        d2 = exact_d2(dim, dx);
        pass = nonneg_less(d2, R2);
        if (pass && use_hs) pass = nonpositive(exact_dot(dim, nrm, dx));
        j = cl.sorted[pos];
      }
      unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        int slot = count + __popc(m & ((1u << lane) - 1u));
        if (slot < wb.cap) {
          wb.d2[slot] = d2;
          wb.id[slot] = j;
        }
      }
      count += __popc(m);
    }
    return count;
  }
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    const int32_t total = load_rows(cl, g, lo, hi, ny, nrows, r0, wb);
    for (int32_t p0 = 0; p0 < total; p0 += 32) {
      const int32_t p = p0 + lane;
      bool pass = false;
      int32_t j = 0;
      double d2 = 0.0;
      if (p < total) {
        const int64_t pos = row_position(wb, p);
        double dx[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; ++c) dx[c] = __dsub_rn(cl.xs[c * cl.n + pos], xT[c]);
        d2 = exact_d2(dim, dx);
        pass = nonneg_less(d2, R2);
        if (pass && use_hs) pass = nonpositive(exact_dot(dim, nrm, dx));
        j = cl.sorted[pos];
      }
      unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        int slot = count + __popc(m & ((1u << lane) - 1u));
        if (slot < wb.cap) {
          wb.d2[slot] = d2;
          wb.id[slot] = j;
        }
      }
      count += __popc(m);
    }
    __syncwarp();
  }
  return count;
}

// Collect every particle with exact FP64 d2 < R2 (after the optional
// half-space filter) into the warp's buffer.  The box of cells covers
// |x_c - x_T,c| <= Rbox, Rbox >= sqrt(R2).  A first pass tests each
// particle of the box in FP32 against a bound that no particle inside
// sqrt(R2) can exceed (rounding of the float coordinates and of the FP32 sum
// included) and compacts the survivors; only those get the exact FP64 d2, so
// the FP64 pipe sees about the ball's share of the box.  If the survivors do
// not fit the buffer the box is searched again with exact distances only.
// Returns the number that passed (may exceed wb.cap: overflow).
// The half-space filter is applied in the FP32 pass too (kept side
// n . dx <= 0): with unit-roundoff u = 2^-24, the float coordinates, their
// difference, the float normal and the float dot product together err by at
// most |n|_1 2^-23 (max_c |x_T,c| + 4 Rbox), so the pass keeps every particle
// whose float dot product is at most 8 times that bound (hs_scale is
// |n|_1 2^-20) and the exact test decides.
template <int D>
__device__ int gather_candidates(const CloudDev& cl, const GridParams& g, const QueryGeo& gq, const double* xT,
                                 const float* xTf, float Rbox, double R2, bool use_hs, const double* nrm,
                                 const float* nrmf, float hs_scale, WarpBuf& wb) {
  const int lane = threadIdx.x & 31;
  constexpr int dim = D;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int c = 0; c < dim; ++c) cell_range(gq, c, xTf[c], Rbox, lo[c], hi[c]);
  const int ny = hi[1] - lo[1] + 1;
  const int nrows = ny * (hi[2] - lo[2] + 1);
  float bf = Rbox + gq.e2;
  bf = bf * bf * (1.0f + 0x1p-19f);
  float xmax = 0.0f;
  for (int c = 0; c < dim; ++c) xmax = fmaxf(xmax, fabsf(xTf[c]));
  const float hs_tol = hs_scale * (xmax + 4.0f * Rbox);
  // pass 1: FP32 pre-filter, positions of the survivors into wb.id
  int staged = 0;
  if (box_is_whole_grid<D>(g, lo, hi)) {
    // every particle: the cell-ordered arrays in one coalesced sweep
    for (int64_t p0 = 0; p0 < cl.n; p0 += 32) {
      const int64_t pos = p0 + lane;
      bool pass = false;
      if (pos < cl.n) {
        float d2f = 0.0f, dotf = 0.0f;
        for (int c = 0; c < dim; ++c) {
          const float dxf = cl.xsf[c * cl.n + pos] - xTf[c];
          d2f = fmaf(dxf, dxf, d2f);
          dotf = fmaf(nrmf[c], dxf, dotf);
        }
        pass = d2f <= bf && (!use_hs || dotf <= hs_tol);
      }
      unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        int slot = staged + __popc(m & ((1u << lane) - 1u));
        if (slot < wb.cap) wb.id[slot] = (int32_t)pos;
      }
      staged += __popc(m);
    }
  }
  for (int r0 = 0; r0 < (box_is_whole_grid<D>(g, lo, hi) ? 0 : nrows); r0 += 32) {
    const int32_t total = load_rows(cl, g, lo, hi, ny, nrows, r0, wb);
    for (int32_t p0 = 0; p0 < total; p0 += 32) {
      const int32_t p = p0 + lane;
      bool pass = false;
      int32_t pos = 0;
      if (p < total) {
        pos = (int32_t)row_position(wb, p);
        float d2f = 0.0f, dotf = 0.0f;
        for (int c = 0; c < dim; ++c) {
          const float dxf = cl.xsf[c * cl.n + pos] - xTf[c];
          d2f = fmaf(dxf, dxf, d2f);
          dotf = fmaf(nrmf[c], dxf, dotf);
        }
        pass = d2f <= bf && (!use_hs || dotf <= hs_tol);
      }
      unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        int slot = staged + __popc(m & ((1u << lane) - 1u));
        if (slot < wb.cap) wb.id[slot] = pos;
      }
      staged += __popc(m);
    }
    __syncwarp();
  }
  if (staged > wb.cap) return gather_exact<D>(cl, g, lo, hi, xT, R2, use_hs, nrm, wb);
  // pass 2: exact FP64 distances of the survivors, compacted in place (an
  // entry moves to a slot at or below its own, and each round's reads finish
  // before its writes)
  int count = 0;
  for (int i0 = 0; i0 < staged; i0 += 32) {
    const int i = i0 + lane;
    const int32_t pos = (i < staged) ? wb.id[i] : 0;
    __syncwarp();
    bool pass = false;
    double d2 = 0.0;
    if (i < staged) {
      double dx[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < dim; ++c) dx[c] = __dsub_rn(cl.xs[c * cl.n + pos], xT[c]);
      d2 = exact_d2(dim, dx);
      pass = nonneg_less(d2, R2);
      if (pass && use_hs) pass = nonpositive(exact_dot(dim, nrm, dx));
    }
    unsigned m = __ballot_sync(0xffffffffu, pass);
    if (pass) {
      const int slot = count + __popc(m & ((1u << lane) - 1u));
      wb.d2[slot] = d2;
      wb.id[slot] = cl.sorted[pos];
    }
    count += __popc(m);
    __syncwarp();
  }
  return count;
}

// Bitonic sort of the first `count` candidates by (d2, id) within one warp.
__device__ void warp_sort_candidates(WarpBuf& wb, int count) {
  const int lane = threadIdx.x & 31;
  int n2 = 1;
  while (n2 < count) n2 <<= 1;
  for (int i = count + lane; i < n2; i += 32) {
    wb.d2[i] = DBL_MAX;
    wb.id[i] = INT_MAX;
  }
  __syncwarp();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < (n2 >> 1); i += 32) {
        // stride is a power of two: a = 2 stride (i / stride) + i % stride
        const int a = ((i & ~(stride - 1)) << 1) | (i & (stride - 1));
        const int b = a + stride;
        bool asc = (a & size) == 0;
        double da = wb.d2[a], db = wb.d2[b];
        int32_t ia = wb.id[a], ib = wb.id[b];
        bool gt = cand_less(db, ib, da, ia);
        if (gt == asc) {
          wb.d2[a] = db;
          wb.d2[b] = da;
          wb.id[a] = ib;
          wb.id[b] = ia;
        }
      }
      __syncwarp();
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kQueryWarps * 32, 7) nbr_query_kernel(NbrQuery q, int buf_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpBuf wb = warpbuf_at(smem_raw + (size_t)(threadIdx.x >> 5) * warpbuf_bytes(buf_cap), buf_cap);
  const int lane = threadIdx.x & 31;
  const CloudDev& cl = q.cloud;
  const GridParams g = *cl.grid;
  const double* org = cl.grid->org;
  constexpr int dim = D;
  const QueryGeo gq = make_query_geo(g, dim);
  // unit-ball volume and the initial radius: about 1.2 k particles expected
  // (on quasi-uniform clouds the count then stays between k and the next
  // power of two above k, which keeps the sort short)
  const double ball = (dim == 1) ? 2.0 : (dim == 2) ? 3.141592653589793 : 4.1887902047863905;
  const double dens = (double)cl.n / (g.volume > 0.0 ? g.volume : 1.0);
  const float inv_dens_ball = (float)(1.0 / (dens * ball));
  // no two points of the grid box are farther apart than the sum of its
  // extents: a search radius above it has seen every particle
  double span = 0.0, ext_min = 1e300;
  for (int c = 0; c < dim; ++c) {
    span += g.h[c] * g.nc[c];
    ext_min = fmin(ext_min, g.h[c] * g.nc[c]);
  }
  const float big = __double2float_ru(1.001 * span + 1e-30);
  // a search that still lacks neighbours once its box spans half the grid in
  // some direction goes straight to the whole grid (one more pass, not a
  // chain of ever larger boxes -- targets whose kept half-space holds too few
  // particles would otherwise rescan most of the cloud several times)
  const float jump = (float)(0.25 * ext_min);
  for (int64_t to = blockIdx.x * (int64_t)kQueryWarps + (threadIdx.x >> 5); to < q.n_tgt;
       to += (int64_t)gridDim.x * kQueryWarps) {
    const int64_t t = q.tgt ? q.tgt[to] : to;
    double xT[3] = {0.0, 0.0, 0.0}, nrm[3] = {0.0, 0.0, 0.0};
    float xTf[3] = {0.0f, 0.0f, 0.0f};
    for (int c = 0; c < dim; ++c) xT[c] = cl.x[c * cl.n + t];
    {
      // the FP32 offset from the grid origin: lane c rounds coordinate c (one
      // FP64 subtraction per lane instead of dim on every lane: GB300's FP64
      // pipe is narrow), then every lane takes the dim values
      float own = 0.0f;
      const double xc = lane == 0 ? xT[0] : (lane == 1 ? xT[1] : xT[2]);
      if (lane < dim) own = __double2float_rn(__dsub_rn(xc, org[lane]));
      for (int c = 0; c < dim; ++c) xTf[c] = __shfl_sync(0xffffffffu, own, c);
    }
    bool use_hs = false;
    float nrmf[3] = {0.0f, 0.0f, 0.0f}, hs_scale = 0.0f;
    if (q.halfspace) {
      for (int c = 0; c < dim; ++c) {
        nrm[c] = q.halfspace[to * dim + c];
        use_hs |= (nrm[c] != 0.0);
        nrmf[c] = __double2float_rn(nrm[c]);
        hs_scale += fabsf(nrmf[c]);
      }
      hs_scale *= 0x1p-20f * 1.0001f;
    }
    uint8_t st = GMLS_T_OK;
    int kq = q.k_pt ? q.k_pt[to] : q.k;  // per-target k is clamped to 1..cap
    kq = kq < 1 ? 1 : (kq > q.cap ? q.cap : kq);
    // search radius R in FP32 (any value is correct: the search widens or
    // narrows it); the exact test is d2 < R2 = fl32(R * R) in FP64, and the
    // box half-width R (1 + 2^-20) covers sqrt(R2)
    float R = powf(1.2f * (float)kq * inv_dens_ball, 1.0f / (float)dim);
    int count = 0;
    float r_lo = 0.0f, r_hi = INFINITY;  // radii known to give too few / too many
    for (int attempt = 0; attempt < 64; ++attempt) {
      count = gather_candidates<D>(cl, g, gq, xT, xTf, R * (1.0f + 0x1p-20f), (double)(R * R), use_hs, nrm, nrmf,
                                   hs_scale, wb);
      // rescale R by the count it gave (ball volume ~ R^dim), within bounds,
      // and inside the bracket (r_lo, r_hi) the earlier attempts established
      if (count > wb.cap) {
        r_hi = R;
        R *= fmaxf(0.5f, fminf(0.9f, powf(0.8f * (float)wb.cap / (float)count, 1.0f / (float)dim)));
        if (R <= r_lo) R = 0.5f * (r_lo + r_hi);
        continue;
      }
      if (count >= kq) break;
      if (R > big) break;  // whole cloud inside: too few exist
      r_lo = R;
      // grow by the count's shortfall (ball volume ~ R^dim), at least 10 %; from
      // the fourth attempt on at least 50 % (targets whose kept half-space is
      // nearly empty: fewer rescans of ever larger boxes)
      const float min_growth = attempt >= 3 ? 1.5f : 1.1f;
      R *= (count > 0) ? fminf(2.0f, fmaxf(min_growth, powf(1.3f * (float)kq / (float)count, 1.0f / (float)dim)))
                       : 2.0f;
      if (R > jump) R = fmaxf(R, big * 1.001f);
      if (R >= r_hi) R = 0.5f * (r_lo + r_hi);
    }
    if (count > wb.cap) {  // could not bring the candidate set under the buffer size
      st |= GMLS_T_OVERFLOW;
      count = wb.cap;
    }
    if (count < kq) st |= GMLS_T_TOO_FEW_NEIGHBOURS;
    warp_sort_candidates(wb, count);
    const int kk = count < kq ? count : kq;
    // k-nearest lists: eps = eps_factor sqrt(d2_k) waits until after the
    // loop, where each lane takes one of the warp's targets (the k-th d2, or
    // -1 when the list came up short, parks in out_eps); radius lists need it
    // here
    double eps = 0.0;
    if (q.mode == GMLS_NBR_KNN)
      eps = kk == kq ? wb.d2[kq - 1] : -1.0;
    else if (kk == kq)
      eps = __dmul_rn(q.eps_factor, __dsqrt_rn(wb.d2[kq - 1]));
    if (q.mode == GMLS_NBR_KNN && !q.k_pt) {
      for (int i = lane; i < q.k; i += 32) q.out_idx[to * q.k + i] = (i < kk) ? wb.id[i] : -1;
    } else if (q.mode == GMLS_NBR_KNN) {  // per-target k: padded rows, compacted later
      for (int i = lane; i < kq; i += 32) q.out_idx[to * q.cap + i] = (i < kk) ? wb.id[i] : -1;
      if (lane == 0) q.out_cnt[to] = kq;
    } else {
      int keep = 0;
      if (kk == kq) {
        __syncwarp();
        count = gather_candidates<D>(cl, g, gq, xT, xTf, __double2float_ru(eps) * (1.0f + 0x1p-20f),
                                     __dmul_rn(eps, eps), use_hs, nrm, nrmf, hs_scale, wb);
        if (count > wb.cap) {
          st |= GMLS_T_OVERFLOW;
          count = wb.cap;
        }
        warp_sort_candidates(wb, count);
        keep = count < q.cap ? count : q.cap;
      }
      for (int i = lane; i < keep; i += 32) q.out_idx[to * q.cap + i] = wb.id[i];
      if (lane == 0) q.out_cnt[to] = keep;
    }
    if (lane == 0) {
      q.out_eps[to] = eps;
      q.out_status[to] = st;
    }
    __syncwarp();
  }
  if (q.mode == GMLS_NBR_KNN) {
    // eps of this warp's targets, one per lane (the warp's own writes above
    // are ordered before these reads by the __syncwarp that ends each target)
    const int64_t w0 = blockIdx.x * (int64_t)kQueryWarps + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kQueryWarps;
    for (int64_t to = w0 + lane * stride; to < q.n_tgt; to += 32 * stride) {
      const double d2 = q.out_eps[to];
      q.out_eps[to] = d2 >= 0.0 ? __dmul_rn(q.eps_factor, __dsqrt_rn(d2)) : 0.0;
    }
  }
}

cudaError_t launch_nbr_query(const Launch& L, const NbrQuery& q) {
  if (q.n_tgt == 0) return cudaSuccess;
  // candidate buffer: about twice k for k-nearest lists (a fuller buffer only
  // triggers a smaller search radius), the full 1024 for radius lists, which
  // must hold every candidate inside eps
  // k-nearest: a buffer of at least twice k (up to 2048 for k = 1024), so a
  // radius that gathers between k and the buffer size always exists on
  // quasi-uniform clouds; radius lists: the 1024 entries a list may hold
  int cap = 64;
  const int want = q.mode == GMLS_NBR_KNN ? 2 * q.k : kNbrCap;
  const int limit = q.mode == GMLS_NBR_KNN ? 2 * kNbrCap : kNbrCap;
  while (cap < want && cap < limit) cap <<= 1;
  const size_t smem = warpbuf_bytes(cap) * kQueryWarps;
  const void* fn = q.cloud.dim == 2 ? (const void*)nbr_query_kernel<2> : (const void*)nbr_query_kernel<3>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (q.n_tgt + kQueryWarps - 1) / kQueryWarps;
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  if (q.cloud.dim == 2)
    nbr_query_kernel<2><<<(unsigned)blocks, kQueryWarps * 32, smem, L.stream>>>(q, cap);
  else
    nbr_query_kernel<3><<<(unsigned)blocks, kQueryWarps * 32, smem, L.stream>>>(q, cap);
  *L.counter += 1;
  return cudaGetLastError();
}

__global__ void fill_offsets_fixed_kernel(int64_t* off, int64_t n_tgt, int k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n_tgt; i += (int64_t)gridDim.x * blockDim.x)
    off[i] = i * (int64_t)k;
}

cudaError_t launch_fill_offsets_fixed(const Launch& L, int64_t* off, int64_t n_tgt, int k) {
  fill_offsets_fixed_kernel<<<blocks_for(n_tgt + 1, 256), 256, 0, L.stream>>>(off, n_tgt, k);
  *L.counter += 1;
  return cudaGetLastError();
}

__global__ void fill_identity_kernel(int32_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)i;
}

cudaError_t launch_fill_identity(const Launch& L, int32_t* out, int64_t n) {
  fill_identity_kernel<<<blocks_for(n, 256), 256, 0, L.stream>>>(out, n);
  *L.counter += 1;
  return cudaGetLastError();
}

// The k' nearest of a target are the first k' entries of its k-nearest list
// (both are prefixes of one total order by (d^2, id)); eps' = f * sqrt(d^2 of
// entry k'-1), with d^2 recomputed by the search's exact formula.  A warp
// takes 32 consecutive targets: lane l computes eps' of target l, then the
// warp copies the 32 k'-prefixes as one contiguous, coalesced output range.
__global__ void nbr_prefix_kernel(int dim, int64_t n, const double* __restrict__ x, const int32_t* __restrict__ tgt,
                                  int64_t n_tgt, const int32_t* __restrict__ idx, int k, int kp, double eps_factor,
                                  int32_t* __restrict__ out_idx, double* __restrict__ out_eps,
                                  uint8_t* __restrict__ out_status) {
  const int lane = threadIdx.x & 31;
  const int64_t n_tiles = (n_tgt + 31) >> 5;
  for (int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; tile < n_tiles;
       tile += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t t0 = tile << 5;
    const int nt = (int)((n_tgt - t0) < 32 ? (n_tgt - t0) : 32);
    if (lane < nt) {
      const int64_t t = t0 + lane;
      const int32_t last = idx[t * k + kp - 1];
      if (last < 0) {
        out_eps[t] = 0.0;
        out_status[t] = GMLS_T_TOO_FEW_NEIGHBOURS;
      } else {
        const int64_t tt = tgt[t];
        double dx[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; ++c) dx[c] = __dsub_rn(x[c * n + last], x[c * n + tt]);
        out_eps[t] = __dmul_rn(eps_factor, __dsqrt_rn(exact_d2(dim, dx)));
        out_status[t] = 0;
      }
    }
    // element e of the tile's output is entry (e % kp) of target e / kp;
    // the quotient and remainder are carried along instead of divided
    const int total = nt * kp;
    int q = lane / kp, r = lane - (lane / kp) * kp;
    for (int e = lane; e < total; e += 32) {
      out_idx[t0 * kp + e] = idx[(t0 + q) * k + r];
      r += 32;
      while (r >= kp) {
        r -= kp;
        ++q;
      }
    }
  }
}

cudaError_t launch_nbr_prefix(const Launch& L, int dim, int64_t n, const double* x, const int32_t* tgt, int64_t n_tgt,
                              const int32_t* idx, int k, int kp, double eps_factor, int32_t* out_idx, double* out_eps,
                              uint8_t* out_status) {
  if (n_tgt == 0) return cudaSuccess;
  nbr_prefix_kernel<<<blocks_for((n_tgt + 31) / 32 * 32, 256), 256, 0, L.stream>>>(dim, n, x, tgt, n_tgt, idx, k, kp,
                                                                                     eps_factor, out_idx, out_eps,
                                                                                     out_status);
  *L.counter += 1;
  return cudaGetLastError();
}

// warp per target: copy cnt[t] entries of the padded row into the CSR slot
__global__ void compact_padded_kernel(const int32_t* __restrict__ padded, int cap, const int32_t* __restrict__ cnt,
                                      const int64_t* __restrict__ off, int32_t* __restrict__ out, int64_t n_tgt) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < n_tgt;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int c = cnt[t];
    const int64_t o = off[t];
    for (int i = lane; i < c; i += 32) out[o + i] = padded[t * cap + i];
  }
}

cudaError_t launch_compact_padded(const Launch& L, const int32_t* padded, int cap, const int32_t* cnt,
                                  const int64_t* off, int32_t* out, int64_t n_tgt) {
  compact_padded_kernel<<<blocks_for(n_tgt * 32, 256), 256, 0, L.stream>>>(padded, cap, cnt, off, out, n_tgt);
  *L.counter += 1;
  return cudaGetLastError();
}

}  // namespace gmls
