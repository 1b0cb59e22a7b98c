// gmls_internal.cuh -- shared declarations of the CUDA side of libgmls.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cfloat>
#include <climits>

#include "../../include/gmls.h"

namespace gmls {

constexpr int kMaxDim = 3;
constexpr int kWarp = 32;
constexpr int kMaxSolveRows = 4;   // distinct functional rows solved per target
constexpr int kNbrCap = 1024;      // candidate buffer per warp in the neighbour query
constexpr int kMaxK = 1024;        // largest neighbour count per target

// ------------------------------------------------------------------ exact FP64
// Squared distance ((dx*dx + dy*dy) + dz*dz), dx = x_j - x_T, every operation
// rounded separately (no contraction into fused multiply-adds), so that the
// value is reproducible bit for bit.
__device__ __forceinline__ double exact_d2(int dim, const double* dx) {
  double d2 = __dmul_rn(dx[0], dx[0]);
  if (dim > 1) d2 = __dadd_rn(d2, __dmul_rn(dx[1], dx[1]));
  if (dim > 2) d2 = __dadd_rn(d2, __dmul_rn(dx[2], dx[2]));
  return d2;
}

// n . (x_j - x_T) with the same evaluation order.
__device__ __forceinline__ double exact_dot(int dim, const double* nrm, const double* dx) {
  double s = __dmul_rn(nrm[0], dx[0]);
  if (dim > 1) s = __dadd_rn(s, __dmul_rn(nrm[1], dx[1]));
  if (dim > 2) s = __dadd_rn(s, __dmul_rn(nrm[2], dx[2]));
  return s;
}

// candidate order: by d2, then by particle id.  Squared distances are
// non-negative (never -0), and for non-negative doubles the IEEE bit patterns
// order exactly like the values, so the order is decided with 64-bit integer
// compares on the ALU instead of FP64 compares on GB300's narrow FP64 pipe.
__device__ __forceinline__ bool cand_less(double da, int32_t ia, double db, int32_t ib) {
  const long long ua = __double_as_longlong(da), ub = __double_as_longlong(db);
  return (ua < ub) || (ua == ub && ia < ib);
}
// a < b for non-negative doubles, as an integer compare
__device__ __forceinline__ bool nonneg_less(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
// s <= 0 (including -0) as a signed integer test of the bit pattern
__device__ __forceinline__ bool nonpositive(double s) { return __double_as_longlong(s) <= 0; }

// ----------------------------------------------------------------- grid state
struct GridParams {
  double lo[kMaxDim];
  double org[kMaxDim];  // bounding-box centre: origin of the FP32 coordinate copies
  double inv_h[kMaxDim];
  double h[kMaxDim];
  int32_t nc[kMaxDim];
  double volume;  // bounding-box volume (for the initial search radius)
};

struct CloudDev {
  int dim;
  int64_t n;
  const double* x;         // SoA [dim][n]
  const double* xs;        // SoA [dim][n], in cell order
  const int32_t* sorted;   // cell order -> particle id
  const int32_t* cell_start;  // [ncell + 1]
  const GridParams* grid;
  int64_t ncell;
  const float* xsf;        // SoA [dim][n], fl32(xs - org) (the query's FP32 pre-filter)
};

// ------------------------------------------------------------ launch helpers
// streaming multiprocessors of the current device (queried once per device);
// grid sizes are multiples of it
int device_sm_count();

struct Launch {
  cudaStream_t stream;
  int64_t* counter;  // kernels launched
};

cudaError_t launch_bbox_and_grid(const Launch& L, int dim, int64_t n, const double* x, const int32_t nc_axis[3],
                                 GridParams* grid, double* scratch_partials, int n_partials);
cudaError_t launch_cell_count(const Launch& L, int dim, int64_t n, const double* x, const GridParams* grid,
                              int32_t* cell_of, int32_t* counts);
cudaError_t launch_scan_i32(const Launch& L, const int32_t* in, int32_t* out_excl, int64_t n, int32_t* scratch,
                            int64_t scratch_elems);
cudaError_t launch_scan_i64_from_i32(const Launch& L, const int32_t* in, int64_t* out_excl, int64_t n,
                                     int64_t* scratch, int64_t scratch_elems);
int64_t scan_scratch_elems(int64_t n);
cudaError_t launch_cell_scatter(const Launch& L, int dim, int64_t n, const double* x, const GridParams* grid,
                                const int32_t* cell_of, const int32_t* cell_start, int32_t* fill, int32_t* sorted,
                                double* xs, float* xsf);

struct NbrQuery {
  CloudDev cloud;
  int64_t n_tgt;
  const int32_t* tgt;        // [n_tgt] or NULL (= identity)
  const double* halfspace;   // [n_tgt][dim] or NULL
  int mode;                  // GMLS_NBR_*
  int k;
  const int32_t* k_pt;       // per-target k or NULL
  int cap;                   // radius mode
  double eps_factor;
  // outputs
  int32_t* out_idx;          // kNN: [n_tgt*k]; radius: padded [n_tgt*cap]
  int32_t* out_cnt;          // radius: [n_tgt]
  double* out_eps;           // [n_tgt]
  uint8_t* out_status;       // [n_tgt]
};
cudaError_t launch_nbr_query(const Launch& L, const NbrQuery& q);
cudaError_t launch_fill_offsets_fixed(const Launch& L, int64_t* off, int64_t n_tgt, int k);
cudaError_t launch_compact_padded(const Launch& L, const int32_t* padded, int cap, const int32_t* cnt,
                                  const int64_t* off, int32_t* out, int64_t n_tgt);
cudaError_t launch_fill_identity(const Launch& L, int32_t* out, int64_t n);
cudaError_t launch_nbr_prefix(const Launch& L, int dim, int64_t n, const double* x, const int32_t* tgt, int64_t n_tgt,
                              const int32_t* idx, int k, int kp, double eps_factor, int32_t* out_idx, double* out_eps,
                              uint8_t* out_status);

// ----------------------------------------------------------------- stencils
struct StencilJob {
  // cloud
  int dim;
  int64_t n;
  const double* x;
  const double* normals;   // SoA [dim][n] or NULL
  const uint8_t* bflag;    // [n] or NULL
  // neighbours
  int64_t n_tgt;
  const int32_t* tgt;      // [n_tgt]
  const int64_t* off;      // [n_tgt+1]
  const int32_t* idx;
  const double* eps;
  const uint8_t* nbr_status;
  // work list: items[0..*n_items) are target ordinals; NULL items = all
  const int32_t* items;
  const int32_t* n_items;
  // basis
  int kind;                // GMLS_BASIS_*
  int degree;
  const int8_t* degree_pt; // [n_tgt] or NULL
  int nc;                  // components per neighbour (1 or dim)
  double wpow;
  int wpow_half;           // p / 2 for even p (float-float path)
  int neumann;
  // solve rows: row r of the L solve rows is functional code lam_fn[r], sub-row lam_row[r]
  int L;
  int lam_fn[kMaxSolveRows];
  int lam_row[kMaxSolveRows];
  int lam_order[kMaxSolveRows];  // |beta| of the row (power of 1/eps)
  // outputs per requested functional
  int nout;
  int out_fn[5];
  int out_rows[5];
  int out_ncomp[5];
  int out_src[5];          // first solve row it reads (-1: zeros)
  int out_sign[5];         // +1 or -1 (curl curl = -vector Laplacian)
  double* out_w[5];
  double* beta;            // [n_tgt][L] or NULL
  uint8_t* status;         // [n_tgt]
  uint8_t* iters;          // [n_tgt]
  // precision
  int max_refine;
  double tol;
  int32_t* fb_items;       // FP32 path: targets to redo in FP64
  int32_t* fb_count;
  int32_t* gen_items;      // register kernel: targets it does not cover (tile
  int32_t* gen_count;      // misfit), for the shared-memory FP32 kernel
  int32_t* neu_items;      // register kernel: Neumann targets, for its Neumann
  int32_t* neu_count;      // instantiation (NULL: they go to gen_items)
  int fallback_run;        // 1: this FP64 launch redoes targets of the FP32 path
  // launch shape
  int ld;                  // tile leading dimension (>= max rows)
  int nmax;                // max basis size
  int warps_per_target;    // 1, 2 or 4 (block = 128 threads)
  unsigned char* dscratch; // factored div-free kernel: [grid blocks * warps][slot] (DfxShape)
};

constexpr int kMaxBuckets = 48;

// How one launch of the shared-memory stencil kernel walks its targets.
struct BatchPlan {
  int single;                   // 1: one bucket over job.items (or all targets)
  int nb;                       // buckets
  const int32_t* items;         // bucket-sorted target ordinals (bucketed mode)
  const int32_t* bucket_start;  // [nb + 1]
  const int32_t* task_start;    // [nb + 1] block tasks
  int32_t* task_counter;        // zeroed before the launch
  int G[kMaxBuckets];           // warps per target
  int ld[kMaxBuckets];          // tile rows
  int nmax[kMaxBuckets];        // tile columns
  int gtile[kMaxBuckets];       // tile placement (kPlaceShared / kPlaceSplit / kPlaceGlobal)
  unsigned char* gscratch;      // [grid blocks][4 / G][gslot_bytes] global tiles
  size_t gslot_bytes;
};

struct BucketJob {
  int64_t n_tgt;
  const int64_t* off;
  const int8_t* degree_pt;
  int degree;
  int nc;
  int n_classes;
  int class_rows[16];
  int nb;                       // n_classes * 4 + 1 (the last: too large)
  int gpb[kMaxBuckets];         // targets per block task
  int32_t* counts;
  int32_t* fill;
  int32_t* bucket_of;
  int32_t* bucket_start;
  int32_t* task_start;
  int32_t* items;
};

// tile placement of the shared-memory kernel (BatchPlan::gtile)
constexpr int kPlaceShared = 0, kPlaceSplit = 1, kPlaceGlobal = 2;
size_t tile_bytes(int ld, int nmax, bool fp32_refine, int place = kPlaceShared);
size_t global_tile_bytes(int ld, int nmax, bool fp32_refine, int place);
int stencil_blocks_per_sm(bool fp32_refine, size_t smem);
cudaError_t launch_stencils(const Launch& L, const StencilJob& j, const BatchPlan& plan, bool fp32_refine,
                            size_t smem, int grid_blocks);
cudaError_t launch_bucketing(const Launch& L, const BucketJob& b);
// register kernel with groups of hw lanes (32 or 16) per target: is this
// shape instantiated, and with how many rows per lane (smallest that fits)
bool fast_path_available(int kind, int dim, int deg, int rows, int L, int hw, int* mr_out);
// the preferred group width for a shape: fewest padded row slots, then 32
int fast_path_preferred(int kind, int dim, int deg, int rows, int L, int* mr_out);
cudaError_t launch_stencils_fast(const Launch& L, const StencilJob& j, int mr, int hw, int sms, bool neu = false);
// is the Neumann instantiation of this register-kernel shape built
bool fast_neu_available(int dim, int deg, int mr, int L, int hw);
// factored divergence-free kernel (dfx.cu): is (dim, degree) instantiated for
// lists of at most kmax neighbours and L solve rows, and its launch
bool dfx_path_available(int dim, int deg, int kmax, int L);
struct DfxShape {
  int grid, warps;  // blocks, warps (targets in flight) per block
  size_t smem;      // shared bytes per block
  size_t scratch;   // global bytes the launch needs in StencilJob::dscratch
};
cudaError_t dfx_launch_shape(const StencilJob& j, int sms, DfxShape* s);
// global scratch of a launch over n_tgt targets (0 if the shape is not instantiated)
size_t dfx_scratch_bytes(int dim, int deg, int64_t n_tgt, int sms);
cudaError_t launch_stencils_dfx(const Launch& L, const StencilJob& j, const DfxShape& s);

// -------------------------------------------------------------------- CSR
// id order of neighbour lists (see nbr_order_kernel): order[off[t] + r] =
// position of target t's entry of rank r by particle id; n_points (the
// cloud's size) selects the sort-key width
cudaError_t launch_nbr_order(const Launch& L, int64_t n_tgt, const int64_t* off, const int32_t* idx, int kcap,
                             int16_t* order, int64_t n_points);
// id order of the k-prefix of fixed-k lists from the order of the full lists
// (kp entries per target): the positions below k, kept in their order
cudaError_t launch_nbr_order_prefix(const Launch& L, int64_t n_tgt, const int16_t* parent_order, int kp, int k,
                                    int16_t* order);

struct CsrJob {
  const int16_t* order;  // id order of the lists
  int64_t n_tgt;
  const int64_t* off;
  const int32_t* idx;
  const double* w;
  int rows;
  int nc;
  int64_t* row_ptr;
  int32_t* col;
  double* val;
  int64_t nnz_base;  // added to every row pointer (ranges of one larger operator)
};
cudaError_t launch_csr(const Launch& L, const CsrJob& j);

// ------------------------------------------------------------ Stokes system
// Collocation system of Sec. 3.2 from per-point stencils (targets = all
// points in order).  Weight layouts as in the stencil handles: functional
// rows R, components C, element offset off[t] R C.
struct StokesJob {
  int dim;
  int64_t n;                 // points
  double nu;                 // viscosity
  const int64_t* off_v;      // velocity lists
  const int32_t* idx_v;
  const double* w_cc;        // curl curl: [off_v[I] d d + c (k d) + j d + c']
  const int64_t* off_p;      // pressure lists
  const int32_t* idx_p;
  const double* w_grad;      // gradient: [off_p[I] d + c k + j]
  const double* w_lap;       // Laplacian (Neumann-constrained at boundary points): [off_p[I] + j]
  const double* beta;        // [I * beta_stride + beta_col]: beta of the Laplacian row
  int beta_stride, beta_col;
  const uint8_t* bflag;      // [n]
  const double* normals;     // [c n + I]
  const int64_t* off_s;      // staggered interior Laplacian lists (nullptr: interior
  const int32_t* idx_s;      //   pressure rows take w_lap on the pressure lists)
  const double* w_stag;      // [off_s[I] + j]
  const int16_t* order_v;    // id order of the velocity lists
  const int16_t* order_p;    // id order of the pressure lists
  const int16_t* order_s;    // id order of the staggered lists
  int32_t* row_len;          // scratch [n d + n + 1]
  int64_t* row_ptr;          // [n d + n + 2]
  int32_t* col;
  double* val;
};
cudaError_t launch_stokes_rowlen(const Launch& L, const StokesJob& j);
cudaError_t launch_stokes_fill(const Launch& L, const StokesJob& j);
cudaError_t launch_stokes_rhs(const Launch& L, const StokesJob& j, const double* f, const double* w,
                              const double* div_f, double* b);
// scratch: long_rows int32 [n_rows], n_long int32, partial double [csr_spmv_partial_elems()]
size_t csr_spmv_partial_elems();
cudaError_t launch_csr_spmv(const Launch& L, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                            const double* val, const double* x, double* y, int32_t* long_rows, int32_t* n_long,
                            double* partial);

// ------------------------------------------------------------- GMRES pieces
// (krylov.cu) V holds basis vectors [i][n]; partial has
// krylov_partial_elems(ncols) doubles; every reduction has a fixed order
size_t krylov_partial_elems(int max_cols);
cudaError_t krylov_dots(const Launch& L, int64_t n, int ncols, const double* V, const double* w, double* partial,
                        double* out);
cudaError_t krylov_axpy(const Launch& L, int64_t n, int ncols, const double* V, const double* h, double* w);
cudaError_t krylov_update(const Launch& L, int64_t n, int ncols, const double* V, const double* y, const double* dinv,
                          double* x);
cudaError_t krylov_scale(const Launch& L, int64_t n, const double* dinv, const double* v, double* z);
cudaError_t krylov_scaled_copy(const Launch& L, int64_t n, const double* src, double s, double* dst);
cudaError_t krylov_residual(const Launch& L, int64_t n, const double* b, double* r);
// rinv = 1 / (largest |entry| of each row), dinv = 1 / diagonal of the
// row-scaled matrix (1 where either is absent or zero)
cudaError_t krylov_row_equilibration(const Launch& L, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                     const double* val, double* rinv, double* dinv);
cudaError_t krylov_scale_in_place(const Launch& L, int64_t n, const double* d, double* v);
cudaError_t krylov_inverse_diagonal(const Launch& L, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                    const double* val, double* dinv);

}  // namespace gmls
