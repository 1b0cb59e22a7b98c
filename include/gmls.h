/*
 * gmls.h -- C ABI of the GB300 GMLS stencil library (libgmls.so).
 *
 * The library generates generalized-moving-least-squares (GMLS) stencils, the
 * local hot path of the compatible meshless Stokes scheme of "Parallel
 * implementation of a compatible high-order meshless method for the Stokes'
 * equations" (arXiv 2104.14447):
 *
 *   gmls_neighbors     the particles within the support of each target
 *                      (Sec. 2.1, the set N_T of Eq. optimization-discretized-4)
 *   gmls_stencils      for each target: weighted, eps-scaled basis matrix
 *                      (Eqs. matrix-P, matrix-W, basis-functions-3d; the
 *                      divergence-free basis of Sec. 2.2), the weighted
 *                      least-squares solve (Eqs. matrix-A, matrix-B, vector-c),
 *                      optionally the Neumann constraint of Sec. 2.3, and the
 *                      target functionals (Sec. 2.5, Eq.
 *                      polynomial-approximation-derivative) giving the
 *                      stencil weights alpha_Ij of Sec. 3.2
 *   gmls_assemble_csr  scatter of one operator's weights into CSR through the
 *                      local-to-global map J = LTG(I, j) of Sec. 3.2
 *   gmls_stokes_*      the block collocation system of Sec. 3.2 from velocity
 *                      and pressure stencils, its right-hand side, and a CSR
 *                      matrix-vector product to apply it
 *   gmls_gmres         its global solve (Sec. 3.3) by restarted GMRES
 *
 * Conventions
 *   - Every function returns a gmls_status; 0 is success, negative values are
 *     errors.  Argument errors are detected on the host and returned before
 *     any work is queued.  gmls_last_error() describes the last error.
 *   - Work is queued asynchronously on the context's CUDA stream.  Device-side
 *     per-target conditions are reported in the per-target status array
 *     (GMLS_T_* bits), never by aborting.
 *   - Device memory: the context sub-allocates everything it owns from one
 *     caller-provided device buffer (the arena); the library itself never
 *     calls cudaMalloc.  Outputs of gmls_assemble_csr and gmls_export go to
 *     caller-owned buffers.
 *   - Pointers documented as "host or device" may be either; the library asks
 *     the CUDA driver which one it is.
 *   - Coordinates are FP64 structure-of-arrays: x[c * n + i] is coordinate c
 *     of particle i.
 *   - A context is not thread-safe; use one context per host thread.
 *   - There is no CPU fallback: without a CUDA device every call that needs
 *     one fails with GMLS_ECUDA.
 */
#ifndef GMLS_H
#define GMLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmls_ctx gmls_ctx;
typedef int32_t gmls_status;

/* call status */
#define GMLS_OK 0
#define GMLS_EINVAL (-1)    /* bad argument or unsupported (d, m, basis)      */
#define GMLS_ENOMEM (-2)    /* the arena cannot hold the request             */
#define GMLS_ECUDA (-3)     /* a CUDA call failed (message in last_error)    */
#define GMLS_ETIMEOUT (-4)  /* reserved: no call returns it (no kernel of this
                               library waits on a device flag or a peer)   */
#define GMLS_EBUSY (-5)     /* handle still in use                           */
#define GMLS_ENOTFOUND (-6) /* unknown handle                                */
#define GMLS_ECANCELED (-7) /* the server request was cancelled before it ran */

/* per-target status bits (uint8 per target) */
#define GMLS_T_OK 0
#define GMLS_T_RANK_DEFICIENT 1      /* |r_ii| <= 64 n u max|r| (FP64): weights set to zero   */
#define GMLS_T_ILL_CONDITIONED 2     /* max|r_ii| / min|r_ii| > 1e6                            */
#define GMLS_T_REFINE_NOT_CONVERGED 4 /* FP32 refinement missed its tolerance: FP64 redone */
#define GMLS_T_TOO_FEW_NEIGHBOURS 8  /* fewer candidates than requested (weights zero)       */
#define GMLS_T_FP64_FALLBACK 16      /* result recomputed by the FP64 path                    */
#define GMLS_T_OVERFLOW 32           /* candidate buffer exceeded (neighbour list truncated) */
#define GMLS_T_UNSUPPORTED 64        /* rows x basis size exceed every tile the library has (weights zero) */

/* neighbour modes */
#define GMLS_NBR_KNN 0    /* k nearest by (d^2, index); eps = eps_factor * d_k                */
#define GMLS_NBR_RADIUS 1 /* all with d^2 < eps^2, eps = eps_factor * d_k, nearest cap kept    */

/* bases */
#define GMLS_BASIS_SCALAR 0  /* scaled Taylor monomials, Q = C(m+d, d)          (Sec. 2.1) */
#define GMLS_BASIS_DIVFREE 1 /* divergence-free vector polynomials of degree m  (Sec. 2.2) */
#define GMLS_BASIS_STAGGERED 2 /* staggered GMLS (Sec. 2.4): the gradient is fitted by vector
                                  polynomials of degree m through their line integrals
                                  from x_T to each neighbour, against p_j - p(x_T); the
                                  line integrals span the monomials of degree 1..m+1,
                                  which form the basis used.  Functionals GMLS_F_GRAD
                                  (q_h(x_T)) and GMLS_F_LAPLACIAN (div q_h(x_T)); the
                                  weights act on point values: the target's own entry
                                  carries minus the sum of the others.  The target must
                                  be in its own neighbour list (k-nearest lists always
                                  hold it); otherwise GMLS_T_UNSUPPORTED and zero
                                  weights.  No Neumann constraint.                     */

/* weights */
#define GMLS_WEIGHT_POLY 0 /* W(r) = (1 - r/eps)_+^p  (Eq. kernel, p = weight_power) */

/* functionals (rows per target) */
#define GMLS_F_GRAD 0          /* scalar basis: d rows, d/dx_c                                 */
#define GMLS_F_LAPLACIAN 1     /* scalar basis: 1 row                                          */
#define GMLS_F_DIV 2           /* 1 row over (neighbour, component): scalar basis applies
                                  d/dx_c to component c; divergence-free basis gives zeros     */
#define GMLS_F_VEC_LAPLACIAN 3 /* divergence-free basis: d rows over (neighbour, component)   */
#define GMLS_F_CURLCURL 4      /* divergence-free basis: d rows, curl curl = -Laplacian        */

/* precision */
#define GMLS_FP64 0        /* FP64 basis, QR and apply                                       */
#define GMLS_FP32_REFINE 1 /* FP32 QR, FP64-class residuals, FP32 corrections (FP64 redo)     */

/* export selectors */
#define GMLS_X_NBR_OFFSETS 0 /* int64 [n_targets + 1]                          */
#define GMLS_X_NBR_INDEX 1   /* int32 [nnz]                                    */
#define GMLS_X_NBR_EPS 2     /* double [n_targets]                             */
#define GMLS_X_NBR_STATUS 3  /* uint8 [n_targets]                              */
#define GMLS_X_WEIGHTS 4     /* double, layout of gmls_stencil_info            */
#define GMLS_X_BETA 5        /* double [n_targets][rows] Neumann coefficient   */
#define GMLS_X_STATUS 6      /* uint8 [n_targets] stencil status               */
#define GMLS_X_ITERS 7       /* uint8 [n_targets] refinement iterations used   */

typedef struct {
  int32_t mode;              /* GMLS_NBR_KNN or GMLS_NBR_RADIUS                              */
  int32_t k;                 /* k (>= 1)                                                     */
  double eps_factor;         /* eps = eps_factor * (distance of the k-th neighbour), > 0     */
  int32_t cap;               /* radius mode: at most cap neighbours (nearest kept); >= k     */
  int32_t reserved;          /* must be 0                                                    */
  const int32_t* targets;    /* host or device int32 [n_targets] particle ids; NULL = all    */
  int64_t n_targets;         /* ignored when targets is NULL                                 */
  const double* halfspace;   /* NULL, or host or device [n_targets][dim]: keep only j with
                                n . (x_j - x_T) <= 0; an all-zero row disables the filter    */
  const int32_t* k_per_target; /* NULL, or host or device int32 [n_targets] (1..cap): k of each
                                target (KNN: list length; RADIUS: the k whose distance sets
                                eps); k above is then the largest value                      */
} gmls_nbr_params;

typedef struct {
  int32_t basis;              /* GMLS_BASIS_*                                                */
  int32_t degree;             /* m in 1..4 (used when degree_per_target is NULL)             */
  int32_t weight;             /* GMLS_WEIGHT_POLY                                            */
  int32_t weight_power;       /* p >= 1 (4 in the paper's configuration)                     */
  int32_t precision;          /* GMLS_FP64 or GMLS_FP32_REFINE                               */
  int32_t n_functionals;      /* 1..5                                                        */
  int32_t functionals[5];     /* GMLS_F_*, no repeats                                        */
  int32_t neumann;            /* 1: targets whose cloud boundary flag is set take the
                                 Neumann constraint n . grad u = h (scalar basis only)       */
  int32_t max_refine;         /* FP32_REFINE: iteration cap (0 = default 3)                  */
  double refine_tol;          /* FP32_REFINE: stop when the estimated error left, |ds|_inf x
                                 (contraction estimate), is <= tol |s|_inf (0 = 1e-10)       */
  const int8_t* degree_per_target; /* NULL, or host or device int8 [n_targets], m in 1..4    */
} gmls_stencil_params;

/*
 * Create a context on CUDA device `device`, queueing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  `arena` is a device buffer
 * of `arena_bytes` bytes owned by the caller, which must outlive the context;
 * all the context's device memory is carved out of it.
 * Errors: GMLS_EINVAL (NULL out/arena, arena_bytes < 1 MiB), GMLS_ECUDA.
 */
gmls_status gmls_create(gmls_ctx** out, int device, void* cuda_stream, void* arena, size_t arena_bytes);

/* Wait for queued work, then free the context (not the arena). */
gmls_status gmls_destroy(gmls_ctx* ctx);

/* Switch the stream later calls queue on (previous work is not waited for). */
gmls_status gmls_set_stream(gmls_ctx* ctx, void* cuda_stream);

/*
 * Register a point cloud (Sec. 2.1: particles x_i, i = 1..N).  dim is 2 or 3;
 * xyz is host or device FP64 SoA [dim][n]; normals (SoA [dim][n], outward unit
 * normals, used for Neumann targets) and bflags (uint8 [n], nonzero = on the
 * boundary Gamma) may be NULL.  The context copies them into its arena and
 * builds the cell list on the device.  Returns a handle in *cloud_id.
 */
gmls_status gmls_cloud(gmls_ctx* ctx, int dim, int64_t n, const double* xyz, const double* normals,
                       const uint8_t* bflags, int64_t* cloud_id);

/*
 * Neighbour lists for the targets of a cloud (Sec. 2.1, "the particles within
 * a distance eps of x_T").  Distances are exact FP64 squared distances
 * ((dx*dx + dy*dy) + dz*dz, dx = x_j - x_T, no fused multiply-add); lists are
 * sorted by (d^2, particle id) and include the target itself.  The result
 * handle owns CSR offsets (int64), indices (int32), eps (double) and a status
 * byte per target (GMLS_T_TOO_FEW_NEIGHBOURS, GMLS_T_OVERFLOW).
 */
gmls_status gmls_neighbors(gmls_ctx* ctx, int64_t cloud_id, const gmls_nbr_params* params, int64_t* nbrs_id);

/*
 * The k nearest neighbours of every target of a fixed-k nearest-neighbour
 * handle with at least k neighbours, without a new search: under the order by
 * (d^2, particle id) the k nearest are the first k entries of the longer list,
 * and eps = eps_factor * (distance of entry k), recomputed with the same
 * exact formula -- identical to gmls_neighbors(KNN, k, eps_factor).
 */
gmls_status gmls_neighbors_prefix(gmls_ctx* ctx, int64_t nbrs_id, int32_t k, double eps_factor, int64_t* nbrs_id_out);

/*
 * Stencil weights for every target of a neighbour handle.  For functional f
 * with R_f rows and c_in components (1 for the scalar basis, d for the
 * divergence-free basis and for GMLS_F_DIV), the weights of target t occupy
 * R_f * k_t * c_in doubles starting at element off[t] * R_f * c_in (off = the
 * neighbour offsets), ordered [row][neighbour][component], neighbours in list
 * order.  Weight w satisfies, for every polynomial field q of the basis span,
 * sum w q(x_j) = (L q)(x_T) (plus beta * h for Neumann targets).
 * Besides the weights, a launch takes temporary scratch from the arena for
 * the duration of the kernel: the factored divergence-free kernel about
 * 29 KB per resident warp (3D degree 3: 152 SMs x 12 warps, 53 MB; on a
 * smaller arena it runs a smaller grid, down to one block of 12 warps), the
 * shared-memory kernel its global tiles for shapes too large for shared
 * memory; GMLS_ENOMEM when the arena cannot hold them.
 */
gmls_status gmls_stencils(gmls_ctx* ctx, int64_t nbrs_id, const gmls_stencil_params* params, int64_t* stencil_id);

/* Shape of one functional's weights: rows per target, components, total doubles. */
gmls_status gmls_stencil_info(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* n_targets,
                              int32_t* rows, int32_t* ncomp, int64_t* n_values);

/*
 * CSR operator of one functional (Sec. 3.2).  Operator row t * R_f + r holds
 * the weights of target t, row r, at columns (particle id * c_in + component),
 * sorted ascending; explicit zeros are kept.  gmls_csr_size waits for the
 * stream (it reads the nonzero count) and returns n_rows, n_cols, nnz; the
 * caller then passes device buffers row_ptr (int64 [n_rows + 1]), col (int32
 * [nnz]) and val (double [nnz]) to gmls_assemble_csr, which is asynchronous.
 */
gmls_status gmls_csr_size(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* n_rows, int64_t* n_cols,
                          int64_t* nnz);
gmls_status gmls_assemble_csr(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t* row_ptr, int32_t* col,
                              double* val);

/*
 * As gmls_assemble_csr, with nnz_offset (>= 0) added to every row pointer.
 * For an operator assembled in target ranges (one neighbour handle per
 * contiguous range of targets, in order): pass row_ptr + the range's first
 * operator row, col + nnz_offset and val + nnz_offset, nnz_offset being the
 * nonzeros of the ranges before it.  The last row pointer a range writes is
 * the first of the next range (the same value).  For a handle without
 * targets only row_ptr[0] is written and col / val may be NULL.
 * Asynchronous; GMLS_EINVAL for a negative offset.
 */
gmls_status gmls_assemble_csr_at(gmls_ctx* ctx, int64_t stencil_id, int32_t functional, int64_t nnz_offset,
                                 int64_t* row_ptr, int32_t* col, double* val);

/*
 * Stokes collocation system (Sec. 3.2, Eq. stokes-block-system) of the
 * problem of Sec. 3.1 (nu curl curl v + grad phi = f in the interior,
 * v = w on the boundary, Laplacian phi = div f with the Neumann condition
 * n . grad phi = n . f - nu n . curl curl v on the boundary), assembled from
 * two stencil handles over ONE cloud that carries boundary flags and outward
 * normals, both computed for every point of the cloud in order (neighbour
 * handles made without a target list):
 *   velocity: divergence-free basis, functional GMLS_F_CURLCURL;
 *   pressure: scalar basis, GMLS_F_GRAD and GMLS_F_LAPLACIAN, neumann = 1
 *             (boundary points get the constrained Laplacian and its beta).
 * Unknowns: velocity of point J, component c at column J d + c; pressure of
 * J at n d + J; the zero-mean multiplier at n d + n (n = points, d = dim).
 * Rows, in this order:
 *   I d + c, interior I:  nu * curl curl weights (velocity columns), then the
 *                         gradient row c (pressure columns)
 *   I d + c, boundary I:  1 at column I d + c (Dirichlet)
 *   n d + I, interior I:  Laplacian weights, then 1 at the multiplier; with
 *                         pressure_interior != 0 the staggered Laplacian
 *                         weights on that handle's neighbour lists
 *                         (Sec. 3.2, Eq. laplacian-pressure-stencil)
 *   n d + I, boundary I:  -nu * beta_I * (n_I . curl curl weights) on the
 *                         velocity columns (n . a evaluated
 *                         ((n_0 a_0) + (n_1 a_1)) + (n_2 a_2), then
 *                         nu * (beta * (n . a))), the constrained Laplacian
 *                         weights, 1 at the multiplier
 *   n d + n:              1 at every pressure column (zero mean)
 * Columns ascend within each row; neighbour lists enter in particle-id order.
 * The right-hand side (gmls_stokes_rhs) is f (interior momentum rows), w
 * (Dirichlet rows), div f (interior pressure rows), div f - beta n . f
 * (boundary pressure rows) and 0; f and w are SoA [d][n], div_f [n], b
 * [n d + n + 1], all device buffers.
 * gmls_stokes_size waits for the stream (it counts the nonzeros); the caller
 * then passes device buffers row_ptr (int64 [n_rows + 1]), col (int32 [nnz])
 * and val (double [nnz]) to gmls_stokes_assemble, which is asynchronous.
 * GMLS_EINVAL for handles of the wrong kind, different clouds, target lists,
 * a cloud without flags or normals, or more than 2^31 unknowns;
 * GMLS_ENOTFOUND for a handle that does not exist.
 */
typedef struct {
  int64_t velocity;          /* stencil handle (divergence-free basis, curl curl) */
  int64_t pressure;          /* stencil handle (scalar basis, gradient + Laplacian, neumann = 1) */
  double nu;                 /* kinematic viscosity, >= 0 */
  int64_t pressure_interior; /* 0, or a stencil handle (staggered basis, Laplacian; every point
                                of the same cloud in order) whose weights form the interior
                                pressure rows; the boundary rows keep the scalar handle's
                                constrained Laplacian.  The right-hand side does not depend on it.
                                Zero-initialise the struct: 0 keeps the scalar Laplacian. */
} gmls_stokes_params;

gmls_status gmls_stokes_size(gmls_ctx* ctx, const gmls_stokes_params* params, int64_t* n_rows, int64_t* nnz);
gmls_status gmls_stokes_assemble(gmls_ctx* ctx, const gmls_stokes_params* params, int64_t* row_ptr, int32_t* col,
                                 double* val);
gmls_status gmls_stokes_rhs(gmls_ctx* ctx, const gmls_stokes_params* params, const double* f, const double* w,
                            const double* div_f, double* b);

/*
 * y = A x for a CSR matrix with n_rows rows (row_ptr int64 [n_rows + 1], col
 * int32, val double; x and y double), FP64, all device buffers; asynchronous
 * on the context stream.  The sum order within a row is not sequential but
 * fixed (it depends only on the row's length): repeated calls give the same
 * bits.  Rows of more than 8192 entries are summed by thread blocks (cut
 * into 128 slices when there are at most 64 such rows).
 */
gmls_status gmls_csr_spmv(gmls_ctx* ctx, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                          const double* val, const double* x, double* y);

/*
 * Solve A x = b (square CSR, n rows; FP64) by restarted GMRES(restart) with
 * right Jacobi preconditioning (diag A: the sum of the row's entries in
 * column r when the column appears more than once, as A x adds them; 1 where
 * it is zero or absent), on
 * the row-equilibrated system when params->row_scaling = 1 -- the global
 * solve of the collocation system of Sec. 3.2 (the paper uses a
 * block-preconditioned Krylov method).  x: device buffer holding the initial
 * guess on entry and the solution on return.  Synchronous: returns after
 * ||b - A x|| <= rtol ||b|| (with row scaling ||R (b - A x)|| <= rtol ||R b||;
 * the true residual, recomputed at every restart) or
 * max_iter iterations; *iters and *rel_residual report them (a solve that
 * stops at max_iter still returns GMLS_OK: check *rel_residual).  Scratch
 * ((restart + 1) n doubles and a few vectors) comes from the arena
 * (GMLS_ENOMEM if it does not fit); GMLS_EBUSY during stream capture.  Every
 * reduction has a fixed order: repeated solves give the same bits.
 */
typedef struct {
  int32_t restart;     /* Krylov basis size, 1..256 */
  int32_t max_iter;    /* iterations over all restarts, >= 0 */
  double rtol;         /* relative residual target, > 0 */
  int32_t row_scaling; /* 0: as above.  1: GMRES on R A D y = R b, x = D y, with R the
                          row equilibration (1 / largest |entry| of each row) and D the
                          Jacobi scaling of R A; residuals (rtol, *rel_residual) are then
                          |R (b - A x)| / |R b|.  Rows of very different magnitudes (the
                          Stokes system's pressure rows against its Dirichlet rows) make
                          the unscaled residual norm stall restarted GMRES. */
  int32_t reserved;    /* must be 0 */
} gmls_gmres_params;

gmls_status gmls_gmres(gmls_ctx* ctx, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* b, double* x, const gmls_gmres_params* params, int32_t* iters,
                       double* rel_residual);

/*
 * Copy one array of a handle to dst (host or device), `bytes` = capacity of
 * dst; GMLS_EINVAL if too small.  Host destinations are synchronous.
 */
gmls_status gmls_export(gmls_ctx* ctx, int64_t id, int32_t what, int32_t functional, void* dst, size_t bytes);

/* Size in bytes of what gmls_export would copy (waits for the stream when the
   size depends on device results). */
gmls_status gmls_export_size(gmls_ctx* ctx, int64_t id, int32_t what, int32_t functional, size_t* bytes);

/* Free a handle (cloud, neighbours or stencils) and its arena memory.  A cloud
   with live neighbour handles, or neighbours with live stencils, is EBUSY. */
gmls_status gmls_release(gmls_ctx* ctx, int64_t id);

/* Wait for all queued work.  GMLS_ECUDA on an asynchronous CUDA error. */
gmls_status gmls_sync(gmls_ctx* ctx);

/* Arena use in bytes: in use now, high-water mark, capacity. */
gmls_status gmls_arena_usage(gmls_ctx* ctx, size_t* used, size_t* peak, size_t* capacity);

/* Number of kernels this context has launched since creation. */
gmls_status gmls_launch_count(gmls_ctx* ctx, int64_t* launches);

/* options of gmls_set_option */
#define GMLS_OPT_FORCE_GENERIC 0 /* 1: every shape uses the shared-memory tile kernel, not the
                                    warp-per-target register kernel (testing and tuning)    */
#define GMLS_OPT_AUTOTUNE 1      /* 1 (default): the first gmls_stencils call for a shape times
                                    the kernel variants (register kernel with a warp or a half
                                    warp per target; for the divergence-free basis the
                                    factored kernel; 1, 2 or 4 warps per target, and for tiles
                                    that leave one block per SM the split and global tile
                                    placements) on up to 8192 targets and caches the fastest;
                                    this call waits for the stream.  0: heuristic choice      */
#define GMLS_OPT_CLEAR_TUNING 2  /* any value: forget the cached choices and timings         */
#define GMLS_OPT_FORCE_VARIANT 3 /* testing: the kernel variant for shapes with uniform
                                    neighbour counts and degree: -1 / -2 / -4 register
                                    kernel with 32 / 16 / 8 lanes per target (-4: no
                                    Neumann rows); -3 the factored
                                    divergence-free kernel (div-free basis, FP32 path);
                                    G + 8 * P for the
                                    shared-memory kernel with G = 1, 2 or 4 warps per target
                                    and tile placement P (0: both tiles in shared memory;
                                    1, FP32 path only: the FP32 tile in shared memory, its
                                    float-float copy in global memory; 2: both tiles in
                                    global memory); 0 (default) no forcing.  gmls_stencils
                                    fails with GMLS_EINVAL where the variant does not exist
                                    or does not fit for the shape                            */
#define GMLS_OPT_FAIL_ALLOC 5    /* testing: n >= 1 makes the n-th next sub-allocation from
                                    the context's arena fail as if the arena were full (the
                                    call that makes it returns GMLS_ENOMEM and releases what
                                    it had taken); 0 (default) disarms                        */
#define GMLS_OPT_POISON 4        /* testing: 1 = gmls_stencils first fills the arrays it
                                    returns (weights, beta, status, iteration counts) with
                                    all-ones bytes (NaN weights), so that an entry no kernel
                                    writes cannot pass for a result left in reused memory    */
#define GMLS_OPT_ORDER_KEY64 6   /* testing: 1 = the id order of neighbour lists (CSR column
                                    order) is sorted on 64-bit keys even where the cloud is
                                    small enough for 32-bit ones; the order is the same      */

/* Set a context option (GMLS_OPT_*); applies to later calls. */
gmls_status gmls_set_option(gmls_ctx* ctx, int32_t option, int64_t value);

/*
 * k-nearest-neighbour lists of every particle of a cloud without allocating
 * device memory (the paper has no counterpart; this entry point is for
 * callers that cannot allocate at the point of use -- e.g. a solver embedded
 * in a larger simulation code that reserves all device memory at start-up
 * and treats any later cudaMalloc as an error, since cudaMalloc synchronises
 * the device and can fail in the middle of a time step).
 *
 * Same results as gmls_cloud + gmls_neighbors(GMLS_NBR_KNN, k, eps_factor)
 * with every particle a target: out_idx [n][k] sorted by (d^2, id), out_eps
 * [n], out_status [n] (GMLS_T_* bits).  xyz (FP64 SoA [dim][n]) and the
 * outputs are caller-owned buffers in the memory of the CURRENT device
 * (GMLS_EINVAL for host memory or another device's); work is queued on
 * cuda_stream.
 * No context is needed and nothing is allocated or freed: the cell-list
 * scratch is one static device array of about 14 MB that every GPU loading
 * the library holds until exit, sized for at most GMLS_NOALLOC_MAX_POINTS
 * particles (GMLS_EINVAL beyond that, message in gmls_last_error(NULL)).
 * All calls on a device share that array and it keeps the last call's
 * contents (the counters that must start at zero are cleared at the start of
 * each call): calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  The first call on a device looks up the array's
 * address once for that device; make it before any stream capture.
 */
#define GMLS_NOALLOC_MAX_POINTS 262144
gmls_status gmls_knn_noalloc(int dim, int64_t n, const double* xyz, int32_t k, double eps_factor, int32_t* out_idx,
                             double* out_eps, uint8_t* out_status, void* cuda_stream);

/*
 * Autotuner record `index` (0-based, in the order taken): fields[9] =
 * {basis, dim, degree, precision, tile rows, solve rows, neumann, bucketed,
 * variant (-1 register kernel with 32 lanes per target, -2 with 16 lanes per
 * target, -3 factored divergence-free kernel, else G + 8 * P for the
 * shared-memory kernel as in
 * GMLS_OPT_FORCE_VARIANT)}, *ms its time.
 * GMLS_ENOTFOUND past the last record.
 */
gmls_status gmls_tune_info(gmls_ctx* ctx, int32_t index, int32_t* fields, float* ms);

/*
 * CUDA-graph capture of a pipeline on the context's stream (which must not
 * be the legacy default stream).  Calls between gmls_capture_begin and
 * gmls_capture_end are recorded, not run; the handles they return stay valid
 * and every gmls_graph_launch rewrites their outputs.  Capture the pipeline
 * after one uncaptured run of the same shapes, so that the autotuner does not
 * need to time anything (it never runs while capturing; uncached shapes then
 * use the heuristic choice).  Calls that must read device results on the host
 * (gmls_csr_size of radius-mode lists, exports to host) return GMLS_EBUSY or
 * fail during capture.  The graph handle is freed by gmls_release.
 */
gmls_status gmls_capture_begin(gmls_ctx* ctx);
gmls_status gmls_capture_end(gmls_ctx* ctx, int64_t* graph_id);
gmls_status gmls_graph_launch(gmls_ctx* ctx, int64_t graph_id);

/*
 * Continuous-batching request server (a stream of independent stencil
 * requests of mixed sizes; the paper has no serving layer).  A scheduler
 * thread admits submitted requests whenever an in-flight slot and a slice of
 * the server arena (first-fit, sized from the request) are free, and issues
 * each request's pipeline -- cloud and cell list, k-nearest neighbours,
 * stencils -- on the least loaded of n_streams CUDA streams, so concurrent
 * requests overlap on the GPU.  Results stay on the device until
 * gmls_server_release.  Each request runs in its own context with a fixed
 * kernel choice per shape (no autotuning), so its result is bit-for-bit the
 * same alone or in the mix.  The arena is a caller-owned device buffer; the
 * server never calls cudaMalloc.  Latency = submit to
 * completion of the request's last kernel (host steady clock).
 */
typedef struct gmls_server gmls_server;

typedef struct {
  int32_t dim;               /* 2 or 3                                               */
  int64_t n;                 /* particles; every particle is a target                */
  const double* xyz;         /* HOST FP64 SoA [dim][n]; copied by gmls_server_submit */
  int32_t basis;             /* GMLS_BASIS_*                                         */
  int32_t degree;            /* m in 1..4                                            */
  int32_t k;                 /* neighbours (k nearest, eps = eps_factor * d_k)       */
  double eps_factor;
  int32_t precision;         /* GMLS_FP64 or GMLS_FP32_REFINE                        */
  int32_t n_functionals;
  int32_t functionals[5];
} gmls_request;

typedef struct {
  int64_t completed, targets, pending, inflight;
  double p50_ms, p99_ms, mean_ms; /* latency of completed requests                 */
  double elapsed_s;               /* first submit to last completion               */
  double targets_per_s;           /* completed targets / elapsed_s                 */
} gmls_serve_stats;

gmls_status gmls_server_create(gmls_server** out, int device, void* arena, size_t arena_bytes, int32_t n_streams,
                               int32_t max_inflight);
/* Queue a request; returns at once with a ticket. */
gmls_status gmls_server_submit(gmls_server* s, const gmls_request* req, int64_t* ticket);
/* Wait up to timeout_ms; *done = 1 when finished (return value: its status). */
gmls_status gmls_server_wait(gmls_server* s, int64_t ticket, int32_t timeout_ms, int32_t* done);
/* Copy one array of a finished request (GMLS_X_* selector, as gmls_export) to
   dst (host or device, `bytes` capacity); dst NULL only reports *needed. */
gmls_status gmls_server_result(gmls_server* s, int64_t ticket, int32_t what, int32_t functional, void* dst,
                               size_t bytes, size_t* needed);
/* Cancel a request that waits for admission: GMLS_OK and it never runs
   (wait then reports it done with GMLS_ECANCELED, result returns
   GMLS_ECANCELED, release frees its record); GMLS_EBUSY once it has been
   admitted or has finished; GMLS_ENOTFOUND for an unknown ticket.  The
   paper has no counterpart (serving is not part of its method). */
gmls_status gmls_server_cancel(gmls_server* s, int64_t ticket);
/* Free a finished request's device memory (GMLS_EBUSY while it runs). */
gmls_status gmls_server_release(gmls_server* s, int64_t ticket);
gmls_status gmls_server_stats(gmls_server* s, gmls_serve_stats* out);
/* Stop the scheduler, wait for the streams, free everything. */
gmls_status gmls_server_destroy(gmls_server* s);

/* Message of the last error on this context (NULL ctx: the last error of a
   call without a context: gmls_create or gmls_knn_noalloc). */
const char* gmls_last_error(gmls_ctx* ctx);

/* Library version string. */
const char* gmls_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GMLS_H */
