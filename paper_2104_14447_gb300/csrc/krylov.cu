// krylov.cu -- restarted GMRES on the GPU for the collocation system of
// Sec. 3.2 (the global solve of Sec. 3.3; the paper uses a block-
// preconditioned Krylov method, this is a plain right-Jacobi-preconditioned
// GMRES(m), optionally on the row-equilibrated system R A D y = R b).
//
// Vectors are FP64 device arrays.  The Krylov basis V ([m + 1][n], basis
// vector i contiguous) lives in the context arena.  Orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2): two batched dot-product passes
// and two batched updates per iteration instead of 2 (j + 1) kernels.  Every
// reduction has a fixed order (per-block partial sums over fixed row ranges,
// then the partials in block order), so a solve is reproducible bit for bit.
// The small Hessenberg least-squares problem (Givens rotations) runs on the
// host, which reads one column of doubles per iteration.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gmls_internal.cuh"

namespace gmls {

namespace {

// Fixed partition of the batched dot products (304 block partials, two per SM
// of a GB300): the summation order, and so the result, does not depend on
// the device
constexpr int kDotBlocks = 304;
constexpr int kDotThreads = 256;
constexpr int kDotChunk = 8;  // basis vectors per pass of a thread

__device__ __forceinline__ void block_row_range(int64_t n, int64_t* a, int64_t* e) {
  *a = n * blockIdx.x / gridDim.x;
  *e = n * (blockIdx.x + 1) / gridDim.x;
}

// partial[b * ncols + i] = sum over block b's rows of V_i . w (i < ncols)
__global__ void __launch_bounds__(kDotThreads) multi_dot_kernel(int64_t n, int ncols, const double* __restrict__ V,
                                                                const double* __restrict__ w,
                                                                double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32][kDotChunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t a, e;
  block_row_range(n, &a, &e);
  for (int i0 = 0; i0 < ncols; i0 += kDotChunk) {
    double acc[kDotChunk];
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) acc[c] = 0.0;
    for (int64_t p = a + threadIdx.x; p < e; p += kDotThreads) {
      const double wp = w[p];
#pragma unroll
      for (int c = 0; c < kDotChunk; ++c)
        if (i0 + c < ncols) acc[c] = fma(V[(int64_t)(i0 + c) * n + p], wp, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) {
      double s = acc[c];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < kDotChunk && i0 + (int)threadIdx.x < ncols) {
      double s = 0.0;
      for (int wi = 0; wi < kDotThreads / 32; ++wi) s += red[wi][threadIdx.x];
      partial[(int64_t)blockIdx.x * ncols + i0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// out[i] = sum over blocks of partial[b * ncols + i], in block order
__global__ void reduce_partials_kernel(int ncols, int nblocks, const double* __restrict__ partial,
                                       double* __restrict__ out) {
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * ncols + i];
    out[i] = s;
  }
}

// w -= sum_i h[i] V_i   (i < ncols)
__global__ void multi_axpy_kernel(int64_t n, int ncols, const double* __restrict__ V, const double* __restrict__ h,
                                  double* __restrict__ w) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double s = w[p];
    for (int i = 0; i < ncols; ++i) s = fma(-h[i], V[(int64_t)i * n + p], s);
    w[p] = s;
  }
}

// x += dinv .* (sum_i y[i] V_i)
__global__ void update_solution_kernel(int64_t n, int ncols, const double* __restrict__ V,
                                       const double* __restrict__ y, const double* __restrict__ dinv,
                                       double* __restrict__ x) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < ncols; ++i) s = fma(y[i], V[(int64_t)i * n + p], s);
    x[p] = fma(dinv[p], s, x[p]);
  }
}

// z = dinv .* v
__global__ void scale_kernel(int64_t n, const double* __restrict__ dinv, const double* __restrict__ v,
                             double* __restrict__ z) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    z[p] = dinv[p] * v[p];
}

// dst = src * s
__global__ void scaled_copy_kernel(int64_t n, const double* __restrict__ src, double s, double* __restrict__ dst) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    dst[p] = src[p] * s;
}

// r = b - r (r holds A x on entry)
__global__ void residual_kernel(int64_t n, const double* __restrict__ b, double* __restrict__ r) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    r[p] = b[p] - r[p];
}

// dinv[r] = 1 / A[r][r] (1 where the diagonal entry is absent or zero).  A
// row may list column r more than once; as in A x, the entries add up, so
// the diagonal is their sum (the same in both scalings).
__global__ void inverse_diagonal_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                        const int32_t* __restrict__ col, const double* __restrict__ val,
                                        double* __restrict__ dinv) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
      if (col[p] == (int32_t)r) d += val[p];
    dinv[r] = (d != 0.0) ? 1.0 / d : 1.0;
  }
}

// row equilibration: rinv[r] = 1 / max_j |A[r][j]| (1 for an empty or zero
// row), and dinv[r] = 1 / (rinv[r] A[r][r]), the Jacobi scaling of the
// equilibrated matrix (1 where that diagonal entry is absent or zero)
__global__ void row_equilibration_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                         const int32_t* __restrict__ col, const double* __restrict__ val,
                                         double* __restrict__ rinv, double* __restrict__ dinv) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double amax = 0.0, d = 0.0;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      amax = fmax(amax, fabs(val[p]));
      if (col[p] == (int32_t)r) d += val[p];
    }
    const double ri = amax > 0.0 ? 1.0 / amax : 1.0;
    const double ds = ri * d;
    rinv[r] = ri;
    dinv[r] = ds != 0.0 ? 1.0 / ds : 1.0;
  }
}

// v = d .* v
__global__ void scale_in_place_kernel(int64_t n, const double* __restrict__ d, double* v) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    v[p] = d[p] * v[p];
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > (int64_t)device_sm_count() * 16) b = (int64_t)device_sm_count() * 16;
  return (unsigned)b;
}

}  // namespace

cudaError_t krylov_dots(const Launch& L, int64_t n, int ncols, const double* V, const double* w, double* partial,
                        double* out) {
  multi_dot_kernel<<<kDotBlocks, kDotThreads, 0, L.stream>>>(n, ncols, V, w, partial);
  reduce_partials_kernel<<<1, 256, 0, L.stream>>>(ncols, kDotBlocks, partial, out);
  *L.counter += 2;
  return cudaGetLastError();
}

size_t krylov_partial_elems(int max_cols) { return (size_t)kDotBlocks * max_cols; }

cudaError_t krylov_axpy(const Launch& L, int64_t n, int ncols, const double* V, const double* h, double* w) {
  multi_axpy_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, ncols, V, h, w);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_update(const Launch& L, int64_t n, int ncols, const double* V, const double* y, const double* dinv,
                          double* x) {
  update_solution_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, ncols, V, y, dinv, x);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_scale(const Launch& L, int64_t n, const double* dinv, const double* v, double* z) {
  scale_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, dinv, v, z);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_scaled_copy(const Launch& L, int64_t n, const double* src, double s, double* dst) {
  scaled_copy_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, src, s, dst);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_residual(const Launch& L, int64_t n, const double* b, double* r) {
  residual_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, b, r);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_inverse_diagonal(const Launch& L, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                    const double* val, double* dinv) {
  inverse_diagonal_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, row_ptr, col, val, dinv);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_row_equilibration(const Launch& L, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                     const double* val, double* rinv, double* dinv) {
  row_equilibration_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, row_ptr, col, val, rinv, dinv);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t krylov_scale_in_place(const Launch& L, int64_t n, const double* d, double* v) {
  scale_in_place_kernel<<<grid_for(n), 256, 0, L.stream>>>(n, d, v);
  *L.counter += 1;
  return cudaGetLastError();
}

}  // namespace gmls
