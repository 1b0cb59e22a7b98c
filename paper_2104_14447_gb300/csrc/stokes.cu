// stokes.cu -- the Stokes collocation system of Sec. 3.2 (Eq.
// stokes-block-system) assembled on the GPU from per-point stencils, its
// right-hand side, and a CSR matrix-vector product.
//
// Unknowns: velocity (point J, component c at J d + c), pressure (n d + J),
// the zero-mean multiplier (n d + n).  Rows (Eqs. stokes-velocity-target ..
// stokes-pressure-neumann-target):
//   interior point I, component c:  nu (curl curl stencil) v + (gradient stencil) phi
//   boundary point I, component c:  v_{I,c}                            (delta rows)
//   interior point I, pressure:     (Laplacian stencil) phi + lambda, the
//                                   staggered one (Sec. 2.4) when given
//   boundary point I, pressure:     -nu beta_I n_I . (curl curl stencil) v
//                                   + (Neumann-constrained Laplacian stencil) phi + lambda
//   last row:                       sum_J phi_J                        (zero mean)
// The boundary pressure row eliminates the Neumann datum n . grad phi =
// n . f - nu n . curl curl v (Eq. stokes-pressure-neumann) through the
// constrained stencil (Laplacian ~ sum w_j phi_j + beta h, Sec. 2.3), which
// puts -nu beta n . (curl curl stencil) on the velocity and div f - beta n . f
// on the right.  Columns ascend within every row (velocity block first, then
// pressure, then the multiplier), each neighbour list in particle-id order
// (the lists' cached id order).
#include <cuda_runtime.h>

#include <climits>

#include "gmls_internal.cuh"

namespace gmls {

namespace {

constexpr int kStokesWarps = 8;

inline unsigned grid_for(int64_t n, int per_block) {
  int64_t b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > (int64_t)device_sm_count() * 32) b = (int64_t)device_sm_count() * 32;
  return (unsigned)b;
}

__global__ void stokes_rowlen_kernel(StokesJob j) {
  const int d = j.dim;
  const int64_t nd = j.n * d;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < j.n; I += (int64_t)gridDim.x * blockDim.x) {
    const int kv = (int)(j.off_v[I + 1] - j.off_v[I]);
    const int kp = (int)(j.off_p[I + 1] - j.off_p[I]);
    const bool bnd = j.bflag[I] != 0;
    for (int c = 0; c < d; ++c) j.row_len[I * d + c] = bnd ? 1 : kv * d + kp;
    const int kl = j.off_s ? (int)(j.off_s[I + 1] - j.off_s[I]) : kp;  // interior Laplacian row
    j.row_len[nd + I] = bnd ? kv * d + kp + 1 : kl + 1;
    if (I == 0) j.row_len[nd + j.n] = (int32_t)j.n;
  }
}

template <int D>
__global__ void __launch_bounds__(kStokesWarps * 32) stokes_fill_kernel(StokesJob j) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = j.n, nd = n * D;
  const double nu = j.nu;
  for (int64_t I = blockIdx.x * (int64_t)kStokesWarps + warp; I < n; I += (int64_t)gridDim.x * kStokesWarps) {
    const int64_t ov = j.off_v[I], op = j.off_p[I];
    const int kv = (int)(j.off_v[I + 1] - ov), kp = (int)(j.off_p[I + 1] - op);
    const int kvd = kv * D;
    const double* acc = j.w_cc + ov * D * D;  // this point's curl curl weights
    if (!j.bflag[I]) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int64_t r = I * D + c, s = j.row_ptr[r];
        for (int e = lane; e < kvd; e += 32) {
          const int q = e / D, cc = e - q * D;
          const int pv = j.order_v[ov + q];
          j.col[s + e] = j.idx_v[ov + pv] * D + cc;
          j.val[s + e] = __dmul_rn(nu, acc[(int64_t)c * kvd + pv * D + cc]);
        }
        for (int e = lane; e < kp; e += 32) {
          const int pp = j.order_p[op + e];
          j.col[s + kvd + e] = (int32_t)(nd + j.idx_p[op + pp]);
          j.val[s + kvd + e] = j.w_grad[op * D + (int64_t)c * kp + pp];
        }
      }
      // Laplacian row: the staggered stencil on its own list, else the
      // scalar one on the pressure list
      const int64_t s = j.row_ptr[nd + I];
      const bool stag = j.off_s != nullptr;
      const int64_t ol = stag ? j.off_s[I] : op;
      const int kl = stag ? (int)(j.off_s[I + 1] - ol) : kp;
      const int16_t* ord = stag ? j.order_s : j.order_p;
      const int32_t* idx = stag ? j.idx_s : j.idx_p;
      const double* wl = stag ? j.w_stag : j.w_lap;
      for (int e = lane; e < kl; e += 32) {
        const int pp = ord[ol + e];
        j.col[s + e] = (int32_t)(nd + idx[ol + pp]);
        j.val[s + e] = wl[ol + pp];
      }
      if (lane == 0) {
        j.col[s + kl] = (int32_t)(nd + n);
        j.val[s + kl] = 1.0;
      }
    } else {
      if (lane < D) {
        const int64_t r = I * D + lane, s = j.row_ptr[r];
        j.col[s] = (int32_t)r;
        j.val[s] = 1.0;
      }
      const double beta = j.beta[I * j.beta_stride + j.beta_col];
      double nrm[D];
#pragma unroll
      for (int c = 0; c < D; ++c) nrm[c] = j.normals[c * n + I];
      const int64_t s = j.row_ptr[nd + I];
      for (int e = lane; e < kvd; e += 32) {
        const int q = e / D, cc = e - q * D;
        const int pv = j.order_v[ov + q];
        const int64_t w0 = (int64_t)pv * D + cc;
        // n . a, evaluated ((n_0 a_0) + (n_1 a_1)) + (n_2 a_2)
        double nda = __dmul_rn(nrm[0], acc[w0]);
#pragma unroll
        for (int c = 1; c < D; ++c) nda = __dadd_rn(nda, __dmul_rn(nrm[c], acc[(int64_t)c * kvd + w0]));
        j.col[s + e] = j.idx_v[ov + pv] * D + cc;
        j.val[s + e] = -__dmul_rn(nu, __dmul_rn(beta, nda));
      }
      for (int e = lane; e < kp; e += 32) {
        const int pp = j.order_p[op + e];
        j.col[s + kvd + e] = (int32_t)(nd + j.idx_p[op + pp]);
        j.val[s + kvd + e] = j.w_lap[op + pp];
      }
      if (lane == 0) {
        j.col[s + kvd + kp] = (int32_t)(nd + n);
        j.val[s + kvd + kp] = 1.0;
      }
    }
  }
}

__global__ void stokes_last_row_kernel(int64_t nd, int64_t n, const int64_t* __restrict__ row_ptr,
                                       int32_t* __restrict__ col, double* __restrict__ val) {
  const int64_t s = row_ptr[nd + n];
  for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < n; J += (int64_t)gridDim.x * blockDim.x) {
    col[s + J] = (int32_t)(nd + J);
    val[s + J] = 1.0;
  }
}

__global__ void stokes_rhs_kernel(StokesJob j, const double* __restrict__ f, const double* __restrict__ w,
                                  const double* __restrict__ div_f, double* __restrict__ b) {
  const int d = j.dim;
  const int64_t n = j.n, nd = n * d;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < n; I += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = j.bflag[I] != 0;
    for (int c = 0; c < d; ++c) b[I * d + c] = bnd ? w[c * n + I] : f[c * n + I];
    if (bnd) {
      double nf = __dmul_rn(j.normals[I], f[I]);
      for (int c = 1; c < d; ++c) nf = __dadd_rn(nf, __dmul_rn(j.normals[c * n + I], f[c * n + I]));
      b[nd + I] = __dsub_rn(div_f[I], __dmul_rn(j.beta[I * j.beta_stride + j.beta_col], nf));
    } else {
      b[nd + I] = div_f[I];
    }
    if (I == 0) b[nd + n] = 0.0;
  }
}

// y = A x, FP64.  Pass 1: eight lanes per row (they stride the row, then a
// butterfly); rows longer than kLongRow (the zero-mean row of the Stokes
// system holds every pressure column) are queued instead.  When at most
// kLongSplitRows rows are queued, every one is cut into kLongSlices slices,
// one block each (pass 2), and the slice sums are added in slice order
// (pass 3); otherwise every queued row takes one whole block (pass 2').
// Which path a row takes depends on the number of long rows, not on the
// queue order, and each path sums in a fixed order: repeated calls give the
// same bits.
constexpr int64_t kLongRow = 8192;
constexpr int kLongSplitRows = 64;
constexpr int kLongSlices = 128;
constexpr int kSpmvBlock = 256;

// Eight lanes per row: on rows of a few dozen to a few hundred entries the
// FP64 adds of the final reduction (three levels, shared by four rows per
// warp instruction) stay small next to the one FMA per entry -- FP64 runs at
// 1/64 of the FP32 rate on this GPU.
constexpr int kRowLanes = 8;

__global__ void csr_spmv_kernel(int64_t n_rows, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                                int32_t* __restrict__ long_rows, int32_t* __restrict__ n_long) {
  const int sub = threadIdx.x & (kRowLanes - 1);
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / kRowLanes;
  // every lane of the warp runs the same number of iterations (the shuffles
  // below need the whole warp)
  const int64_t r0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kRowLanes;
  const int64_t warp_first = r0 - ((threadIdx.x & 31) / kRowLanes);
  for (int64_t base = warp_first; base < n_rows; base += stride) {
    const int64_t r = base + ((threadIdx.x & 31) / kRowLanes);
    double s = 0.0;
    bool store = false;
    if (r < n_rows) {
      const int64_t a = row_ptr[r], e = row_ptr[r + 1];
      if (e - a > kLongRow) {
        if (sub == 0) long_rows[atomicAdd(n_long, 1)] = (int32_t)r;
      } else {
        for (int64_t p = a + sub; p < e; p += kRowLanes) s = fma(val[p], x[col[p]], s);
        store = true;
      }
    }
    for (int o = kRowLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, kRowLanes);
    if (store && sub == 0) y[r] = s;
  }
}

// fixed-order sum of a value per thread over the block (kSpmvBlock threads);
// the result is valid in thread 0
__device__ __forceinline__ double block_sum(double s, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < kSpmvBlock / 32 ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// sum of val[p] x[col[p]] over [p0, p1) by the block, four accumulators per
// thread (memory-level parallelism), fixed order
__device__ __forceinline__ double block_dot(int64_t p0, int64_t p1, const int32_t* __restrict__ col,
                                            const double* __restrict__ val, const double* __restrict__ x,
                                            double* part) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t p = p0 + threadIdx.x;
  for (; p + 3 * kSpmvBlock < p1; p += 4 * kSpmvBlock) {
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(val[p + u * kSpmvBlock], x[col[p + u * kSpmvBlock]], acc[u]);
  }
  for (int u = 0; p < p1; p += kSpmvBlock, ++u) acc[u] = fma(val[p], x[col[p]], acc[u]);
  return block_sum((acc[0] + acc[1]) + (acc[2] + acc[3]), part);
}

__global__ void __launch_bounds__(kSpmvBlock) csr_spmv_long_kernel(const int64_t* __restrict__ row_ptr,
                                                                   const int32_t* __restrict__ col,
                                                                   const double* __restrict__ val,
                                                                   const double* __restrict__ x, double* __restrict__ y,
                                                                   const int32_t* __restrict__ long_rows,
                                                                   const int32_t* __restrict__ n_long,
                                                                   double* __restrict__ partial) {
  __shared__ double part[kSpmvBlock / 32];
  const int cnt = *n_long;
  if (cnt <= kLongSplitRows) {
    // block b takes slice b % kLongSlices of queued row b / kLongSlices, ...
    for (int task = blockIdx.x; task < cnt * kLongSlices; task += gridDim.x) {
      const int i = task / kLongSlices, sl = task % kLongSlices;
      const int64_t r = long_rows[i];
      const int64_t a = row_ptr[r], len = row_ptr[r + 1] - a;
      const double s = block_dot(a + len * sl / kLongSlices, a + len * (sl + 1) / kLongSlices, col, val, x, part);
      if (threadIdx.x == 0) partial[task] = s;
    }
  } else {
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
      const int64_t r = long_rows[i];
      const double s = block_dot(row_ptr[r], row_ptr[r + 1], col, val, x, part);
      if (threadIdx.x == 0) y[r] = s;
    }
  }
}

__global__ void csr_spmv_long_finish_kernel(double* __restrict__ y, const int32_t* __restrict__ long_rows,
                                            const int32_t* __restrict__ n_long, const double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = *n_long;
  if (cnt > kLongSplitRows) return;
  for (int i = warp; i < cnt; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int b = lane; b < kLongSlices; b += 32) s += partial[(int64_t)i * kLongSlices + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[long_rows[i]] = s;
  }
}

}  // namespace

cudaError_t launch_stokes_rowlen(const Launch& L, const StokesJob& j) {
  stokes_rowlen_kernel<<<grid_for(j.n, 256), 256, 0, L.stream>>>(j);
  *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t launch_stokes_fill(const Launch& L, const StokesJob& j) {
  int64_t blocks = (j.n + kStokesWarps - 1) / kStokesWarps;
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  if (j.dim == 2)
    stokes_fill_kernel<2><<<(unsigned)blocks, kStokesWarps * 32, 0, L.stream>>>(j);
  else
    stokes_fill_kernel<3><<<(unsigned)blocks, kStokesWarps * 32, 0, L.stream>>>(j);
  stokes_last_row_kernel<<<grid_for(j.n, 256), 256, 0, L.stream>>>(j.n * j.dim, j.n, j.row_ptr, j.col, j.val);
  *L.counter += 2;
  return cudaGetLastError();
}

cudaError_t launch_stokes_rhs(const Launch& L, const StokesJob& j, const double* f, const double* w,
                              const double* div_f, double* b) {
  stokes_rhs_kernel<<<grid_for(j.n, 256), 256, 0, L.stream>>>(j, f, w, div_f, b);
  *L.counter += 1;
  return cudaGetLastError();
}

size_t csr_spmv_partial_elems() { return (size_t)kLongSplitRows * kLongSlices; }

cudaError_t launch_csr_spmv(const Launch& L, int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                            const double* val, const double* x, double* y, int32_t* long_rows, int32_t* n_long,
                            double* partial) {
  if (n_rows <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(n_long, 0, sizeof(int32_t), L.stream);
  if (e != cudaSuccess) return e;
  csr_spmv_kernel<<<grid_for(n_rows * kRowLanes, 256), 256, 0, L.stream>>>(n_rows, row_ptr, col, val, x, y,
                                                                              long_rows, n_long);
  csr_spmv_long_kernel<<<4 * device_sm_count(), kSpmvBlock, 0, L.stream>>>(row_ptr, col, val, x, y, long_rows, n_long, partial);
  csr_spmv_long_finish_kernel<<<1, 512, 0, L.stream>>>(y, long_rows, n_long, partial);
  *L.counter += 3;
  return cudaGetLastError();
}

}  // namespace gmls
