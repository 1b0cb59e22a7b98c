// stencil.cu -- per-target GMLS stencils on the device.
//
// For each target x_T with neighbours x_j (Sec. 2.1) and support eps:
//   1. B = sqrt(W) P with P_{j,i} = p_i((x_j - x_T)/eps)  (Eqs. matrix-P,
//      matrix-W, basis-functions-3d; divergence-free basis of Sec. 2.2 with
//      rows (j, component)), W = (1 - r/eps)_+^p (Eq. kernel);
//   2. Householder QR  B = Q R  (the local solve of Eqs. matrix-A, matrix-B,
//      vector-c done without forming P^T W P);
//   3. functional rows lambda_i = L(p_i)(x_T)  (Sec. 2.5);
//   4. s = Q [R^{-T} lambda^T; 0], so that w = sqrt(W) s = W P (P^T W P)^{-1}
//      lambda^T  (Eq. polynomial-approximation-derivative);
//   5. optionally (FP32 path) iterative refinement of the augmented system
//      [[I, B], [B^T, 0]] [s; -y] = [0; lambda^T] with FP64 residuals and FP32
//      corrections (Bjorck's method); targets that do not converge are queued
//      for the FP64 path;
//   6. Neumann targets (Sec. 2.3) first eliminate the constraint
//      F^T c = h, F = grad p(x_T)^T n, with a reflector H_F: the least-squares
//      problem runs on B H_F without the pivot column, and the coefficient of h
//      is beta = (lambda~_piv - w^T p~_piv) / rho.
//
// One group of G warps (G = 1, 2 or 4; 128-thread blocks) owns one target at a
// time; its tiles live in shared memory, column-major with leading dimension
// ld.  The block loops over a work list (persistent).
#include <cuda_runtime.h>

#include "basis_tables.cuh"
#include "gmls_internal.cuh"

namespace gmls {

constexpr int kBlock = 128;

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct Lay {
  size_t A, B64, tau, dots, sw, lam, S, Y, Z, D, pt, misc, total;
};

__host__ __device__ inline Lay make_lay(int ld, int nmax, bool refine, int tqs) {
  Lay l;
  size_t o = 0;
  l.A = o;
  o += align16((size_t)nmax * ld * tqs);
  l.B64 = o;
  if (refine) o += align16((size_t)nmax * ld * 8);
  l.tau = o;
  o += align16((size_t)nmax * tqs);
  l.dots = o;
  o += align16((size_t)nmax * tqs);
  l.sw = o;
  o += align16((size_t)ld * 8);
  l.lam = o;
  o += align16((size_t)kMaxSolveRows * nmax * 8);
  l.S = o;
  o += align16((size_t)kMaxSolveRows * ld * 8);
  l.Y = o;
  o += align16((size_t)kMaxSolveRows * nmax * 8);
  l.Z = o;
  o += align16((size_t)kMaxSolveRows * ld * tqs);
  l.D = o;
  o += align16((size_t)kMaxSolveRows * nmax * tqs);
  l.pt = o;
  o += align16((size_t)ld * 8);
  l.misc = o;
  o += 256;
  l.total = o;
  return l;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

__device__ __forceinline__ void group_sync(int gid, int nthr) {
  if (nthr == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(nthr) : "memory");
}

template <typename T>
struct Eps;
template <>
struct Eps<float> {
  static constexpr double u = 5.9604644775390625e-08;
};
template <>
struct Eps<double> {
  static constexpr double u = 1.1102230246251565e-16;
};

struct Group {
  int gid, nthr, tid, wg, G, lane;
};

// ---------------------------------------------------------------- QR (in TQ)
// Householder QR of the M x n tile A (column-major, leading dimension ld).
// Column k below the diagonal keeps v_k (v_k[k] = 1 implied), tau[k] its scale.
template <typename TQ>
__device__ void tile_qr(const Group& g, TQ* A, int ld, int M, int n, TQ* tau, TQ* dots) {
  for (int k = 0; k < n; ++k) {
    TQ* a = A + (size_t)k * ld;
    if (g.wg == 0) {
      TQ sig = 0;
      for (int r = k + 1 + g.lane; r < M; r += 32) sig += a[r] * a[r];
      sig = warp_sum(sig);
      TQ alpha = a[k];
      if (sig == TQ(0)) {
        if (g.lane == 0) tau[k] = 0;
      } else {
        TQ nrm = sqrt(alpha * alpha + sig);
        TQ beta = alpha >= TQ(0) ? -nrm : nrm;
        TQ scale = TQ(1) / (alpha - beta);
        for (int r = k + 1 + g.lane; r < M; r += 32) a[r] *= scale;
        __syncwarp();
        if (g.lane == 0) {
          tau[k] = (beta - alpha) / beta;
          a[k] = beta;
        }
      }
    }
    group_sync(g.gid, g.nthr);
    const TQ tk = tau[k];
    if (tk != TQ(0) && k + 1 < n) {
      for (int jc = k + 1 + g.wg; jc < n; jc += g.G) {
        const TQ* aj = A + (size_t)jc * ld;
        TQ s = (g.lane == 0) ? aj[k] : TQ(0);
        for (int r = k + 1 + g.lane; r < M; r += 32) s += a[r] * aj[r];
        s = warp_sum(s);
        if (g.lane == 0) dots[jc] = s * tk;
      }
      group_sync(g.gid, g.nthr);
      const int rows = M - k;
      const int total = (n - k - 1) * rows;
      for (int e = g.tid; e < total; e += g.nthr) {
        const int jc = k + 1 + e / rows;
        const int r = k + e % rows;
        const TQ v = (r == k) ? TQ(1) : a[r];
        A[(size_t)jc * ld + r] -= dots[jc] * v;
      }
      group_sync(g.gid, g.nthr);
    }
  }
}

// y = R^{-T} b for the L rows (b and y: [L][nmax]); one warp per row.
template <typename TQ, typename TB>
__device__ void solve_rt(const Group& g, const TQ* A, int ld, int n, int L, int nmax, const TB* b, TQ* y) {
  for (int l = g.wg; l < L; l += g.G) {
    const TB* bl = b + l * nmax;
    TQ* yl = y + l * nmax;
    for (int i = 0; i < n; ++i) {
      const TQ* ri = A + (size_t)i * ld;  // column i of R: R[p][i] = ri[p], p <= i
      TQ s = 0;
      for (int p = g.lane; p < i; p += 32) s += ri[p] * yl[p];
      s = warp_sum(s);
      if (g.lane == 0) yl[i] = (TQ(bl[i]) - s) / ri[i];
      __syncwarp();
    }
  }
}

// x = R^{-1} b in place on [L][nmax] rows; one warp per row.
template <typename TQ>
__device__ void solve_r(const Group& g, const TQ* A, int ld, int n, int L, int nmax, TQ* x) {
  for (int l = g.wg; l < L; l += g.G) {
    TQ* xl = x + l * nmax;
    for (int i = n - 1; i >= 0; --i) {
      TQ s = 0;
      for (int p = i + 1 + g.lane; p < n; p += 32) s += A[(size_t)p * ld + i] * xl[p];
      s = warp_sum(s);
      if (g.lane == 0) xl[i] = (xl[i] - s) / A[(size_t)i * ld + i];
      __syncwarp();
    }
  }
}

// z <- Q z (reverse reflector order) or z <- Q^T z (forward order) for L rows
// z: [L][ld]; one warp per row.
template <typename TQ, bool TRANS>
__device__ void apply_q(const Group& g, const TQ* A, int ld, int M, int n, const TQ* tau, int L, TQ* z) {
  for (int l = g.wg; l < L; l += g.G) {
    TQ* zl = z + (size_t)l * ld;
    for (int s = 0; s < n; ++s) {
      const int k = TRANS ? s : n - 1 - s;
      const TQ tk = tau[k];
      if (tk == TQ(0)) continue;
      const TQ* a = A + (size_t)k * ld;
      TQ d = (g.lane == 0) ? zl[k] : TQ(0);
      for (int r = k + 1 + g.lane; r < M; r += 32) d += a[r] * zl[r];
      d = warp_sum(d) * tk;
      for (int r = k + 1 + g.lane; r < M; r += 32) zl[r] -= d * a[r];
      if (g.lane == 0) zl[k] -= d;
      __syncwarp();
    }
  }
}

template <typename TQ, bool REFINE>
__global__ void __launch_bounds__(kBlock) stencil_kernel(StencilJob j) {
  extern __shared__ __align__(16) unsigned char smem[];
  Group g;
  g.G = j.warps_per_target;
  g.nthr = 32 * g.G;
  g.gid = (threadIdx.x >> 5) / g.G;
  g.wg = (threadIdx.x >> 5) % g.G;
  g.tid = threadIdx.x % g.nthr;
  g.lane = threadIdx.x & 31;
  const int groups_per_block = kBlock / g.nthr;
  const Lay lay = make_lay(j.ld, j.nmax, REFINE, (int)sizeof(TQ));
  unsigned char* base = smem + (size_t)g.gid * lay.total;
  TQ* A = reinterpret_cast<TQ*>(base + lay.A);
  double* B64 = REFINE ? reinterpret_cast<double*>(base + lay.B64) : nullptr;
  TQ* tau = reinterpret_cast<TQ*>(base + lay.tau);
  TQ* dots = reinterpret_cast<TQ*>(base + lay.dots);
  double* sw = reinterpret_cast<double*>(base + lay.sw);
  double* lam = reinterpret_cast<double*>(base + lay.lam);
  double* S = reinterpret_cast<double*>(base + lay.S);
  double* Y = reinterpret_cast<double*>(base + lay.Y);
  TQ* Z = reinterpret_cast<TQ*>(base + lay.Z);
  TQ* D = reinterpret_cast<TQ*>(base + lay.D);
  double* pt = reinterpret_cast<double*>(base + lay.pt);
  double* misc = reinterpret_cast<double*>(base + lay.misc);  // [0] rho, [1..L] lambda~_piv, [8] flags
  int* imisc = reinterpret_cast<int*>(misc + 8);

  const int ld = j.ld, nmax = j.nmax, L = j.L, dim = j.dim, nc = j.nc;
  const int64_t n_items = j.items ? (int64_t)(*j.n_items) : j.n_tgt;

  for (int64_t it = (int64_t)blockIdx.x * groups_per_block + g.gid; it < n_items;
       it += (int64_t)gridDim.x * groups_per_block) {
    const int64_t to = j.items ? (int64_t)j.items[it] : it;
    const int64_t t = j.tgt[to];
    const int64_t o0 = j.off[to];
    const int k = (int)(j.off[to + 1] - o0);
    const int32_t* nbr = j.idx + o0;
    const double eps = j.eps[to];
    const int m = j.degree_pt ? (int)j.degree_pt[to] : j.degree;
    const int nb = gmls_gen::basis_size(j.kind, dim, m);
    const int M = k * nc;
    const bool neu = j.neumann && j.bflag && j.bflag[t] && j.normals && j.kind == GMLS_BASIS_SCALAR;
    const int n = neu ? nb - 1 : nb;
    uint8_t st = j.nbr_status ? j.nbr_status[to] : 0;
    if (j.fallback_run)  // FP64 redo of an FP32 target: keep why it was redone
      st |= GMLS_T_FP64_FALLBACK | (j.status[to] & (GMLS_T_ILL_CONDITIONED | GMLS_T_REFINE_NOT_CONVERGED));
    bool skip = (st & GMLS_T_TOO_FEW_NEIGHBOURS) || k <= 0 || nb <= 0 || M > ld || nb > nmax || !(eps > 0.0);
    if (!skip && M < n) {
      st |= GMLS_T_RANK_DEFICIENT;
      skip = true;
    }
    const double inv_eps = skip ? 0.0 : 1.0 / eps;

    if (!skip) {
      // ---- 1. sqrt(W) P, rows (neighbour, component)
      double* Bd = REFINE ? B64 : reinterpret_cast<double*>(A);
      double xT[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < dim; ++c) xT[c] = j.x[c * j.n + t];
      for (int q = g.tid; q < k; q += g.nthr) {
        const int32_t jj = nbr[q];
        double xi[3] = {0.0, 0.0, 0.0};
        double r2 = 0.0;
        for (int c = 0; c < dim; ++c) {
          double dx = j.x[c * j.n + jj] - xT[c];
          xi[c] = dx * inv_eps;
          r2 += dx * dx;
        }
        const double u = 1.0 - sqrt(r2) * inv_eps;
        const double s = (u > 0.0) ? (j.wpow == 4.0 ? u * u : pow(u, 0.5 * j.wpow)) : 0.0;
        gmls_gen::eval_basis<double>(j.kind, dim, m, xi, Bd + q * nc, ld, s);
        for (int c = 0; c < nc; ++c) sw[q * nc + c] = s;
      }
      // ---- 3. functional rows lambda (before Neumann)
      for (int e = g.tid; e < L * nb; e += g.nthr) {
        const int l = e / nb, i = e % nb;
        double f = 1.0;
        for (int p = 0; p < j.lam_order[l]; ++p) f *= inv_eps;
        lam[l * nmax + i] = gmls_gen::lam_coef(j.kind, dim, m, j.lam_fn[l], j.lam_row[l], i) * f;
      }
      group_sync(g.gid, g.nthr);

      // ---- 6. Neumann: reflect the linear columns (indices 1..dim), move the
      //         pivot column to the end, and keep it aside as p~
      if (neu) {
        double nv[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0};
        double fn = 0.0;
        int piv = 0;
        for (int c = 0; c < dim; ++c) {
          nv[c] = j.normals[c * j.n + t];
          fn += nv[c] * nv[c];
          if (fabs(nv[c]) > fabs(nv[piv])) piv = c;
        }
        fn = sqrt(fn) * inv_eps;
        const double rho = nv[piv] >= 0.0 ? -fn : fn;
        double vv = 0.0;
        for (int c = 0; c < dim; ++c) {
          v[c] = nv[c] * inv_eps - (c == piv ? rho : 0.0);
          vv += v[c] * v[c];
        }
        const double two_vv = 2.0 / vv;
        for (int r = g.tid; r < M; r += g.nthr) {
          double d = 0.0;
          for (int c = 0; c < dim; ++c) d += Bd[(size_t)(1 + c) * ld + r] * v[c];
          d *= two_vv;
          for (int c = 0; c < dim; ++c) Bd[(size_t)(1 + c) * ld + r] -= d * v[c];
          // swap pivot column with the last column
          const double pc = Bd[(size_t)(1 + piv) * ld + r];
          Bd[(size_t)(1 + piv) * ld + r] = Bd[(size_t)(nb - 1) * ld + r];
          Bd[(size_t)(nb - 1) * ld + r] = pc;
          pt[r] = pc;
        }
        if (g.tid < L) {
          const int l = g.tid;
          double* ll = lam + l * nmax;
          double d = 0.0;
          for (int c = 0; c < dim; ++c) d += ll[1 + c] * v[c];
          d *= two_vv;
          for (int c = 0; c < dim; ++c) ll[1 + c] -= d * v[c];
          const double lp = ll[1 + piv];
          ll[1 + piv] = ll[nb - 1];
          ll[nb - 1] = lp;
          misc[1 + l] = lp;
        }
        if (g.tid == 0) misc[0] = rho;
        group_sync(g.gid, g.nthr);
      }

      if (REFINE) {
        for (int e = g.tid; e < n * M; e += g.nthr) {
          const int i = e / M, r = e % M;
          A[(size_t)i * ld + r] = (TQ)B64[(size_t)i * ld + r];
        }
        group_sync(g.gid, g.nthr);
      }

      // ---- 2. QR
      tile_qr<TQ>(g, A, ld, M, n, tau, dots);
      if (g.wg == 0) {
        TQ rmax = 0, rmin = TQ(3.0e38);
        for (int i = g.lane; i < n; i += 32) {
          TQ r = fabs(A[(size_t)i * ld + i]);
          rmax = r > rmax ? r : rmax;
          rmin = r < rmin ? r : rmin;
        }
        rmax = warp_max(rmax);
        rmin = -warp_max(-rmin);
        if (g.lane == 0) {
          int fl = 0;
          // rank deficiency is judged against FP64 roundoff (a property of the
          // problem); an FP32 factor with a large ratio is caught as ill-conditioned
          if (!((double)rmin > 64.0 * n * Eps<double>::u * (double)rmax)) fl |= GMLS_T_RANK_DEFICIENT;
          if (!((double)rmin * 1e6 >= (double)rmax)) fl |= GMLS_T_ILL_CONDITIONED;
          imisc[0] = fl;
        }
      }
      group_sync(g.gid, g.nthr);
      st |= (uint8_t)imisc[0];

      // ---- 4. s = Q [R^{-T} lambda; 0]
      solve_rt<TQ, double>(g, A, ld, n, L, nmax, lam, D);
      group_sync(g.gid, g.nthr);
      for (int e = g.tid; e < L * M; e += g.nthr) {
        const int l = e / M, r = e % M;
        Z[(size_t)l * ld + r] = (r < n) ? D[l * nmax + r] : TQ(0);
      }
      group_sync(g.gid, g.nthr);
      apply_q<TQ, false>(g, A, ld, M, n, tau, L, Z);
      group_sync(g.gid, g.nthr);
      for (int e = g.tid; e < L * M; e += g.nthr) {
        const int l = e / M, r = e % M;
        S[(size_t)l * ld + r] = (double)Z[(size_t)l * ld + r];
      }
      int used_iters = 0;
      if (REFINE) {
        // y = R^{-1} R^{-T} lambda (the least-squares coefficients), FP64 copy
        solve_r<TQ>(g, A, ld, n, L, nmax, D);
        group_sync(g.gid, g.nthr);
        for (int e = g.tid; e < L * n; e += g.nthr) Y[(e / n) * nmax + e % n] = (double)D[(e / n) * nmax + e % n];
        group_sync(g.gid, g.nthr);
        bool conv = (st & GMLS_T_ILL_CONDITIONED) != 0;  // ill-conditioned: straight to FP64
        double prev = 0.0;
        const int maxit = j.max_refine;
        for (int iter = 0; iter < maxit && !conv; ++iter) {
          // f = B y - s (into Z), FP64 residual rounded to TQ for the correction
          for (int e = g.tid; e < L * M; e += g.nthr) {
            const int l = e / M, r = e % M;
            double acc = -S[(size_t)l * ld + r];
            const double* yl = Y + l * nmax;
            for (int i = 0; i < n; ++i) acc = fma(B64[(size_t)i * ld + r], yl[i], acc);
            Z[(size_t)l * ld + r] = (TQ)acc;
          }
          // g = lambda - B^T s (into D), one warp per (l, i)
          for (int p = g.wg; p < L * n; p += g.G) {
            const int l = p / n, i = p % n;
            const double* bi = B64 + (size_t)i * ld;
            const double* sl = S + (size_t)l * ld;
            double acc = 0.0;
            for (int r = g.lane; r < M; r += 32) acc = fma(bi[r], sl[r], acc);
            acc = warp_sum(acc);
            if (g.lane == 0) D[l * nmax + i] = (TQ)(lam[l * nmax + i] - acc);
          }
          group_sync(g.gid, g.nthr);
          // d = Q^T f; a = R^{-T} g; dy = R^{-1}(a - d_1); ds = Q [a; d_2]
          apply_q<TQ, true>(g, A, ld, M, n, tau, L, Z);
          group_sync(g.gid, g.nthr);
          // a into D (in place forward substitution from g)
          solve_rt<TQ, TQ>(g, A, ld, n, L, nmax, D, D);
          group_sync(g.gid, g.nthr);
          // dy = R^{-1}(a - d_1) into the first n entries of Z after saving a
          for (int e = g.tid; e < L * n; e += g.nthr) {
            const int l = e / n, i = e % n;
            const TQ a = D[l * nmax + i];
            const TQ d1 = Z[(size_t)l * ld + i];
            D[l * nmax + i] = a - d1;  // becomes dy after the back substitution
            Z[(size_t)l * ld + i] = a;
          }
          group_sync(g.gid, g.nthr);
          solve_r<TQ>(g, A, ld, n, L, nmax, D);
          apply_q<TQ, false>(g, A, ld, M, n, tau, L, Z);
          group_sync(g.gid, g.nthr);
          // s += ds, y += dy; norms
          double dmax = 0.0, smax = 0.0;
          for (int e = g.tid; e < L * M; e += g.nthr) {
            const int l = e / M, r = e % M;
            const double ds = (double)Z[(size_t)l * ld + r];
            const double sv = S[(size_t)l * ld + r] + ds;
            S[(size_t)l * ld + r] = sv;
            dmax = fmax(dmax, fabs(ds));
            smax = fmax(smax, fabs(sv));
          }
          for (int e = g.tid; e < L * n; e += g.nthr) Y[(e / n) * nmax + e % n] += (double)D[(e / n) * nmax + e % n];
          dmax = warp_max(dmax);
          smax = warp_max(smax);
          if (g.G > 1) {
            if (g.lane == 0) {
              misc[16 + 2 * g.wg] = dmax;
              misc[17 + 2 * g.wg] = smax;
            }
            group_sync(g.gid, g.nthr);
            dmax = 0.0;
            smax = 0.0;
            for (int w = 0; w < g.G; ++w) {
              dmax = fmax(dmax, misc[16 + 2 * w]);
              smax = fmax(smax, misc[17 + 2 * w]);
            }
          }
          used_iters = iter + 1;
          // error after this correction ~ |ds| * (contraction |ds|/|ds_prev|)
          const double est = (iter == 0) ? dmax : dmax * fmin(1.0, dmax / fmax(prev, 1e-300));
          conv = est <= j.tol * smax;
          prev = dmax;
          group_sync(g.gid, g.nthr);
        }
        if (!conv || (st & GMLS_T_ILL_CONDITIONED)) {
          st |= (st & GMLS_T_ILL_CONDITIONED) ? 0 : GMLS_T_REFINE_NOT_CONVERGED;
          if (g.tid == 0) {
            int slot = atomicAdd(j.fb_count, 1);
            j.fb_items[slot] = (int32_t)to;
          }
        }
      }

      // ---- Neumann coefficient of h: beta = (lambda~_piv - s^T p~) / rho
      if (neu && j.beta) {
        for (int l = g.wg; l < L; l += g.G) {
          double acc = 0.0;
          for (int r = g.lane; r < M; r += 32) acc += S[(size_t)l * ld + r] * pt[r];
          acc = warp_sum(acc);
          if (g.lane == 0) j.beta[to * L + l] = (misc[1 + l] - acc) / misc[0];
        }
      } else if (j.beta) {
        for (int l = g.tid; l < L; l += g.nthr) j.beta[to * L + l] = 0.0;
      }
      if (g.tid == 0 && j.iters) j.iters[to] = (uint8_t)used_iters;
      group_sync(g.gid, g.nthr);
    }

    // ---- store w = sqrt(W) s in [row][neighbour][component] per functional
    for (int f = 0; f < j.nout; ++f) {
      const int R = j.out_rows[f], C = j.out_ncomp[f], src = j.out_src[f];
      const double sgn = (double)j.out_sign[f];
      double* w = j.out_w[f] + o0 * (int64_t)R * C;
      const int total = R * k * C;
      for (int e = g.tid; e < total; e += g.nthr) {
        double val = 0.0;
        if (!skip && src >= 0) {
          const int r = e / (k * C), rem = e % (k * C), q = rem / C, c = rem % C;
          if (j.out_fn[f] == GMLS_F_DIV) {  // scalar basis: component c uses the d/dx_c row
            val = S[(size_t)(src + c) * ld + q] * sw[q];
          } else {
            const int row = q * nc + c;
            val = sgn * S[(size_t)(src + r) * ld + row] * sw[row];
          }
        }
        w[e] = val;
      }
    }
    if (g.tid == 0) {
      j.status[to] = st;
      if (skip && j.iters) j.iters[to] = 0;
    }
    if (skip && j.beta)
      for (int l = g.tid; l < L; l += g.nthr) j.beta[to * L + l] = 0.0;
    group_sync(g.gid, g.nthr);
  }
}

size_t stencil_smem_bytes(const StencilJob& j, bool fp32_refine) {
  const Lay l = make_lay(j.ld, j.nmax, fp32_refine, fp32_refine ? 4 : 8);
  return l.total * (size_t)(kBlock / (32 * j.warps_per_target));
}

cudaError_t launch_stencils(const Launch& L, const StencilJob& j, bool fp32_refine, int grid_blocks) {
  const size_t smem = stencil_smem_bytes(j, fp32_refine);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (fp32_refine) {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    stencil_kernel<float, true><<<grid_blocks, kBlock, smem, L.stream>>>(j);
  } else {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    stencil_kernel<double, false><<<grid_blocks, kBlock, smem, L.stream>>>(j);
  }
  *L.counter += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ CSR
// Warp per target: order the neighbours by particle id once (bitonic sort of
// (id, position) pairs in shared memory) and write every row of the target.
constexpr int kCsrWarps = 4;

__global__ void __launch_bounds__(kCsrWarps * 32) csr_kernel(CsrJob j) {
  __shared__ int32_t sid[kCsrWarps][kMaxK];
  __shared__ int16_t spos[kCsrWarps][kMaxK];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* ids = sid[w];
  int16_t* pos = spos[w];
  for (int64_t t = (int64_t)blockIdx.x * kCsrWarps + w; t < j.n_tgt; t += (int64_t)gridDim.x * kCsrWarps) {
    const int64_t o = j.off[t];
    const int k = (int)(j.off[t + 1] - o);
    int n2 = 1;
    while (n2 < k) n2 <<= 1;
    for (int i = lane; i < n2; i += 32) {
      ids[i] = (i < k) ? j.idx[o + i] : INT_MAX;
      pos[i] = (int16_t)i;
    }
    __syncwarp();
    for (int size = 2; size <= n2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = lane; i < (n2 >> 1); i += 32) {
          int a = 2 * stride * (i / stride) + (i % stride), b = a + stride;
          bool asc = (a & size) == 0;
          int32_t ia = ids[a], ib = ids[b];
          if ((ib < ia) == asc) {
            ids[a] = ib;
            ids[b] = ia;
            int16_t pa = pos[a];
            pos[a] = pos[b];
            pos[b] = pa;
          }
        }
        __syncwarp();
      }
    }
    const int C = j.nc, rowlen = k * C;
    const int64_t base = o * (int64_t)j.rows * C;
    for (int r = 0; r < j.rows; ++r) {
      const int64_t row = t * j.rows + r;
      const int64_t start = base + (int64_t)r * rowlen;
      if (lane == 0) j.row_ptr[row] = start;
      const double* wr = j.w + base + (int64_t)r * rowlen;
      for (int e = lane; e < rowlen; e += 32) {
        const int q = e / C, c = e % C;
        j.col[start + e] = ids[q] * C + c;
        j.val[start + e] = wr[pos[q] * C + c];
      }
    }
    if (t == j.n_tgt - 1 && lane == 0) j.row_ptr[j.n_tgt * j.rows] = base + (int64_t)j.rows * rowlen;
    __syncwarp();
  }
}

cudaError_t launch_csr(const Launch& L, const CsrJob& j) {
  if (j.n_tgt == 0) {
    cudaMemsetAsync(j.row_ptr, 0, sizeof(int64_t), L.stream);
    return cudaGetLastError();
  }
  int64_t blocks = (j.n_tgt + kCsrWarps - 1) / kCsrWarps;
  if (blocks > 152 * 16) blocks = 152 * 16;
  csr_kernel<<<(unsigned)blocks, kCsrWarps * 32, 0, L.stream>>>(j);
  *L.counter += 1;
  return cudaGetLastError();
}

}  // namespace gmls
