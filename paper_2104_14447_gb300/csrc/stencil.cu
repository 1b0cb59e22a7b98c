// stencil.cu -- per-target GMLS stencils, shared-memory tiles, any shape.
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
//   5. FP32 path: refinement of the augmented system [[I, B], [B^T, 0]]
//      [s; -y] = [0; lambda^T] (Bjorck) with float-float residuals and FP32
//      corrections; targets that miss the tolerance go to the FP64 redo list;
//   6. Neumann targets (Sec. 2.3) first eliminate the constraint
//      F^T c = h, F = grad p(x_T)^T n, with a reflector H_F: the least-squares
//      problem runs on B H_F without the pivot column, and the coefficient of h
//      is beta = (lambda~_piv - s^T p~_piv) / rho.
//
// Precision is a template pair (TQ, HP): (double, double) is the FP64 path;
// (float, ff) factors in FP32 and keeps B, sqrt(W), lambda and the iterates
// in float-float (ff.cuh) so that no FP64 instruction runs in the loop.
//
// The kernel is persistent and bucketed: the targets are grouped on the device
// into buckets of equal (degree, row class); a block of 4 warps repeatedly
// takes a "block task" (G warps per target, 4/G targets of one bucket) from a
// global counter.  G and the tile shape (ld rows, nmax columns) are per bucket
// (chosen by the host, or by the autotuner), so one launch covers every shape.
#include <cuda_runtime.h>

#include "basis_tables.cuh"
#include "ff.cuh"
#include "gmls_internal.cuh"

namespace gmls {

constexpr int kBlock = 128;

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// ------------------------------------------------------- precision helpers
__device__ __forceinline__ double hp_from(double v, double) { return v; }
__device__ __forceinline__ ff hp_from(double v, ff) { return ff(v); }
__device__ __forceinline__ double hp_to_double(double v) { return v; }
__device__ __forceinline__ double hp_to_double(ff v) { return to_double(v); }
__device__ __forceinline__ double hp_hi_d(double v) { return v; }
__device__ __forceinline__ float hp_hi_f(ff v) { return v.h; }
__device__ __forceinline__ double hp_recip(double v) { return 1.0 / v; }
__device__ __forceinline__ ff hp_recip(ff v) { return recip(v); }
__device__ __forceinline__ double hp_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ ff hp_sqrt(ff v) { return sqrt_ff(v); }
__device__ __forceinline__ double hp_add_f(double a, double b) { return a + b; }
__device__ __forceinline__ ff hp_add_f(ff a, float b) { return add_f(a, b); }
__device__ __forceinline__ bool hp_pos(double v) { return v > 0.0; }
__device__ __forceinline__ bool hp_pos(ff v) { return v.h > 0.0f; }
__device__ __forceinline__ double hp_zero(double) { return 0.0; }
__device__ __forceinline__ ff hp_zero(ff) { return ff(0.0f, 0.0f); }
__device__ __forceinline__ double hp_one(double) { return 1.0; }
__device__ __forceinline__ ff hp_one(ff) { return ff(1.0f, 0.0f); }

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
// float-float all-reduce across the warp
__device__ __forceinline__ ff warp_sum_ff(float h, float l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    const ff s = two_sum(h, oh);
    h = s.h;
    l = __fadd_rn(l, __fadd_rn(ol, s.l));
  }
  return quick_two_sum(h, l);
}

// float-float all-reduce across the warp of R independent accumulators
// (rows >= L untouched); the R reduction chains interleave
template <int R>
__device__ __forceinline__ void warp_sum_ff_rows(Dot2 (&acc)[R], int L) {
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (q >= L) continue;
      const float oh = __shfl_xor_sync(0xffffffffu, acc[q].h, o);
      const float ol = __shfl_xor_sync(0xffffffffu, acc[q].l, o);
      const ff s = two_sum(acc[q].h, oh);
      acc[q].h = s.h;
      acc[q].l = __fadd_rn(acc[q].l, __fadd_rn(ol, s.l));
    }
  }
}

__device__ __forceinline__ void group_sync(int gid, int nthr) {
  if (nthr == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(nthr) : "memory");
}

struct Group {
  int gid, nthr, tid, wg, G, lane;
};

// ------------------------------------------------------------ tile layout
struct Lay {
  size_t A, HB, gtotal, tau, dots, sw, lam, S, Y, Z, D, pt, misc, total;
};

// Leading dimension of the tiles: the row capacity made odd, so that a row of
// R (stride ld) falls in distinct shared-memory banks across a warp.
__host__ __device__ inline int pad_ld(int ld) { return ld | 1; }

// tqs: bytes of TQ; hps: bytes of HP; hb: separate high-precision tile (FP32
// path).  place: where the two tiles live --
//   kPlaceShared  both in shared memory (offsets A, HB in the shared slice);
//   kPlaceSplit   the working tile A in shared memory, the float-float copy HB
//                 in a global-memory slot (offset HB there, gtotal its size);
//                 HB is only read by the refinement passes, A by every QR step;
//   kPlaceGlobal  both in a global-memory slot (offsets A, HB there).
// The per-target vectors (tau, S, Y, ...) always stay in shared memory.
__host__ __device__ inline Lay make_lay(int ld, int nmax, int tqs, int hps, bool hb, int place = kPlaceShared) {
  ld = pad_ld(ld);
  Lay l;
  size_t o = 0;
  const size_t a_bytes = align16((size_t)nmax * ld * tqs);
  const size_t hb_bytes = hb ? align16((size_t)nmax * ld * hps) : 0;
  if (place == kPlaceSplit && hb) {
    l.HB = 0;
    l.gtotal = hb_bytes;
    l.A = 0;
    o = a_bytes;
  } else {
    l.A = 0;
    l.HB = a_bytes;
    o = a_bytes + hb_bytes;
    l.gtotal = place == kPlaceGlobal ? o : 0;
    if (place == kPlaceGlobal) o = 0;
  }
  l.tau = o;
  o += align16((size_t)nmax * tqs);
  l.dots = o;
  o += align16((size_t)nmax * tqs);
  l.sw = o;
  o += align16((size_t)ld * hps);
  l.lam = o;
  o += align16((size_t)kMaxSolveRows * nmax * hps);
  l.S = o;
  o += align16((size_t)kMaxSolveRows * ld * hps);
  l.Y = o;
  o += align16((size_t)kMaxSolveRows * nmax * hps);
  l.Z = o;
  o += align16((size_t)kMaxSolveRows * ld * tqs);
  l.D = o;
  o += align16((size_t)kMaxSolveRows * nmax * tqs);
  l.pt = o;
  o += align16((size_t)ld * hps);
  l.misc = o;
  o += 256;
  l.total = o;
  return l;
}

size_t tile_bytes(int ld, int nmax, bool fp32_refine, int place) {
  return fp32_refine ? make_lay(ld, nmax, 4, 8, true, place).total : make_lay(ld, nmax, 8, 8, false, place).total;
}
size_t global_tile_bytes(int ld, int nmax, bool fp32_refine, int place) {
  return fp32_refine ? make_lay(ld, nmax, 4, 8, true, place).gtotal : make_lay(ld, nmax, 8, 8, false, place).gtotal;
}

// ---------------------------------------------------------------- QR (in TQ)
// Householder QR of the M x n tile A (column-major, leading dimension ld).
// Column k below the diagonal keeps v_k (v_k[k] = 1 implied), tau[k] its scale.
// Per column: warp 0 forms the reflector; then each warp takes the trailing
// columns kQrCols at a time, so that one load of the reflector feeds that many
// independent dot-product chains and their warp reductions interleave.
constexpr int kQrCols = 4;

template <typename TQ>
__device__ void tile_qr(const Group& g, TQ* A, int ld, int M, int n, TQ* tau) {
  for (int k = 0; k < n; ++k) {
    TQ* a = A + (size_t)k * ld;
    if (g.wg == 0) {
      TQ sig = 0;
#pragma unroll 4
      for (int r = k + 1 + g.lane; r < M; r += 32) sig += a[r] * a[r];
      sig = warp_sum(sig);
      const TQ alpha = a[k];
      if (sig == TQ(0)) {
        if (g.lane == 0) tau[k] = 0;
      } else {
        const TQ nrm = sqrt(alpha * alpha + sig);
        const TQ beta = alpha >= TQ(0) ? -nrm : nrm;
        const TQ scale = TQ(1) / (alpha - beta);
#pragma unroll 4
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
      for (int j0 = k + 1 + g.wg * kQrCols; j0 < n; j0 += g.G * kQrCols) {
        const int nc = min(kQrCols, n - j0);
        TQ* aj = A + (size_t)j0 * ld;
        TQ s[kQrCols];
#pragma unroll
        for (int c = 0; c < kQrCols; ++c) s[c] = (g.lane == 0 && c < nc) ? aj[(size_t)c * ld + k] : TQ(0);
#pragma unroll 4
        for (int r = k + 1 + g.lane; r < M; r += 32) {
          const TQ ar = a[r];
#pragma unroll
          for (int c = 0; c < kQrCols; ++c)
            if (c < nc) s[c] += ar * aj[(size_t)c * ld + r];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int c = 0; c < kQrCols; ++c) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
#pragma unroll
        for (int c = 0; c < kQrCols; ++c) s[c] *= tk;
#pragma unroll 4
        for (int r = k + 1 + g.lane; r < M; r += 32) {
          const TQ ar = a[r];
#pragma unroll
          for (int c = 0; c < kQrCols; ++c)
            if (c < nc) aj[(size_t)c * ld + r] -= s[c] * ar;
        }
        if (g.lane == 0)
#pragma unroll
          for (int c = 0; c < kQrCols; ++c)
            if (c < nc) aj[(size_t)c * ld + k] -= s[c];
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
#pragma unroll 4
      for (int r = k + 1 + g.lane; r < M; r += 32) d += a[r] * zl[r];
      d = warp_sum(d) * tk;
#pragma unroll 4
      for (int r = k + 1 + g.lane; r < M; r += 32) zl[r] -= d * a[r];
      if (g.lane == 0) zl[k] -= d;
      __syncwarp();
    }
  }
}

// ------------------------------------------------ register-chunked variants
// For tiles of at most 32 RPL rows: lane owns rows lane + 32 t (t < RPL), so
// the row loops unroll at compile time, the reflector and the columns being
// updated sit in registers for a whole column step (one load and one store
// per element and step) and the vector that Q acts on stays in registers for
// all n reflectors.  Same arithmetic as tile_qr / apply_q; only the order of
// the partial sums in apply_q's dot products differs.
// Warp all-reduce of Q independent partial sums (Q a power of two <= 32) by
// recursive halving: at each of the first log2 Q steps a lane keeps half of
// its values and adds the partner's copy of them, so one value is left per
// lane after Q - 1 shuffles; five minus log2 Q plain butterfly steps finish
// it, and lane q << (5 - log2 Q) then holds sum q, which is broadcast.
// Q - 1 + 5 - log2 Q + Q shuffles instead of 5 Q.
template <typename T, int Q>
__device__ __forceinline__ void warp_sum_halving(T (&s)[Q], int lane) {
  constexpr int LOGQ = Q <= 1 ? 0 : Q <= 2 ? 1 : Q <= 4 ? 2 : Q <= 8 ? 3 : Q <= 16 ? 4 : 5;
  static_assert((1 << LOGQ) == Q, "Q must be a power of two");
  T v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) v[i] = s[i];
#pragma unroll
  for (int h = Q / 2, off = 16; h >= 1; h /= 2, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (int off = 16 >> LOGQ; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
#pragma unroll
  for (int q = 0; q < Q; ++q) s[q] = __shfl_sync(0xffffffffu, v[0], q << (5 - LOGQ));
}

// QC columns per warp pass (fewer for FP64: twice the registers per element)
template <typename TQ, int RPL, int QC = (sizeof(TQ) == 8 ? (RPL >= 16 ? 1 : 2) : kQrCols)>
__device__ void tile_qr_rows(const Group& g, TQ* A, int ld, int M, int n, TQ* tau) {
  for (int k = 0; k < n; ++k) {
    TQ* a = A + k * ld;
    bool live[RPL];  // row below the diagonal and inside the tile
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = g.lane + 32 * t;
      live[t] = r > k && r < M;
    }
    TQ v[RPL];
    if (g.wg == 0) {
      TQ sig = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        v[t] = live[t] ? a[g.lane + 32 * t] : TQ(0);
        sig += v[t] * v[t];
      }
      sig = warp_sum(sig);
      const TQ alpha = a[k];
      if (sig == TQ(0)) {
        if (g.lane == 0) tau[k] = 0;
      } else {
        const TQ nrm = sqrt(alpha * alpha + sig);
        const TQ beta = alpha >= TQ(0) ? -nrm : nrm;
        const TQ scale = TQ(1) / (alpha - beta);
#pragma unroll
        for (int t = 0; t < RPL; ++t)
          if (live[t]) a[g.lane + 32 * t] = v[t] * scale;
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
#pragma unroll
      for (int t = 0; t < RPL; ++t) v[t] = live[t] ? a[g.lane + 32 * t] : TQ(0);
      for (int j0 = k + 1 + g.wg * QC; j0 < n; j0 += g.G * QC) {
        const int nc = min(QC, n - j0);
        TQ* aj = A + j0 * ld;
        TQ c[QC][RPL], s[QC];
#pragma unroll
        for (int q = 0; q < QC; ++q) {
          s[q] = (g.lane == 0 && q < nc) ? aj[q * ld + k] : TQ(0);
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            c[q][t] = (live[t] && q < nc) ? aj[q * ld + g.lane + 32 * t] : TQ(0);
            s[q] += v[t] * c[q][t];
          }
        }
        warp_sum_halving<TQ, QC>(s, g.lane);
#pragma unroll
        for (int q = 0; q < QC; ++q) {
          s[q] *= tk;
          if (q < nc) {
#pragma unroll
            for (int t = 0; t < RPL; ++t)
              if (live[t]) aj[q * ld + g.lane + 32 * t] = c[q][t] - s[q] * v[t];
            if (g.lane == 0) aj[q * ld + k] -= s[q];
          }
        }
      }
      group_sync(g.gid, g.nthr);
    }
  }
}

// Householder QR of an FP32 tile held in registers (M <= 32 RPL rows,
// n <= CPW G columns): warp w owns the columns j = w + u G (u < CPW), lane
// owns rows lane + 32 t.  Per column step the reflector v_k is published in
// shared memory (vbuf, two buffers of 32 RPL floats: rows < k zero, row k
// one) and each warp applies it to its own trailing columns, four at a time
// with one halving reduction.  The owner of column k + 1 updates that column
// first and publishes reflector k + 1 before its other columns (look-ahead),
// so a step costs one barrier.  The factor goes back to A at the end, in the
// layout tile_qr leaves.
template <int RPL, int CPW>
__device__ void tile_qr_regs(const Group& g, float* A, int ld, int M, int n, float* tau, float* vbuf) {
  constexpr int NR = 32 * RPL;
  float c[CPW][RPL];
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int j = g.wg + u * g.G;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = g.lane + 32 * t;
      c[u][t] = (j < n && r < M) ? A[j * ld + r] : 0.0f;
    }
  }
  // reflector of the column held in x (column k): x becomes [R part; beta;
  // v below]; the published copy has zeros above k and one at k
  auto reflect = [&](float (&x)[RPL], int k) {
    float sig = 0.0f, alpha = 0.0f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = g.lane + 32 * t;
      if (r > k && r < M) sig += x[t] * x[t];
      if (r == k) alpha = x[t];
    }
    sig = warp_sum(sig);
    alpha = __shfl_sync(0xffffffffu, alpha, k & 31);
    float* vb = vbuf + (k & 1) * NR;
    float tk = 0.0f;
    if (sig != 0.0f) {
      const float nrm = sqrtf(alpha * alpha + sig);
      const float beta = alpha >= 0.0f ? -nrm : nrm;
      const float scale = 1.0f / (alpha - beta);
      tk = (beta - alpha) / beta;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = g.lane + 32 * t;
        if (r > k && r < M) x[t] *= scale;
        if (r == k) x[t] = beta;
      }
    }
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = g.lane + 32 * t;
      vb[r] = (r > k && r < M) ? x[t] : (r == k ? 1.0f : 0.0f);
    }
    if (g.lane == 0) tau[k] = tk;
  };
  // column k's owner forms reflector 0 before the loop
  if (g.wg == 0 && n > 0) reflect(c[0], 0);
  group_sync(g.gid, g.nthr);
  for (int k = 0; k < n; ++k) {
    const float* vb = vbuf + (k & 1) * NR;
    float v[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) v[t] = vb[g.lane + 32 * t];
    const float tk = tau[k];
    const int la = k + 1;  // look-ahead column
    const bool own_la = la < n && (la % g.G) == g.wg;
    const int u_la = la / g.G;
    if (own_la) {
#pragma unroll
      for (int u = 0; u < CPW; ++u)
        if (u == u_la) {
          if (tk != 0.0f) {
            float s = 0.0f;
#pragma unroll
            for (int t = 0; t < RPL; ++t) s += v[t] * c[u][t];
            s = warp_sum(s) * tk;
#pragma unroll
            for (int t = 0; t < RPL; ++t) c[u][t] -= s * v[t];
          }
          reflect(c[u], la);
        }
    }
    if (tk != 0.0f) {
#pragma unroll
      for (int ub = 0; ub < CPW; ub += 4) {
        if (g.wg + (ub + 3) * g.G <= la) continue;  // every column of the group finished or handled
        float sq[4];
        bool act[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = ub + q;
          const int j = g.wg + u * g.G;
          act[q] = u < CPW && j > la && j < n;
          sq[q] = 0.0f;
          if (u < CPW) {
#pragma unroll
            for (int t = 0; t < RPL; ++t) sq[q] += v[t] * c[u][t];
          }
        }
        warp_sum_halving<float, 4>(sq, g.lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = ub + q;
          if (u < CPW && act[q]) {
            const float sk = sq[q] * tk;
#pragma unroll
            for (int t = 0; t < RPL; ++t) c[u][t] -= sk * v[t];
          }
        }
      }
    }
    group_sync(g.gid, g.nthr);
  }
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int j = g.wg + u * g.G;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = g.lane + 32 * t;
      if (j < n && r < M) A[j * ld + r] = c[u][t];
    }
  }
  group_sync(g.gid, g.nthr);
}

template <typename TQ, bool TRANS, int RPL>
__device__ void apply_q_rows(const Group& g, const TQ* A, int ld, int M, int n, const TQ* tau, int L, TQ* z) {
  for (int l = g.wg; l < L; l += g.G) {
    TQ* zl = z + l * ld;
    TQ zr[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) zr[t] = (g.lane + 32 * t < M) ? zl[g.lane + 32 * t] : TQ(0);
    for (int s = 0; s < n; ++s) {
      const int k = TRANS ? s : n - 1 - s;
      const TQ tk = tau[k];
      if (tk == TQ(0)) continue;
      const TQ* a = A + k * ld;
      TQ av[RPL], d = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = g.lane + 32 * t;
        av[t] = (r > k && r < M) ? a[r] : (r == k ? TQ(1) : TQ(0));  // v_k[k] = 1
        d += av[t] * zr[t];
      }
      d = warp_sum(d) * tk;
#pragma unroll
      for (int t = 0; t < RPL; ++t) zr[t] -= d * av[t];
    }
#pragma unroll
    for (int t = 0; t < RPL; ++t)
      if (g.lane + 32 * t < M) zl[g.lane + 32 * t] = zr[t];
  }
}

// Triangular solves with the right-hand side in registers (lane owns entries
// lane + 32 u, u < NPL; n <= 32 NPL), column-oriented: after x_i is known it
// is broadcast and every later entry takes its update, one shuffle and one
// multiply-add per step instead of a warp reduction.  rdiag[i] = 1 / R_ii.
template <typename TQ, int NPL>
__device__ __forceinline__ TQ pick(const TQ (&x)[NPL], int u) {
  TQ v = x[0];
#pragma unroll
  for (int w = 1; w < NPL; ++w)
    if (u == w) v = x[w];
  return v;
}

// y = R^{-T} b for the L rows (b and y: [L][nmax], may alias)
template <typename TQ, typename TB, int NPL>
__device__ void solve_rt_regs(const Group& g, const TQ* A, int ld, int n, int L, int nmax, const TQ* rdiag,
                              const TB* b, TQ* y) {
  for (int l = g.wg; l < L; l += g.G) {
    TQ yr[NPL];
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int q = g.lane + 32 * u;
      yr[u] = q < n ? TQ(b[l * nmax + q]) : TQ(0);
    }
    for (int i = 0; i < n; ++i) {
      const TQ yi = __shfl_sync(0xffffffffu, pick<TQ, NPL>(yr, i >> 5), i & 31) * rdiag[i];
#pragma unroll
      for (int u = 0; u < NPL; ++u) {
        const int q = g.lane + 32 * u;
        if (q > i && q < n)
          yr[u] -= A[q * ld + i] * yi;  // R[i][q]
        else if (q == i)
          yr[u] = yi;
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int q = g.lane + 32 * u;
      if (q < n) y[l * nmax + q] = yr[u];
    }
  }
}

// x = R^{-1} x in place on [L][nmax] rows
template <typename TQ, int NPL>
__device__ void solve_r_regs(const Group& g, const TQ* A, int ld, int n, int L, int nmax, const TQ* rdiag, TQ* x) {
  for (int l = g.wg; l < L; l += g.G) {
    TQ xr[NPL];
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int q = g.lane + 32 * u;
      xr[u] = q < n ? x[l * nmax + q] : TQ(0);
    }
    for (int i = n - 1; i >= 0; --i) {
      const TQ xi = __shfl_sync(0xffffffffu, pick<TQ, NPL>(xr, i >> 5), i & 31) * rdiag[i];
      const TQ* ri = A + i * ld;  // column i: R[q][i] = ri[q], q <= i
#pragma unroll
      for (int u = 0; u < NPL; ++u) {
        const int q = g.lane + 32 * u;
        if (q < i)
          xr[u] -= ri[q] * xi;
        else if (q == i)
          xr[u] = xi;
      }
    }
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int q = g.lane + 32 * u;
      if (q < n) x[l * nmax + q] = xr[u];
    }
  }
}

constexpr int kSolveNpl = 3;   // register solves for up to 96 basis functions
constexpr int kQrRegCols = 13;  // register QR: up to 52 columns over four warps

// dispatch on the tile's rows: register-chunked up to 512 rows, else the loops
template <typename TQ>
__device__ void qr_any(const Group& g, TQ* A, int ld, int M, int n, TQ* tau) {
  if (M <= 64)
    tile_qr_rows<TQ, 2>(g, A, ld, M, n, tau);
  else if (M <= 128)
    tile_qr_rows<TQ, 4>(g, A, ld, M, n, tau);
  else if (M <= 256)
    tile_qr_rows<TQ, 8>(g, A, ld, M, n, tau);
  else if (M <= 512)
    tile_qr_rows<TQ, 16>(g, A, ld, M, n, tau);
  else
    tile_qr<TQ>(g, A, ld, M, n, tau);
}
template <typename TQ, bool TRANS>
__device__ void apply_q_any(const Group& g, const TQ* A, int ld, int M, int n, const TQ* tau, int L, TQ* z) {
  if (M <= 64)
    apply_q_rows<TQ, TRANS, 2>(g, A, ld, M, n, tau, L, z);
  else if (M <= 128)
    apply_q_rows<TQ, TRANS, 4>(g, A, ld, M, n, tau, L, z);
  else if (M <= 256)
    apply_q_rows<TQ, TRANS, 8>(g, A, ld, M, n, tau, L, z);
  else if (M <= 512)
    apply_q_rows<TQ, TRANS, 16>(g, A, ld, M, n, tau, L, z);
  else
    apply_q<TQ, TRANS>(g, A, ld, M, n, tau, L, z);
}
template <typename TQ, typename TB>
__device__ void solve_rt_any(const Group& g, const TQ* A, int ld, int n, int L, int nmax, const TQ* rdiag,
                             const TB* b, TQ* y) {
  if (n <= 32 * kSolveNpl)
    solve_rt_regs<TQ, TB, kSolveNpl>(g, A, ld, n, L, nmax, rdiag, b, y);
  else
    solve_rt<TQ, TB>(g, A, ld, n, L, nmax, b, y);
}
template <typename TQ>
__device__ void solve_r_any(const Group& g, const TQ* A, int ld, int n, int L, int nmax, const TQ* rdiag, TQ* x) {
  if (n <= 32 * kSolveNpl)
    solve_r_regs<TQ, kSolveNpl>(g, A, ld, n, L, nmax, rdiag, x);
  else
    solve_r<TQ>(g, A, ld, n, L, nmax, x);
}

// per-row offset of neighbour q from the target, in HP, and |x_j - x_T|^2
__device__ __forceinline__ void offsets(const StencilJob& j, int64_t t, int32_t jj, double* dx) {
  for (int c = 0; c < j.dim; ++c) dx[c] = j.x[c * j.n + jj] - j.x[c * j.n + t];
}
__device__ __forceinline__ void offsets(const StencilJob& j, int64_t t, int32_t jj, ff* dx) {
  for (int c = 0; c < j.dim; ++c)
    dx[c] = diff_ff(j.x[c * j.n + jj], j.x[c * j.n + t]);
}

// sqrt(W) = u^(p/2), u = 1 - r/eps > 0
__device__ __forceinline__ double sqrt_weight(double u, const StencilJob& j) {
  return j.wpow == 4.0 ? u * u : pow(u, 0.5 * j.wpow);
}
__device__ __forceinline__ ff sqrt_weight(ff u, const StencilJob& j) {
  ff s = (j.wpow_half * 2 == (int)j.wpow) ? u : sqrt_ff(u);
  const int reps = (j.wpow_half * 2 == (int)j.wpow) ? j.wpow_half - 1 : j.wpow_half;
  const ff base = u;
  for (int p = 0; p < reps; ++p) s = s * base;
  return s;
}

// ------------------------------------------------ refinement residuals
// f = B y - s for the L functional rows: a thread takes tile rows r and
// r + nthr together, so two independent streams of loads of B are in flight;
// per row the products are accumulated in column order (Dot2).
template <typename TQ>
__device__ void resid_f(const Group& g, const ff* B, int ld, int M, int n, int L, int nmax, const ff* Sf,
                        const ff* Yf, TQ* Z) {
  for (int r0 = g.tid; r0 < M; r0 += 2 * g.nthr) {
    const int r1 = r0 + g.nthr;
    const bool two = r1 < M;
    Dot2 a0[kMaxSolveRows], a1[kMaxSolveRows];
#pragma unroll
    for (int l = 0; l < kMaxSolveRows; ++l)
      if (l < L) {
        a0[l].init(-Sf[l * ld + r0]);
        if (two) a1[l].init(-Sf[l * ld + r1]);
      }
#pragma unroll 8
    for (int i = 0; i < n; ++i) {
      const ff b0 = B[i * ld + r0];
      const ff b1 = two ? B[i * ld + r1] : ff(0.0f, 0.0f);
#pragma unroll
      for (int l = 0; l < kMaxSolveRows; ++l)
        if (l < L) {
          const ff y = Yf[l * nmax + i];
          a0[l].add_prod(b0, y);
          a1[l].add_prod(b1, y);
        }
    }
#pragma unroll
    for (int l = 0; l < kMaxSolveRows; ++l)
      if (l < L) {
        Z[l * ld + r0] = (TQ)__fadd_rn(a0[l].h, a0[l].l);
        if (two) Z[l * ld + r1] = (TQ)__fadd_rn(a1[l].h, a1[l].l);
      }
  }
}

// g = lambda - B^T s: a warp per basis column; per lane the rows are
// accumulated in ascending order, then the L sums are all-reduced together.
// (Loading a lane's whole column slice into registers before the products
// raised the kernel's register demand and slowed every phase.)
template <typename TQ>
__device__ void resid_g(const Group& g, const ff* B, int ld, int M, int n, int L, int nmax, const ff* Sf,
                        const ff* lamf, TQ* D) {
  for (int i = g.wg; i < n; i += g.G) {
    const ff* bi = B + i * ld;
    Dot2 acc[kMaxSolveRows];
#pragma unroll 2
    for (int r = g.lane; r < M; r += 32) {
      const ff b = -bi[r];
#pragma unroll
      for (int l = 0; l < kMaxSolveRows; ++l)
        if (l < L) acc[l].add_prod(b, Sf[l * ld + r]);
    }
    warp_sum_ff_rows<kMaxSolveRows>(acc, L);
    if (g.lane < L) {
      const int l = g.lane;
      float h = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < kMaxSolveRows; ++q)
        if (q == l) {
          h = acc[q].h;
          lo = acc[q].l;
        }
      const ff tot = quick_two_sum(h, lo) + lamf[l * nmax + i];
      D[l * nmax + i] = (TQ)__fadd_rn(tot.h, tot.l);
    }
  }
}

// Basis output into the float-float tile and its FP32 working copy at once.
struct DualOut {
  ff* hb;
  float* a;
  struct Ref {
    ff* h;
    float* f;
    __device__ __forceinline__ void operator=(const ff& v) const {
      *h = v;
      *f = v.h;
    }
  };
  __device__ __forceinline__ Ref operator[](int i) const { return Ref{hb + i, a + i}; }
};

// ------------------------------------------------------------ one target
template <typename TQ, typename HP, bool REFINE>
__device__ void process_target(const StencilJob& j, const Group& g, unsigned char* base, unsigned char* gbase,
                               int place, int ld, int nmax, int64_t to) {
  const Lay lay = make_lay(ld, nmax, (int)sizeof(TQ), (int)sizeof(HP), REFINE, place);
  const int ld_rows = ld;  // row capacity; the tiles use the padded stride
  ld = pad_ld(ld);
  TQ* A = reinterpret_cast<TQ*>((place == kPlaceGlobal ? gbase : base) + lay.A);
  HP* HB = REFINE ? reinterpret_cast<HP*>((place == kPlaceShared ? base : gbase) + lay.HB) : reinterpret_cast<HP*>(A);
  TQ* tau = reinterpret_cast<TQ*>(base + lay.tau);
  TQ* rdiag = reinterpret_cast<TQ*>(base + lay.dots);  // 1 / R_ii
  HP* sw = reinterpret_cast<HP*>(base + lay.sw);
  HP* lam = reinterpret_cast<HP*>(base + lay.lam);
  HP* S = reinterpret_cast<HP*>(base + lay.S);
  HP* Y = reinterpret_cast<HP*>(base + lay.Y);
  TQ* Z = reinterpret_cast<TQ*>(base + lay.Z);
  TQ* D = reinterpret_cast<TQ*>(base + lay.D);
  HP* pt = reinterpret_cast<HP*>(base + lay.pt);
  HP* hmisc = reinterpret_cast<HP*>(base + lay.misc);  // [0] rho, [1..L] lambda~_piv
  double* dmisc = reinterpret_cast<double*>(base + lay.misc + 128);  // [0..7] reductions
  int* imisc = reinterpret_cast<int*>(base + lay.misc + 192);
  const HP hz = hp_zero(HP());

  const int L = j.L, dim = j.dim, nc = j.nc;
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
  bool skip = (st & GMLS_T_TOO_FEW_NEIGHBOURS) || k <= 0 || nb <= 0 || M > ld_rows || nb > nmax || !(eps > 0.0);
  if (!(st & GMLS_T_TOO_FEW_NEIGHBOURS) && k > 0 && (M > ld_rows || nb > nmax)) st |= GMLS_T_UNSUPPORTED;
  if (!skip && M < n) {
    st |= GMLS_T_RANK_DEFICIENT;
    skip = true;
  }
  // staggered basis: the weights act on p_j - p(x_T); the target's own entry
  // (its row of the tile is zero) later takes minus the sum of the others
  int self = -1;
  if (j.kind == GMLS_BASIS_STAGGERED && !skip) {
    for (int q = 0; q < k; ++q)
      if (nbr[q] == (int32_t)t) {
        self = q;
        break;
      }
    if (self < 0) {
      st |= GMLS_T_UNSUPPORTED;
      skip = true;
    }
  }
  bool redo = false;
  int used_iters = 0;

  if (!skip) {
    const HP heps = hp_from(eps, HP());
    const HP inv_eps = hp_recip(heps);
    // ---- 1. sqrt(W) P in HP, rows (neighbour, component)
    for (int q = g.tid; q < k; q += g.nthr) {
      HP dx[3] = {hz, hz, hz}, xi[3] = {hz, hz, hz};
      offsets(j, t, nbr[q], dx);
      HP r2 = hz;
      for (int c = 0; c < dim; ++c) {
        xi[c] = dx[c] * inv_eps;
        r2 = r2 + dx[c] * dx[c];
      }
      const HP u = hp_one(HP()) - hp_sqrt(r2) * inv_eps;
      const HP s = hp_pos(u) ? sqrt_weight(u, j) : hz;
      if constexpr (REFINE) {  // the FP32 tile too (rewritten after a Neumann step edits HB)
        gmls_gen::eval_basis<HP>(j.kind, dim, m, xi, DualOut{HB + q * nc, A + q * nc}, ld, s);
      } else {
        gmls_gen::eval_basis<HP>(j.kind, dim, m, xi, HB + q * nc, ld, s);
      }
      for (int c = 0; c < nc; ++c) sw[q * nc + c] = s;
    }
    // ---- 3. functional rows lambda (before Neumann)
    for (int e = g.tid; e < L * nb; e += g.nthr) {
      const int l = e / nb, i = e % nb;
      HP f = hp_from(gmls_gen::lam_coef(j.kind, dim, m, j.lam_fn[l], j.lam_row[l], i), HP());
      for (int p = 0; p < j.lam_order[l]; ++p) f = f * inv_eps;
      lam[l * nmax + i] = f;
    }
    group_sync(g.gid, g.nthr);

    // ---- 6. Neumann: reflect the linear columns (indices 1..dim), move the
    //         pivot column to the end, and keep it aside as p~
    if (neu) {
      double nvd[3] = {0.0, 0.0, 0.0};
      int piv = 0;
      for (int c = 0; c < dim; ++c) {
        nvd[c] = j.normals[c * j.n + t];
        if (fabs(nvd[c]) > fabs(nvd[piv])) piv = c;
      }
      HP v[3] = {hz, hz, hz}, fn2 = hz;
      for (int c = 0; c < dim; ++c) {
        v[c] = hp_from(nvd[c], HP()) * inv_eps;  // F restricted to the linear monomials
        fn2 = fn2 + v[c] * v[c];
      }
      const HP fn = hp_sqrt(fn2);
      const HP rho = nvd[piv] >= 0.0 ? hz - fn : fn;
      v[piv] = v[piv] - rho;  // v = F - rho e_piv
      HP vv = hz;
      for (int c = 0; c < dim; ++c) vv = vv + v[c] * v[c];
      const HP two_vv = hp_from(2.0, HP()) * hp_recip(vv);
      for (int r = g.tid; r < M; r += g.nthr) {
        HP d = hz;
        for (int c = 0; c < dim; ++c) d = d + HB[(size_t)(1 + c) * ld + r] * v[c];
        d = d * two_vv;
        for (int c = 0; c < dim; ++c) HB[(size_t)(1 + c) * ld + r] = HB[(size_t)(1 + c) * ld + r] - d * v[c];
        const HP pc = HB[(size_t)(1 + piv) * ld + r];
        HB[(size_t)(1 + piv) * ld + r] = HB[(size_t)(nb - 1) * ld + r];
        HB[(size_t)(nb - 1) * ld + r] = pc;
        pt[r] = pc;
      }
      if (g.tid < L) {
        const int l = g.tid;
        HP* ll = lam + l * nmax;
        HP d = hz;
        for (int c = 0; c < dim; ++c) d = d + ll[1 + c] * v[c];
        d = d * two_vv;
        for (int c = 0; c < dim; ++c) ll[1 + c] = ll[1 + c] - d * v[c];
        const HP lp = ll[1 + piv];
        ll[1 + piv] = ll[nb - 1];
        ll[nb - 1] = lp;
        hmisc[1 + l] = lp;
      }
      if (g.tid == 0) hmisc[0] = rho;
      group_sync(g.gid, g.nthr);
    }

    if (REFINE && neu) {  // FP32 working copy of the tile after the Neumann step
#pragma unroll 4
      for (int e = g.tid; e < n * M; e += g.nthr) {
        const int i = e / M, r = e - i * M;
        A[i * ld + r] = (TQ)hp_hi_f(reinterpret_cast<ff*>(HB)[i * ld + r]);
      }
      group_sync(g.gid, g.nthr);
    }

    // ---- 2. QR
    if constexpr (REFINE) {  // FP32 tile: in registers where it fits four warps
      if (g.G == 4 && M > 64 && M <= 128 && n <= 4 * kQrRegCols)
        tile_qr_regs<4, kQrRegCols>(g, A, ld, M, n, tau, Z);
      else if (g.G == 4 && M > 128 && M <= 256 && n <= 4 * kQrRegCols)
        tile_qr_regs<8, kQrRegCols>(g, A, ld, M, n, tau, Z);
      else
        qr_any<TQ>(g, A, ld, M, n, tau);
    } else {
      qr_any<TQ>(g, A, ld, M, n, tau);
    }
    for (int i = g.tid; i < n; i += g.nthr) rdiag[i] = TQ(1) / A[i * ld + i];
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
        if (!((double)rmin > 64.0 * n * 1.1102230246251565e-16 * (double)rmax)) fl |= GMLS_T_RANK_DEFICIENT;
        if (!((double)rmin * 1e6 >= (double)rmax)) fl |= GMLS_T_ILL_CONDITIONED;
        imisc[0] = fl;
      }
    }
    group_sync(g.gid, g.nthr);
    st |= (uint8_t)imisc[0];

    // ---- 4. s = Q [R^{-T} lambda; 0]
    for (int e = g.tid; e < L * n; e += g.nthr) D[(e / n) * nmax + e % n] = (TQ)hp_to_double(lam[(e / n) * nmax + e % n]);
    group_sync(g.gid, g.nthr);
    solve_rt_any<TQ, TQ>(g, A, ld, n, L, nmax, rdiag, D, D);
    group_sync(g.gid, g.nthr);
    for (int e = g.tid; e < L * M; e += g.nthr) {
      const int l = e / M, r = e % M;
      Z[(size_t)l * ld + r] = (r < n) ? D[l * nmax + r] : TQ(0);
    }
    group_sync(g.gid, g.nthr);
    apply_q_any<TQ, false>(g, A, ld, M, n, tau, L, Z);
    group_sync(g.gid, g.nthr);
    for (int e = g.tid; e < L * M; e += g.nthr) {
      const int l = e / M, r = e % M;
      S[(size_t)l * ld + r] = hp_from((double)Z[(size_t)l * ld + r], HP());
    }
    if (REFINE) {
      ff* B = reinterpret_cast<ff*>(HB);
      ff* Sf = reinterpret_cast<ff*>(S);
      ff* Yf = reinterpret_cast<ff*>(Y);
      ff* lamf = reinterpret_cast<ff*>(lam);
      // y = R^{-1} R^{-T} lambda (the least-squares coefficients)
      solve_r_any<TQ>(g, A, ld, n, L, nmax, rdiag, D);
      group_sync(g.gid, g.nthr);
      for (int e = g.tid; e < L * n; e += g.nthr) Yf[(e / n) * nmax + e % n] = ff((float)D[(e / n) * nmax + e % n], 0.f);
      group_sync(g.gid, g.nthr);
      bool conv = false;
      float prev = 0.0f;
      const bool ill = (st & GMLS_T_ILL_CONDITIONED) != 0;  // ill-conditioned: straight to FP64
      for (int iter = 0; iter < j.max_refine && !ill; ++iter) {
        // f = B y - s (into Z) and g = lambda - B^T s (into D), compensated
        // float-float (the float-float tile may sit in global memory: the
        // loads of several rows / columns are issued before they are used)
        resid_f<TQ>(g, B, ld, M, n, L, nmax, Sf, Yf, Z);
        resid_g<TQ>(g, B, ld, M, n, L, nmax, Sf, lamf, D);
        group_sync(g.gid, g.nthr);
        // d = Q^T f; a = R^{-T} g; dy = R^{-1}(a - d_1); ds = Q [a; d_2]
        apply_q_any<TQ, true>(g, A, ld, M, n, tau, L, Z);
        group_sync(g.gid, g.nthr);
        solve_rt_any<TQ, TQ>(g, A, ld, n, L, nmax, rdiag, D, D);
        group_sync(g.gid, g.nthr);
        for (int e = g.tid; e < L * n; e += g.nthr) {
          const int l = e / n, i = e % n;
          const TQ a = D[l * nmax + i];
          const TQ d1 = Z[(size_t)l * ld + i];
          D[l * nmax + i] = a - d1;  // becomes dy after the back substitution
          Z[(size_t)l * ld + i] = a;
        }
        group_sync(g.gid, g.nthr);
        solve_r_any<TQ>(g, A, ld, n, L, nmax, rdiag, D);
        apply_q_any<TQ, false>(g, A, ld, M, n, tau, L, Z);
        group_sync(g.gid, g.nthr);
        float dmax = 0.0f, smax = 0.0f;
        for (int e = g.tid; e < L * M; e += g.nthr) {
          const int l = e / M, r = e % M;
          const float ds = (float)Z[(size_t)l * ld + r];
          const ff sv = add_f(Sf[(size_t)l * ld + r], ds);
          Sf[(size_t)l * ld + r] = sv;
          dmax = fmaxf(dmax, fabsf(ds));
          smax = fmaxf(smax, fabsf(sv.h));
        }
        for (int e = g.tid; e < L * n; e += g.nthr)
          Yf[(e / n) * nmax + e % n] = add_f(Yf[(e / n) * nmax + e % n], (float)D[(e / n) * nmax + e % n]);
        dmax = warp_max(dmax);
        smax = warp_max(smax);
        if (g.G > 1) {
          if (g.lane == 0) {
            dmisc[2 * g.wg] = dmax;
            dmisc[2 * g.wg + 1] = smax;
          }
          group_sync(g.gid, g.nthr);
          dmax = 0.0f;
          smax = 0.0f;
          for (int w = 0; w < g.G; ++w) {
            dmax = fmaxf(dmax, (float)dmisc[2 * w]);
            smax = fmaxf(smax, (float)dmisc[2 * w + 1]);
          }
        }
        used_iters = iter + 1;
        // error left after this correction ~ |ds| times the contraction factor,
        // estimated by the relative size of the correction (first iteration)
        // or by the ratio of successive corrections (later ones)
        const float rho = (iter == 0) ? dmax / fmaxf(smax, 1e-37f) : dmax / fmaxf(prev, 1e-37f);
        const float est = dmax * fminf(1.0f, rho);
        conv = (double)est <= j.tol * (double)smax;
        prev = dmax;
        group_sync(g.gid, g.nthr);
        if (conv) break;
      }
      if (!conv) {
        st |= ill ? 0 : GMLS_T_REFINE_NOT_CONVERGED;
        redo = true;
        if (g.tid == 0) {
          const int slot = atomicAdd(j.fb_count, 1);
          j.fb_items[slot] = (int32_t)to;
        }
      }
    }

    // ---- Neumann coefficient of h: beta = (lambda~_piv - s^T p~) / rho
    if (!redo && neu && j.beta) {
      for (int l = g.wg; l < L; l += g.G) {
        HP acc = hz;
        for (int r = g.lane; r < M; r += 32) acc = acc + S[(size_t)l * ld + r] * pt[r];
        double tot;
        if (REFINE) {
          const ff a = *reinterpret_cast<ff*>(&acc);
          tot = 0.0;
          const ff red = warp_sum_ff(a.h, a.l);
          const ff b = (reinterpret_cast<ff*>(hmisc)[1 + l] - red) * recip(reinterpret_cast<ff*>(hmisc)[0]);
          tot = to_double(b);
        } else {
          const double red = warp_sum(hp_to_double(acc));
          tot = (hp_to_double(hmisc[1 + l]) - red) / hp_to_double(hmisc[0]);
        }
        if (g.lane == 0) j.beta[to * L + l] = tot;
      }
    } else if (!redo && j.beta) {
      for (int l = g.tid; l < L; l += g.nthr) j.beta[to * L + l] = 0.0;
    }
    group_sync(g.gid, g.nthr);
  }

  // a rank-deficient system has no unique weights: store zeros (and no beta)
  if (st & GMLS_T_RANK_DEFICIENT) skip = true;
  if (redo) {  // the FP64 redo writes this target's outputs and status
    if (g.tid == 0) j.status[to] = st;
    group_sync(g.gid, g.nthr);
    return;
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
          val = hp_to_double(S[(size_t)(src + c) * ld + q] * sw[q]);
        } else {
          const int row = q * nc + c;
          val = sgn * hp_to_double(S[(size_t)(src + r) * ld + row] * sw[row]);
        }
      }
      w[e] = val;
    }
  }
  if (self >= 0 && !skip) {  // staggered: weights on point values (Sec. 2.4, Eq. vector-rho)
    group_sync(g.gid, g.nthr);
    for (int f = 0; f < j.nout; ++f) {
      const int R = j.out_rows[f];
      double* w = j.out_w[f] + o0 * (int64_t)R;
      for (int r = g.tid; r < R; r += g.nthr) {
        double* wr = w + (int64_t)r * k;
        double sum = 0.0;
        for (int q = 0; q < k; ++q)
          if (q != self) sum += wr[q];
        wr[self] = -sum;
      }
    }
  }
  if (g.tid == 0) {
    j.status[to] = st;
    if (j.iters) j.iters[to] = (uint8_t)used_iters;
  }
  if (skip && j.beta)
    for (int l = g.tid; l < L; l += g.nthr) j.beta[to * L + l] = 0.0;
  group_sync(g.gid, g.nthr);
}

// -------------------------------------------------------- persistent kernel
template <typename TQ, typename HP, bool REFINE>
__global__ void __launch_bounds__(kBlock, 3) stencil_kernel(StencilJob j, BatchPlan plan) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task, s_bucket;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      const int task = atomicAdd(plan.task_counter, 1);
      int b = -1;
      int total;
      if (plan.single) {
        const int64_t cnt = j.items ? (int64_t)(*j.n_items) : j.n_tgt;
        const int gpb = 4 / plan.G[0];
        total = (int)((cnt + gpb - 1) / gpb);
        if (task < total) b = 0;
      } else {
        total = plan.task_start[plan.nb];
        if (task < total) {
          b = 0;
          while (b + 1 < plan.nb && plan.task_start[b + 1] <= task) ++b;
        }
      }
      s_task = task;
      s_bucket = b;
    }
    __syncthreads();
    const int task = s_task, b = s_bucket;
    __syncthreads();
    if (b < 0) break;
    Group g;
    g.G = plan.G[b];
    g.nthr = 32 * g.G;
    g.gid = warp / g.G;
    g.wg = warp % g.G;
    g.tid = threadIdx.x % g.nthr;
    g.lane = threadIdx.x & 31;
    const int gpb = 4 / g.G;
    int64_t item, end;
    if (plan.single) {
      item = (int64_t)task * gpb + g.gid;
      end = j.items ? (int64_t)(*j.n_items) : j.n_tgt;
    } else {
      item = (int64_t)plan.bucket_start[b] + (int64_t)(task - plan.task_start[b]) * gpb + g.gid;
      end = plan.bucket_start[b + 1];
    }
    if (item < end) {
      const int64_t to = plan.items ? (int64_t)plan.items[item] : (j.items ? (int64_t)j.items[item] : item);
      const int place = plan.gtile[b];
      const size_t slice = (REFINE ? make_lay(plan.ld[b], plan.nmax[b], 4, 8, true, place)
                                   : make_lay(plan.ld[b], plan.nmax[b], 8, 8, false, place)).total;
      unsigned char* gslot =
          place != kPlaceShared ? plan.gscratch + ((size_t)blockIdx.x * gpb + g.gid) * plan.gslot_bytes : nullptr;
      process_target<TQ, HP, REFINE>(j, g, smem + (size_t)g.gid * slice, gslot, place, plan.ld[b], plan.nmax[b], to);
    }
  }
}

cudaError_t launch_stencils(const Launch& L, const StencilJob& j, const BatchPlan& plan, bool fp32_refine,
                            size_t smem, int grid_blocks) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (fp32_refine) {
    e = cudaFuncSetAttribute(stencil_kernel<float, ff, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    stencil_kernel<float, ff, true><<<grid_blocks, kBlock, smem, L.stream>>>(j, plan);
  } else {
    e = cudaFuncSetAttribute(stencil_kernel<double, double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    stencil_kernel<double, double, false><<<grid_blocks, kBlock, smem, L.stream>>>(j, plan);
  }
  *L.counter += 1;
  return cudaGetLastError();
}

int stencil_blocks_per_sm(bool fp32_refine, size_t smem) {
  int blocks = 0;
  const void* fn = fp32_refine ? (const void*)stencil_kernel<float, ff, true> : (const void*)stencil_kernel<double, double, false>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kBlock, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return blocks > 0 ? blocks : 1;
}

// ------------------------------------------------------------- bucketing
// bucket = (degree - 1) * n_classes + row class; row class = first class whose
// bound is >= rows (k * components); targets too large for every class get
// bucket -1 and are reported by the stencil kernel as unsupported.
__global__ void bucket_count_kernel(BucketJob b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.n_tgt; t += (int64_t)gridDim.x * blockDim.x) {
    const int m = b.degree_pt ? (int)b.degree_pt[t] : b.degree;
    const int rows = (int)(b.off[t + 1] - b.off[t]) * b.nc;
    int rc = 0;
    while (rc < b.n_classes && b.class_rows[rc] < rows) ++rc;
    int bucket = (m >= 1 && m <= 4 && rc < b.n_classes) ? (m - 1) * b.n_classes + rc : b.nb - 1;
    b.bucket_of[t] = bucket;
    atomicAdd(&b.counts[bucket], 1);
  }
}

__global__ void bucket_plan_kernel(BucketJob b) {
  if (threadIdx.x != 0) return;
  int start = 0, task = 0;
  for (int i = 0; i < b.nb; ++i) {
    b.bucket_start[i] = start;
    b.task_start[i] = task;
    b.fill[i] = 0;
    const int c = b.counts[i];
    start += c;
    task += (c + b.gpb[i] - 1) / b.gpb[i];
  }
  b.bucket_start[b.nb] = start;
  b.task_start[b.nb] = task;
}

__global__ void bucket_scatter_kernel(BucketJob b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.n_tgt; t += (int64_t)gridDim.x * blockDim.x) {
    const int bucket = b.bucket_of[t];
    const int pos = b.bucket_start[bucket] + atomicAdd(&b.fill[bucket], 1);
    b.items[pos] = (int32_t)t;
  }
}

cudaError_t launch_bucketing(const Launch& L, const BucketJob& b) {
  const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)device_sm_count() * 8, (b.n_tgt + 255) / 256 + 1);
  cudaError_t e = cudaMemsetAsync(b.counts, 0, sizeof(int32_t) * b.nb, L.stream);
  if (e != cudaSuccess) return e;
  bucket_count_kernel<<<blocks, 256, 0, L.stream>>>(b);
  bucket_plan_kernel<<<1, 32, 0, L.stream>>>(b);
  bucket_scatter_kernel<<<blocks, 256, 0, L.stream>>>(b);
  *L.counter += 3;
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ CSR
// Id order of the neighbour lists, computed once per list handle: order[o + r]
// is the position within target t's list (offset o) of its entry of rank r by
// particle id (equal ids -- the -1 padding of short lists -- by position).
// Warp per target: bitonic sort of (id, position) keys, in registers for
// lists of up to 128 entries, else in shared memory sized from the longest
// list (kcap entries per warp).
constexpr int kOrderWarps = 8;

// Bitonic sort of 32 R keys held R per lane (element lane + 32 u in key[u]),
// ascending: compare-exchanges across lanes by shuffles, within a lane for
// strides of 32 and more.  Every size and stride is a compile-time constant.
template <int R, typename K>
__device__ __forceinline__ void warp_bitonic_keys(K (&key)[R], int lane) {
  constexpr int NE = 32 * R;
#pragma unroll
  for (int size = 2; size <= NE; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int pu = u ^ (stride >> 5);
          if (pu > u) {  // element lane + 32 u is the lower one of the pair
            const bool asc = ((lane + 32 * u) & size) == 0;
            const K a = key[u], b = key[pu];
            const bool swap = asc ? (b < a) : (a < b);
            key[u] = swap ? b : a;
            key[pu] = swap ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const K other = __shfl_xor_sync(0xffffffffu, key[u], stride);
          const bool lower = (lane & stride) == 0;
          const bool asc = ((lane + 32 * u) & size) == 0;
          const K lo = other < key[u] ? other : key[u];
          const K hi = other < key[u] ? key[u] : other;
          key[u] = (lower == asc) ? lo : hi;
        }
      }
    }
  }
}

// key of a list entry: the id above the position, so equal ids keep their
// list order.  64-bit: the id with its sign bit flipped (unsigned order =
// signed order) in the high word.  32-bit, for clouds of fewer than
// 2^25 - 1 points and lists of at most 128 entries: id + 1 (the -1 of a short
// list becomes 0, first as in signed order) above 7 position bits; the
// largest key, (2^25 - 1) << 7 | 127 = ~0u, is then never a real entry, so
// the padding (~0u) sorts after every entry as in the 64-bit form, and the
// two forms give the same order.
__device__ __forceinline__ unsigned long long order_key(int32_t id, int pos, unsigned long long) {
  return ((unsigned long long)((uint32_t)id ^ 0x80000000u) << 32) | (uint32_t)pos;
}
__device__ __forceinline__ unsigned int order_key(int32_t id, int pos, unsigned int) {
  return ((uint32_t)(id + 1) << 7) | (uint32_t)pos;
}

template <int R, typename K>
__device__ __forceinline__ void order_in_registers(const int32_t* __restrict__ idx, int64_t o, int k, int lane,
                                                   int16_t* __restrict__ order) {
  constexpr uint32_t kPosMask = sizeof(K) == 4 ? 0x7fu : 0xffffffffu;
  K key[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int e = lane + 32 * u;
    key[u] = (e < k) ? order_key(idx[o + e], e, K(0)) : ~K(0);
  }
  warp_bitonic_keys<R>(key, lane);
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int e = lane + 32 * u;
    if (e < k) order[o + e] = (int16_t)((uint32_t)key[u] & kPosMask);
  }
}

__global__ void __launch_bounds__(kOrderWarps * 32) nbr_order_kernel(int64_t n_tgt, const int64_t* __restrict__ off,
                                                                     const int32_t* __restrict__ idx, int kcap,
                                                                     int16_t* __restrict__ order, bool key32) {
  extern __shared__ __align__(16) unsigned char order_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* ids = reinterpret_cast<int32_t*>(order_smem) + (size_t)w * kcap;
  int16_t* pos = reinterpret_cast<int16_t*>(reinterpret_cast<int32_t*>(order_smem) + (size_t)kOrderWarps * kcap) +
                 (size_t)w * kcap;
  for (int64_t t = (int64_t)blockIdx.x * kOrderWarps + w; t < n_tgt; t += (int64_t)gridDim.x * kOrderWarps) {
    const int64_t o = off[t];
    const int k = (int)(off[t + 1] - o);
    if (k <= 64) {  // short lists: keys in registers, no shared memory
      if (key32)
        order_in_registers<2, unsigned int>(idx, o, k, lane, order);
      else
        order_in_registers<2, unsigned long long>(idx, o, k, lane, order);
      continue;
    }
    if (k <= 128) {
      if (key32)
        order_in_registers<4, unsigned int>(idx, o, k, lane, order);
      else
        order_in_registers<4, unsigned long long>(idx, o, k, lane, order);
      continue;
    }
    int n2 = 1;
    while (n2 < k) n2 <<= 1;
    for (int i = lane; i < n2; i += 32) {
      ids[i] = (i < k) ? idx[o + i] : INT_MAX;
      pos[i] = (int16_t)i;
    }
    __syncwarp();
    for (int size = 2; size <= n2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = lane; i < (n2 >> 1); i += 32) {
          // stride is a power of two: a = 2 stride (i / stride) + i % stride
          const int a = ((i & ~(stride - 1)) << 1) | (i & (stride - 1)), b = a + stride;
          const bool asc = (a & size) == 0;
          const int32_t ia = ids[a], ib = ids[b];
          if ((ib < ia) == asc && ia != ib) {
            ids[a] = ib;
            ids[b] = ia;
            const int16_t pa = pos[a];
            pos[a] = pos[b];
            pos[b] = pa;
          }
        }
        __syncwarp();
      }
    }
    for (int r = lane; r < k; r += 32) order[o + r] = pos[r];
    __syncwarp();
  }
}

cudaError_t launch_nbr_order(const Launch& L, int64_t n_tgt, const int64_t* off, const int32_t* idx, int kcap,
                             int16_t* order, int64_t n_points) {
  if (n_tgt == 0) return cudaSuccess;
  if (kcap < 1 || kcap > kMaxK) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kOrderWarps * kcap * (sizeof(int32_t) + sizeof(int16_t));
  cudaError_t e = cudaFuncSetAttribute(nbr_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n_tgt + kOrderWarps - 1) / kOrderWarps;
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  const bool key32 = n_points < (int64_t(1) << 25) - 1;  // 32-bit keys (lists of up to 128 entries)
  nbr_order_kernel<<<(unsigned)blocks, kOrderWarps * 32, smem, L.stream>>>(n_tgt, off, idx, kcap, order, key32);
  *L.counter += 1;
  return cudaGetLastError();
}

// Order of the k-prefix lists: warp per target; the parent's positions are
// scanned in order, 32 at a time, and those below k are compacted (ballot).
__global__ void nbr_order_prefix_kernel(int64_t n_tgt, const int16_t* __restrict__ parent_order, int kp, int k,
                                        int16_t* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tgt;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int16_t* po = parent_order + t * kp;
    int16_t* out = order + t * k;
    int filled = 0;
    for (int i0 = 0; i0 < kp; i0 += 32) {
      const int i = i0 + lane;
      const int pos = i < kp ? (int)po[i] : k;
      const bool keep = pos < k;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) out[filled + __popc(m & ((1u << lane) - 1u))] = (int16_t)pos;
      filled += __popc(m);
    }
  }
}

cudaError_t launch_nbr_order_prefix(const Launch& L, int64_t n_tgt, const int16_t* parent_order, int kp, int k,
                                    int16_t* order) {
  if (n_tgt == 0) return cudaSuccess;
  if (k < 1 || k > kp) return cudaErrorInvalidValue;
  int64_t blocks = (n_tgt * 32 + 255) / 256;
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  nbr_order_prefix_kernel<<<(unsigned)blocks, 256, 0, L.stream>>>(n_tgt, parent_order, kp, k, order);
  *L.counter += 1;
  return cudaGetLastError();
}

// CSR of one functional from the cached id order: warp per target, every
// row's entries written in ascending column order, no sorting.  C
// (components per neighbour) is a compile-time constant.
constexpr int kCsrWarps = 8;

template <int C>
__global__ void __launch_bounds__(kCsrWarps * 32) csr_kernel(CsrJob j) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t t = (int64_t)blockIdx.x * kCsrWarps + w; t < j.n_tgt; t += (int64_t)gridDim.x * kCsrWarps) {
    const int64_t o = j.off[t];
    const int k = (int)(j.off[t + 1] - o);
    const int rowlen = k * C;
    const int64_t base = o * (int64_t)j.rows * C;
    for (int r = lane; r < j.rows; r += 32) j.row_ptr[t * j.rows + r] = j.nnz_base + base + (int64_t)r * rowlen;
    // the target's rows are contiguous: one pass over rows x rowlen entries,
    // row r and in-row position e carried along instead of divided
    const int total = j.rows * rowlen;
    int r = rowlen > 0 ? lane / rowlen : 0, e = lane - r * rowlen;  // (no entries: the loop below is empty)
    for (int g = lane; g < total; g += 32) {
      const int q = e / C, c = e - q * C;
      const int p = j.order[o + q];
      j.col[base + g] = j.idx[o + p] * C + c;
      j.val[base + g] = j.w[base + (int64_t)r * rowlen + p * C + c];
      e += 32;
      while (e >= rowlen) {
        e -= rowlen;
        ++r;
      }
    }
    if (t == j.n_tgt - 1 && lane == 0) j.row_ptr[j.n_tgt * j.rows] = j.nnz_base + base + (int64_t)j.rows * rowlen;
  }
}

// row_ptr[0] of an operator with no rows
__global__ void csr_empty_kernel(int64_t* row_ptr, int64_t nnz_base) { row_ptr[0] = nnz_base; }

cudaError_t launch_csr(const Launch& L, const CsrJob& j) {
  if (j.n_tgt == 0) {
    csr_empty_kernel<<<1, 1, 0, L.stream>>>(j.row_ptr, j.nnz_base);
    *L.counter += 1;
    return cudaGetLastError();
  }
  int64_t blocks = (j.n_tgt + kCsrWarps - 1) / kCsrWarps;
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  if (j.nc == 1)
    csr_kernel<1><<<(unsigned)blocks, kCsrWarps * 32, 0, L.stream>>>(j);
  else if (j.nc == 2)
    csr_kernel<2><<<(unsigned)blocks, kCsrWarps * 32, 0, L.stream>>>(j);
  else if (j.nc == 3)
    csr_kernel<3><<<(unsigned)blocks, kCsrWarps * 32, 0, L.stream>>>(j);
  else
    return cudaErrorInvalidValue;
  *L.counter += 1;
  return cudaGetLastError();
}

}  // namespace gmls
