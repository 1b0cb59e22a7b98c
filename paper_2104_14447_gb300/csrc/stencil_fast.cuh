// stencil_fast.cuh -- warp-per-target GMLS stencils, FP32 QR + float-float refinement.
// (kernel template; the instantiations live in fast_*.cu, the dispatch in
// stencil_fast.cu)
//
// Same mathematics as stencil.cu (Sec. 2.1 / 2.2 / 2.5 of the paper: weighted,
// eps-scaled basis matrix B = sqrt(W) P, least-squares solve through a
// Householder QR, functional rows lambda, weights w = sqrt(W) Q R^{-T}
// lambda^T), laid out for GB300:
//
//  * a group of HW lanes (a whole warp, HW = 32, half of one, HW = 16, or 8)
//    owns one target; lane l of the group holds rows l, l+HW, ... of the FP32
//    QR tile in registers (compile-time basis size N and rows-per-lane MR, so
//    the factorisation is fully unrolled); padded rows are zero and exactly
//    neutral for Householder reflections.  Half-warp groups suit systems of
//    a few dozen rows (36 rows: 48 slots on 16 lanes instead of 64 on 32),
//    and every cross-lane reduction then serves two targets at once (four on
//    8-lane groups: 40 slots for the 36 rows, at 5 rows a lane);
//  * the tile B is built directly in float-float (hi + lo, ~48 bits) from the
//    FP64 offsets x_j - x_T (one FP64 subtraction per coordinate, split into
//    float-float with integer operations), so the result does not depend on
//    where the cloud sits and no other FP64 instruction runs in the hot loop;
//  * one refinement step on the augmented system [[I, B], [B^T, 0]] [s; -y]
//    = [0; lambda^T] (Bjorck), started from s0 = B y0 in float-float (so the
//    residual f = B y0 - s0 vanishes) with g = lambda - B^T s0 in
//    compensated float-float and the correction from the FP32 factors;
//  * w = sqrt(W) s is rounded to FP64 only when stored.
//
// Neumann targets (Sec. 2.3, scalar basis) run in their own instantiation
// (NEU): the constraint F^T c = h, F = grad p(x_T)^T n, is eliminated with a
// reflector H_F on the linear columns, the pivot column moves to the end and
// the least-squares problem runs on the other N - 1 columns; beta =
// (lambda~_piv - s^T p~) / rho.  The plain instantiation appends them to the
// Neumann list when the launch has one.  Targets this path does not cover (a
// basis size other than the instantiation's, more rows than the tile holds)
// are appended to the list of the shared-memory FP32 kernel; those whose FP32
// factor is ill-conditioned or whose refinement misses its tolerance to the
// redo list of the FP64 kernel.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "basis_tables.cuh"
#include "ff.cuh"
#include "gmls_internal.cuh"

namespace gmls {

// Shared memory of one group (one target in flight), kept small so that
// twelve warps fit on an SM for the 96 x 20 systems.
template <int HW, int MR, int N, int NC, bool NEU = false>
struct FastLay {
  static constexpr int LD = HW * MR + 1;  // odd: column walks by different lanes avoid bank conflicts
  static constexpr int NQ = (HW * MR + NC - 1) / NC;            // neighbour slots
  static constexpr int NR = N * (N + 1) / 2;                    // packed upper triangle
  static constexpr size_t B = 0;                                // ff [N][LD]
  static constexpr size_t SW = B + sizeof(ff) * N * LD;         // ff [NQ]  sqrt(W) per neighbour
  static constexpr size_t R = SW + sizeof(ff) * NQ;             // float [NR] R, rows packed
  static constexpr size_t ID = R + sizeof(float) * NR;          // float [N] 1 / r_ii
  static constexpr size_t TAU = ID + sizeof(float) * N;         // float [N]
  static constexpr size_t IEPS = (TAU + sizeof(float) * N + 7) & ~size_t(7);  // ff: 1 / eps
  static constexpr size_t S = IEPS + sizeof(ff);                // ff [L][LD] s iterates
  // the rest depends on the number of solve rows L
  __host__ __device__ static size_t Y(int L) { return S + sizeof(ff) * L * LD; }      // ff [L][N]
  __host__ __device__ static size_t G(int L) { return Y(L) + sizeof(ff) * L * N; }    // float [L][N]
  // Neumann targets: lambda~ ff [L][N] after the reflection and the pivot
  // swap (entry N - 1: lambda~_piv), then rho
  __host__ __device__ static size_t LAMT(int L) { return (G(L) + sizeof(float) * L * N + 15) & ~size_t(15); }
  __host__ __device__ static size_t bytes(int L) {
    return NEU ? ((LAMT(L) + sizeof(ff) * (L * N + 1) + 15) & ~size_t(15)) : LAMT(L);
  }
};

// position of R(i, c), c >= i, in the packed rows of an N-column factor
template <int N>
__host__ __device__ __forceinline__ int rpk(int i, int c) {
  return i * (2 * N - i - 1) / 2 + c;
}

// lanes of this thread's group of HW lanes
template <int HW>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (HW == 32)
    return 0xffffffffu;
  else
    return ((1u << HW) - 1u) << ((threadIdx.x & 31) & ~(HW - 1));
}

template <int HW>
__device__ __forceinline__ float wsum(float v, unsigned mask) {
#pragma unroll
  for (int o = HW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, HW);
  return v;
}
template <int HW>
__device__ __forceinline__ float wmax(float v, unsigned mask) {
#pragma unroll
  for (int o = HW / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, HW));
  return v;
}

// All-reduce over the group of v[B..N) (compile-time range): recursive
// halving (each lane keeps the half of the values picked by its lane bit and
// adds its partner's copy of that half) for up to log2(HW) stages, butterflies
// over the remaining lane bits, then a broadcast of each total.  About
// 2(N - B) shuffles instead of log2(HW) (N - B) for independent butterflies.
template <int HW, int N, int B>
__device__ __forceinline__ void allreduce_tail(float (&v)[N], int lane, unsigned mask) {
  constexpr int C = N - B;
  constexpr int LB = HW == 32 ? 5 : HW == 16 ? 4 : HW == 8 ? 3 : 2;
  static_assert((1 << LB) == HW, "group width must be 4, 8, 16 or 32");
  if constexpr (C <= 0) {
    return;
  } else if constexpr (C <= 2) {
#pragma unroll
    for (int o = HW / 2; o > 0; o >>= 1)
#pragma unroll
      for (int c = B; c < N; ++c) v[c] += __shfl_xor_sync(mask, v[c], o, HW);
  } else {
    constexpr int P = C <= 4 ? 4 : C <= 8 ? 8 : C <= 16 ? 16 : C <= 32 ? 32 : 64;
    constexpr int LP = P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : P == 32 ? 5 : 6;
    constexpr int S = LP < LB ? LP : LB;  // halving stages
    constexpr int M = P >> S;             // totals kept per lane afterwards
    float w[P];
#pragma unroll
    for (int i = 0; i < P; ++i) w[i] = (i < C) ? v[B + (i < C ? i : 0)] : 0.0f;
    // stage st (offset HW/2 >> st) keeps P >> (st+1) values: the upper half
    // on lanes whose bit is set
#pragma unroll
    for (int st = 0; st < S; ++st) {
      const int o = (HW / 2) >> st;
      const bool up = (lane & o) != 0;
      const int h = P >> (st + 1);
#pragma unroll
      for (int i = 0; i < P / 2; ++i) {
        if (i < h) {
          const float send = up ? w[i] : w[i + h];
          const float keep = up ? w[i + h] : w[i];
          w[i] = keep + __shfl_xor_sync(mask, send, o, HW);
        }
      }
    }
    // lanes holding the same totals add up across the remaining lane bits
#pragma unroll
    for (int o = (HW / 2) >> S; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < M; ++i) w[i] += __shfl_xor_sync(mask, w[i], o, HW);
    // total c sits in w[c % M] of the lanes whose top S bits spell c / M
#pragma unroll
    for (int c = 0; c < C; ++c) v[B + c] = __shfl_sync(mask, w[c % M], (c / M) << (LB - S), HW);
  }
}

// One Householder step on column KC of the register tile: reflector from
// rows > KC, then the trailing columns (dot products all-reduced together).
template <int HW, int MR, int N, int KC>
__device__ __forceinline__ void qr_column(float (&a)[MR][N], float* tau, int lane, unsigned mask) {
  float sig = 0.0f;
#pragma unroll
  for (int i = 0; i < MR; ++i)
    if (lane + HW * i > KC) sig = fmaf(a[i][KC], a[i][KC], sig);
  sig = wsum<HW>(sig, mask);
  const float alpha = __shfl_sync(mask, a[KC / HW][KC], KC % HW, HW);
  float tk = 0.0f, beta = alpha;
  if (sig > 0.0f) {
    const float nrm = sqrtf(fmaf(alpha, alpha, sig));
    beta = alpha >= 0.0f ? -nrm : nrm;
    // approximate quotients (a few ulp): the reflector's scaling and tau
    // only need FP32 accuracy, the refinement absorbs the rest
    const float scale = __fdividef(1.0f, alpha - beta);
    tk = __fdividef(beta - alpha, beta);
#pragma unroll
    for (int i = 0; i < MR; ++i)
      if (lane + HW * i > KC) a[i][KC] *= scale;
  }
  if (lane == KC % HW) a[KC / HW][KC] = beta;
  if (lane == 0) tau[KC] = tk;
  float v[MR];
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = lane + HW * i;
    v[i] = (r > KC) ? a[i][KC] : (r == KC ? 1.0f : 0.0f);
  }
  float dots[N];
#pragma unroll
  for (int c = KC + 1; c < N; ++c) {
    float p = 0.0f;
#pragma unroll
    for (int i = 0; i < MR; ++i) p = fmaf(v[i], a[i][c], p);
    dots[c] = p;
  }
  allreduce_tail<HW, N, KC + 1>(dots, lane, mask);
#pragma unroll
  for (int c = KC + 1; c < N; ++c) {
    const float tc = dots[c] * tk;
#pragma unroll
    for (int i = 0; i < MR; ++i) a[i][c] = fmaf(-tc, v[i], a[i][c]);
  }
}

template <int HW, int MR, int N, int... K>
__device__ __forceinline__ void qr_columns(float (&a)[MR][N], float* tau, int lane, unsigned mask,
                                           std::integer_sequence<int, K...>) {
  (qr_column<HW, MR, N, K>(a, tau, lane, mask), ...);
}

// apply Q (REV: H_0 ... H_{N-1} z, i.e. reflectors in reverse order) or Q^T
// to the row-distributed vectors z[l][i], l < L
template <int HW, int MR, int N, int L, bool REV>
__device__ __forceinline__ void apply_q_regs(const float (&a)[MR][N], const float* tau, float (&z)[L][MR], int lane,
                                             unsigned mask) {
#pragma unroll
  for (int s = 0; s < N; ++s) {
    const int k = REV ? N - 1 - s : s;
    const float tk = tau[k];
    float v[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + HW * i;
      v[i] = (r > k) ? a[i][k] : (r == k ? 1.0f : 0.0f);
    }
    float d[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      d[l] = 0.0f;
#pragma unroll
      for (int i = 0; i < MR; ++i) d[l] = fmaf(v[i], z[l][i], d[l]);
    }
#pragma unroll
    for (int o = HW / 2; o > 0; o >>= 1)
#pragma unroll
      for (int l = 0; l < L; ++l) d[l] += __shfl_xor_sync(mask, d[l], o, HW);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float dl = d[l] * tk;
#pragma unroll
      for (int i = 0; i < MR; ++i) z[l][i] = fmaf(-dl, v[i], z[l][i]);
    }
  }
}

// w <- R^{-T} w (forward substitution), w[l][t] holds entry p = lane + HW t
template <int HW, int N, int L>
__device__ __forceinline__ void solve_rt_lanes(const float* Rs, const float* idg,
                                               float (&w)[L][(N + HW - 1) / HW], int lane, unsigned mask) {
  constexpr int NT = (N + HW - 1) / HW;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float inv = idg[i];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float yi = __shfl_sync(mask, w[l][i / HW], i % HW, HW) * inv;
      if (lane == i % HW) w[l][i / HW] = yi;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int p = lane + HW * t;
        if (p > i && p < N) w[l][t] = fmaf(-Rs[rpk<N>(i, p)], yi, w[l][t]);
      }
    }
  }
}

// w <- R^{-1} w (back substitution)
template <int HW, int N, int L>
__device__ __forceinline__ void solve_r_lanes(const float* Rs, const float* idg,
                                              float (&w)[L][(N + HW - 1) / HW], int lane, unsigned mask) {
  constexpr int NT = (N + HW - 1) / HW;
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const float inv = idg[i];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float yi = __shfl_sync(mask, w[l][i / HW], i % HW, HW) * inv;
      if (lane == i % HW) w[l][i / HW] = yi;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int p = lane + HW * t;
        if (p < i) w[l][t] = fmaf(-Rs[rpk<N>(p, i)], yi, w[l][t]);
      }
    }
  }
}

// Block size limit: small register tiles keep twelve warps resident (at
// most 168 registers per thread, blocks of up to 12 warps); larger ones are
// left to the register allocator (blocks of up to 8 warps).  An instantiation
// may set its own limit (GMLS_FAST_T): the 40 x 20 half-warp tile of the 3D
// degree-3 scalar basis runs faster capped at 168 registers (nine warps per
// SM, shared memory deciding, a few hundred bytes of spills) than at 254
// (eight).  The launcher takes the largest block among the shapes with the
// most resident warps, so that an SM works on consecutive targets
// (neighbours shared in L1).
template <int HW, int MR, int N, int L>
constexpr int fast_max_threads() {
  return MR * N * L <= 90 ? 384 : 256;
}

template <int KIND, int D, int DEG, int MR, int L, int HW, bool NEU = false,
          int MAXT = fast_max_threads<HW, MR, gmls_gen::basis_size(KIND, D, DEG), L>()>
__global__ void __launch_bounds__(MAXT, 1) stencil_fast_kernel(StencilJob j) {
  constexpr int NB = gmls_gen::basis_size(KIND, D, DEG);  // basis functions
  constexpr int N = NB - (NEU ? 1 : 0);                    // least-squares columns
  static_assert(!NEU || KIND == GMLS_BASIS_SCALAR, "the Neumann constraint is for the scalar basis");
  // refinement scheme: steps of one Q application each from s0 = B y0
  // (scalar and staggered bases, measured faster there), or Bjorck steps from
  // s0 = Q [R^-T lambda; 0] with both residuals (divergence-free: its one-Q
  // variant was slower on the 96 x 20 systems, 0.222 vs 0.183 ms on 8,192
  // targets, with the same number of steps allowed)
  constexpr bool ONEQ = KIND != GMLS_BASIS_DIVFREE;
  constexpr int NC = (KIND == GMLS_BASIS_DIVFREE) ? D : 1;  // components per neighbour (staggered: 1)
  constexpr int ROWS = HW * MR;
  constexpr int NT = (N + HW - 1) / HW;
  using Lay = FastLay<HW, MR, NB, NC, NEU>;
  constexpr int LD = Lay::LD;
  extern __shared__ __align__(16) unsigned char smem[];
  const int grp = threadIdx.x / HW, lane = threadIdx.x & (HW - 1);
  const int gpb = blockDim.x / HW;
  const unsigned mask = group_mask<HW>();
  unsigned char* base = smem + (size_t)grp * Lay::bytes(L);
  ff* Bs = reinterpret_cast<ff*>(base + Lay::B);
  ff* SWs = reinterpret_cast<ff*>(base + Lay::SW);
  ff* Ss = reinterpret_cast<ff*>(base + Lay::S);
  ff* Ys = reinterpret_cast<ff*>(base + Lay::Y(L));
  ff* IEPSs = reinterpret_cast<ff*>(base + Lay::IEPS);
  float* Rs = reinterpret_cast<float*>(base + Lay::R);
  float* IDs = reinterpret_cast<float*>(base + Lay::ID);
  float* TAUs = reinterpret_cast<float*>(base + Lay::TAU);
  float* Gs = reinterpret_cast<float*>(base + Lay::G(L));
  // functional row l at basis column c (float-float): integer coefficient
  // times eps^-order; Neumann targets read lambda~ from its table
  auto lam0 = [&](int l, int c) {
    ff f(gmls_gen::lam_coef_f(KIND, D, DEG, j.lam_fn[l], j.lam_row[l], c), 0.0f);
    const ff ie = IEPSs[0];
    for (int p = 0; p < j.lam_order[l]; ++p) f = f * ie;
    return f;
  };
  ff* LAMT = NEU ? reinterpret_cast<ff*>(base + Lay::LAMT(L)) : nullptr;
  auto lam = [&](int l, int c) {
    if constexpr (NEU)
      return LAMT[l * NB + c];
    else
      return lam0(l, c);
  };
  const int64_t n = j.n;
  const int64_t n_items = j.items ? (int64_t)(*j.n_items) : j.n_tgt;
  const float tolf = (float)j.tol;

  for (int64_t it = (int64_t)blockIdx.x * gpb + grp; it < n_items; it += (int64_t)gridDim.x * gpb) {
    const int64_t to = j.items ? (int64_t)j.items[it] : it;
    const int64_t t = j.tgt[to];
    const int64_t o0 = j.off[to];
    const int k = (int)(j.off[to + 1] - o0);
    const int M = k * NC;
    uint8_t st = j.nbr_status ? j.nbr_status[to] : 0;
    const bool neu = KIND == GMLS_BASIS_SCALAR && j.neumann && j.bflag && j.bflag[t] && j.normals;
    const bool too_few = (st & GMLS_T_TOO_FEW_NEIGHBOURS) || k <= 0 || !(j.eps[to] > 0.0);
    // staggered basis: the weights act on p_j - p(x_T); the target's own
    // entry (a zero row of the tile) later takes minus the sum of the others
    int self = -1;
    if constexpr (KIND == GMLS_BASIS_STAGGERED) {
      if (!too_few) {
        const int32_t* nb = j.idx + o0;
        int first = 0x7fffffff;
        for (int q = lane; q < k; q += HW)
          if (nb[q] == (int32_t)t) first = min(first, q);
#pragma unroll
        for (int o = HW / 2; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(mask, first, o, HW));
        self = first == 0x7fffffff ? -1 : first;
      }
    }
    const bool no_self = KIND == GMLS_BASIS_STAGGERED && !too_few && self < 0;
    if (!too_few && (neu != NEU || M > ROWS || M < N || no_self)) {
      // not for this instantiation: a Neumann target to the Neumann list when
      // the launch has one, anything else to the shared-memory FP32 kernel
      // (which writes every output)
      if (lane == 0) {
        if (!NEU && neu && j.neu_items) {
          const int slot = atomicAdd(j.neu_count, 1);
          j.neu_items[slot] = (int32_t)to;
        } else {
          const int slot = atomicAdd(j.gen_count, 1);
          j.gen_items[slot] = (int32_t)to;
        }
        j.status[to] = 0;
      }
      continue;
    }
    if (too_few) {
      for (int f = 0; f < j.nout; ++f) {
        const int64_t cnt = (int64_t)j.out_rows[f] * k * j.out_ncomp[f];
        double* w = j.out_w[f] + o0 * (int64_t)j.out_rows[f] * j.out_ncomp[f];
        for (int64_t e = lane; e < cnt; e += HW) w[e] = 0.0;
      }
      if (j.beta)
        for (int l = lane; l < L; l += HW) j.beta[to * L + l] = 0.0;
      if (lane == 0) {
        j.status[to] = st;
        if (j.iters) j.iters[to] = 0;
      }
      continue;
    }

    // ---- 1. float-float tile B = sqrt(W) P, rows (neighbour, component)
    const ff eps(j.eps[to]);
    const ff inv_eps = recip(eps);
    double xt[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < D; ++c) xt[c] = j.x[c * n + t];
    const int half_p = j.wpow_half;
    for (int q = lane; q < ROWS / NC; q += HW) {
      if (q < k) {
        const int32_t jj = j.idx[o0 + q];
        ff dx[3], xi[3];
        ff r2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          dx[c] = diff_ff(j.x[c * n + jj], xt[c]);
          xi[c] = dx[c] * inv_eps;
          r2 = r2 + dx[c] * dx[c];
        }
        const ff u = ff(1.f, 0.f) - sqrt_ff(r2) * inv_eps;
        ff sw(0.f, 0.f);
        if (u.h > 0.0f) {
          sw = u;
          for (int p = 1; p < half_p; ++p) sw = sw * u;
        }
        gmls_gen::BasisEval<KIND, D, DEG>::template run<ff>(xi, Bs + q * NC, LD, sw);
        SWs[q] = sw;
      } else {
        SWs[q] = ff(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
          for (int i = 0; i < NB; ++i) Bs[i * LD + q * NC + c] = ff(0.f, 0.f);
        }
      }
    }
    // rows past the last whole neighbour (ROWS not a multiple of NC)
    for (int r = (ROWS / NC) * NC + lane; r < ROWS; r += HW) {
      if (r % NC == 0) SWs[r / NC] = ff(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NB; ++i) Bs[i * LD + r] = ff(0.f, 0.f);
    }
    if (lane == 0) IEPSs[0] = inv_eps;
    __syncwarp(mask);

    if constexpr (NEU) {
      // ---- Neumann (Sec. 2.3): H_F = I - 2 v v^T / v^T v with v = F - rho
      // e_piv, F = n / eps on the linear columns 1..D (d/dx_c of the scaled
      // monomial xi_c at x_T), rho = -sign(n_piv) |F|; H_F on the linear
      // columns of every row, then columns 1 + piv and NB - 1 swap places.
      // lambda~ = H_F lambda, swapped the same way, into the table.
      int piv = 0;
      double npiv = 0.0;  // n_piv
      ff v[3], fn2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double nc = j.normals[c * n + t];
        if (c == 0 || fabs(nc) > fabs(npiv)) {
          piv = c;
          npiv = nc;
        }
        v[c] = ff(nc) * inv_eps;
        fn2 = fn2 + v[c] * v[c];
      }
      const ff fn = sqrt_ff(fn2);
      const ff rho = npiv >= 0.0 ? ff(-fn.h, -fn.l) : fn;
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c == piv) v[c] = v[c] - rho;
      ff vv(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < D; ++c) vv = vv + v[c] * v[c];
      const ff two_vv = ff(2.f, 0.f) * recip(vv);
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        const int r = lane + HW * i;
        ff d(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < D; ++c) d = d + Bs[(1 + c) * LD + r] * v[c];
        d = d * two_vv;
#pragma unroll
        for (int c = 0; c < D; ++c) Bs[(1 + c) * LD + r] = Bs[(1 + c) * LD + r] - d * v[c];
        const ff pc = Bs[(1 + piv) * LD + r];
        Bs[(1 + piv) * LD + r] = Bs[(NB - 1) * LD + r];
        Bs[(NB - 1) * LD + r] = pc;
      }
      for (int e = lane; e < L * NB; e += HW) {
        const int l = e / NB, c = e - l * NB;
        const int cs = c == 1 + piv ? NB - 1 : (c == NB - 1 ? 1 + piv : c);
        ff lv = lam0(l, cs);
        if (cs >= 1 && cs <= D) {
          ff dl(0.f, 0.f);
#pragma unroll
          for (int c2 = 0; c2 < D; ++c2) dl = dl + lam0(l, 1 + c2) * v[c2];
          dl = dl * two_vv;
          ff vc = v[0];
#pragma unroll
          for (int c2 = 1; c2 < D; ++c2)
            if (cs - 1 == c2) vc = v[c2];
          lv = lv - dl * vc;
        }
        LAMT[e] = lv;
      }
      if (lane == 0) LAMT[L * NB] = rho;
      __syncwarp(mask);
    }

    // ---- 2. FP32 Householder QR in registers
    float a[MR][N];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int c = 0; c < N; ++c) a[i][c] = Bs[c * LD + lane + HW * i].h;
    qr_columns<HW, MR, N>(a, TAUs, lane, mask, std::make_integer_sequence<int, N>{});
    // stage R, 1/r_ii; conditioning of the factor
    float rmax = 0.0f, rmin = 3.0e38f;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + HW * i;
      if (r < N) {
#pragma unroll
        for (int c = 0; c < N; ++c)
          if (c >= r) Rs[rpk<N>(r, c)] = a[i][c];
        float d = 0.0f;
#pragma unroll
        for (int c = 0; c < N; ++c)
          if (c == r) d = a[i][c];
        IDs[r] = 1.0f / d;
        rmax = fmaxf(rmax, fabsf(d));
        rmin = fminf(rmin, fabsf(d));
      }
    }
    rmax = wmax<HW>(rmax, mask);
    rmin = -wmax<HW>(-rmin, mask);
    __syncwarp(mask);
    const bool ill = !(rmin * 1.0e6f >= rmax) || !(rmin > 0.0f);

    int used = 0;
    if constexpr (ONEQ) {
    // ---- 3./4. solve and refinement.  y0 = R^-1 R^-T lambda in FP32; the
    // Bjorck steps on [[I, B], [B^T, 0]] [s; -y] = [0; lambda^T] start from
    // s0 = B y0 evaluated in float-float, so that f = B y0 - s0 = 0 and each
    // correction needs one application of Q:
    //   g = lambda - B^T s,  delta = R^-T g,  ds = Q [delta; 0],  s += ds.
    // (s0 = B y0 is as accurate as Q [R^-T lambda; 0], an error of order
    // kappa u_32, and each step contracts it by about kappa u_32.)  Up to
    // max_refine steps; targets whose correction still misses the
    // tolerance, or whose factor is ill-conditioned, go to the FP64 redo list.
    float w[L][NT];
    float z[L][MR];
    bool conv = false;
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        const int p = lane + HW * tt;
        w[l][tt] = (p < N) ? lam(l, p).h : 0.0f;
      }
    solve_rt_lanes<HW, N, L>(Rs, IDs, w, lane, mask);  // a = R^-T lambda
    solve_r_lanes<HW, N, L>(Rs, IDs, w, lane, mask);   // y0 = R^-1 a
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        const int p = lane + HW * tt;
        if (p < N) Ys[l * N + p] = ff(w[l][tt], 0.0f);
      }
    __syncwarp(mask);
    if (!ill && j.max_refine >= 1) {
      // s0 = B y0 (compensated; y0 is FP32), lanes over rows
#pragma unroll
      for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + HW * i;
          Dot2 acc;
#pragma unroll
          for (int c = 0; c < N; ++c) acc.add_prod_f(Bs[c * LD + r], Ys[l * N + c].h);
          Ss[l * LD + r] = acc.value();
        }
      }
      __syncwarp(mask);
      float prev = 0.0f;
#pragma unroll 1
      for (int it = 1; it <= j.max_refine; ++it) {
      // g = lambda - B^T s over the L*N (l, c) pairs: whole pairs per lane
      // in full rounds of HW, the remaining pairs split into row blocks so
      // that every lane does about the same number of terms
      {
        constexpr int pairs = L * N, full = pairs / HW, rem = pairs % HW;
        for (int u = 0; u < full; ++u) {
          const int e = u * HW + lane, l = e / N, c = e % N;
          // four independent compensated chains over interleaved rows (ILP)
          Dot2 acc[4];
          acc[0].init(lam(l, c));
          const ff* bc = Bs + c * LD;
          const ff* sl = Ss + l * LD;
#pragma unroll 2
          for (int r = 0; r < ROWS; r += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (r + q < ROWS) acc[q].add_prod(-bc[r + q], sl[r + q]);
          }
          const ff tot = (acc[0].value() + acc[1].value()) + (acc[2].value() + acc[3].value());
          Gs[l * N + c] = __fadd_rn(tot.h, tot.l);
        }
        if constexpr (rem > 0) {
          // pair e is split over the lanes blk * rem + (e - full HW), blk <
          // nblk; lane e - full HW gathers the partial sums by shuffles
          constexpr int nblk = HW / rem, chunk = (ROWS + nblk - 1) / nblk;
          const int e = full * HW + lane % rem, blk = lane / rem;
          const int l = e / N, c = e % N;
          Dot2 acc;
          if (blk < nblk) {
            const ff* bc = Bs + c * LD;
            const ff* sl = Ss + l * LD;
            const int r1 = min(ROWS, (blk + 1) * chunk);
            for (int r = blk * chunk; r < r1; ++r) acc.add_prod(-bc[r], sl[r]);
          }
          const ff part = (blk < nblk) ? acc.value() : ff(0.f, 0.f);
          ff sum = (lane < rem) ? lam(l, c) : ff(0.f, 0.f);
#pragma unroll
          for (int b = 0; b < nblk; ++b) {
            const int src = b * rem + lane % rem;
            const ff v(__shfl_sync(mask, part.h, src, HW), __shfl_sync(mask, part.l, src, HW));
            sum = sum + v;
          }
          if (lane < rem) Gs[l * N + c] = __fadd_rn(sum.h, sum.l);
        }
      }
      __syncwarp(mask);
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + HW * tt;
          w[l][tt] = (p < N) ? Gs[l * N + p] : 0.0f;
        }
      solve_rt_lanes<HW, N, L>(Rs, IDs, w, lane, mask);  // delta = R^-T g
      // z = [delta; 0]: rows r < N of z sit in the same lane / slot as entry p = r
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + HW * i;
          z[l][i] = (r < N && i < NT) ? w[l][i < NT ? i : 0] : 0.0f;
        }
      apply_q_regs<HW, MR, N, L, true>(a, TAUs, z, lane, mask);  // ds = Q [delta; 0]
      float dmax = 0.0f, smax = 0.0f;
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + HW * i;
          const ff s1 = add_f(Ss[l * LD + r], z[l][i]);
          Ss[l * LD + r] = s1;
          dmax = fmaxf(dmax, fabsf(z[l][i]));
          smax = fmaxf(smax, fabsf(s1.h));
        }
      dmax = wmax<HW>(dmax, mask);
      smax = wmax<HW>(smax, mask);
      __syncwarp(mask);
      // error left after the correction ~ |ds| times the contraction factor,
      // estimated by the relative size of the correction (first pass) or by
      // the ratio of successive corrections (later ones: s = s_prev + ds keeps
      // B y - s at the rounding of ds, so each pass repeats the same step)
      const float rho = it == 1 ? dmax / fmaxf(smax, 1e-37f) : dmax / fmaxf(prev, 1e-37f);
      conv = dmax * fminf(1.0f, rho) <= tolf * smax;
      prev = dmax;
      used = it;
      if (conv) break;
      }
    }
    if (!conv) {
      if (lane == 0) {
        const int slot = atomicAdd(j.fb_count, 1);
        j.fb_items[slot] = (int32_t)to;
        j.status[to] = ill ? GMLS_T_ILL_CONDITIONED : GMLS_T_REFINE_NOT_CONVERGED;
      }
      continue;
    }
    } else {
    // ---- 3./4. solve and refinement with float-float residuals.  Pass 0 is
    // the plain FP32 solve, i.e. a refinement step from s = y = 0 (f = 0,
    // g = lambda): a = R^{-T} lambda, s0 = Q [a; 0], y0 = R^{-1} a.  Passes
    // it >= 1 correct with the residuals f = B y - s and g = lambda - B^T s:
    // d = Q^T f, a = R^{-T} g, dy = R^{-1} (a - d_1), ds = Q [a; d_2].  One
    // copy of the solve code serves all passes (the kernel is large enough
    // for instruction fetch to matter).
    float w[L][NT];
    float z[L][MR];
    bool conv = false;
    float prev = 0.0f;
#pragma unroll 1
    for (int it = 0; it <= j.max_refine; ++it) {
      if (it > 0) {
        if (ill) break;
        // f = B y - s, lanes over rows
#pragma unroll
        for (int l = 0; l < L; ++l) {
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const int r = lane + HW * i;
            Dot2 acc;
            acc.init(-Ss[l * LD + r]);
#pragma unroll
            for (int c = 0; c < N; ++c) acc.add_prod(Bs[c * LD + r], Ys[l * N + c]);
            z[l][i] = __fadd_rn(acc.h, acc.l);
          }
        }
        // g = lambda - B^T s over the L*N (l, c) pairs: whole pairs per lane
        // in full rounds of HW, the remaining pairs split into row blocks so
        // that every lane does about the same number of terms
        {
          constexpr int pairs = L * N, full = pairs / HW, rem = pairs % HW;
          for (int u = 0; u < full; ++u) {
            const int e = u * HW + lane, l = e / N, c = e % N;
            // four independent compensated chains over interleaved rows (ILP)
            Dot2 acc[4];
            acc[0].init(lam(l, c));
            const ff* bc = Bs + c * LD;
            const ff* sl = Ss + l * LD;
#pragma unroll 2
            for (int r = 0; r < ROWS; r += 4) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (r + q < ROWS) acc[q].add_prod(-bc[r + q], sl[r + q]);
            }
            const ff tot = (acc[0].value() + acc[1].value()) + (acc[2].value() + acc[3].value());
            Gs[l * N + c] = __fadd_rn(tot.h, tot.l);
          }
          if constexpr (rem > 0) {
            // pair e is split over the lanes blk * rem + (e - full HW), blk <
            // nblk; lane e - full HW gathers the partial sums by shuffles
            constexpr int nblk = HW / rem, chunk = (ROWS + nblk - 1) / nblk;
            const int e = full * HW + lane % rem, blk = lane / rem;
            const int l = e / N, c = e % N;
            Dot2 acc;
            if (blk < nblk) {
              const ff* bc = Bs + c * LD;
              const ff* sl = Ss + l * LD;
              const int r1 = min(ROWS, (blk + 1) * chunk);
              for (int r = blk * chunk; r < r1; ++r) acc.add_prod(-bc[r], sl[r]);
            }
            const ff part = (blk < nblk) ? acc.value() : ff(0.f, 0.f);
            ff sum = (lane < rem) ? lam(l, c) : ff(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < nblk; ++b) {
              const int src = b * rem + lane % rem;
              const ff v(__shfl_sync(mask, part.h, src, HW), __shfl_sync(mask, part.l, src, HW));
              sum = sum + v;
            }
            if (lane < rem) Gs[l * N + c] = __fadd_rn(sum.h, sum.l);
          }
        }
        __syncwarp(mask);
        apply_q_regs<HW, MR, N, L, false>(a, TAUs, z, lane, mask);  // d = Q^T f
      } else {
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
          for (int i = 0; i < MR; ++i) z[l][i] = 0.0f;
      }
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + HW * tt;
          w[l][tt] = (p < N) ? (it > 0 ? Gs[l * N + p] : lam(l, p).h) : 0.0f;
        }
      solve_rt_lanes<HW, N, L>(Rs, IDs, w, lane, mask);  // a = R^{-T} g
      float dyv[L][NT];
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + HW * tt;
          // rows r < N of z sit in the same lane/slot as entry p = r
          dyv[l][tt] = (p < N) ? w[l][tt] - z[l][tt < MR ? tt : 0] : 0.0f;
          if (p < N && tt < MR) z[l][tt < MR ? tt : 0] = w[l][tt];
        }
      solve_r_lanes<HW, N, L>(Rs, IDs, dyv, lane, mask);   // dy
      apply_q_regs<HW, MR, N, L, true>(a, TAUs, z, lane, mask);  // ds = Q [a; d_2]
      float dmax = 0.0f, smax = 0.0f;
#pragma unroll
      for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + HW * i;
          const ff s1 = (it > 0) ? add_f(Ss[l * LD + r], z[l][i]) : ff(z[l][i], 0.0f);
          Ss[l * LD + r] = s1;
          dmax = fmaxf(dmax, fabsf(z[l][i]));
          smax = fmaxf(smax, fabsf(s1.h));
        }
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + HW * tt;
          if (p < N) Ys[l * N + p] = (it > 0) ? add_f(Ys[l * N + p], dyv[l][tt]) : ff(dyv[l][tt], 0.0f);
        }
      }
      if (it > 0) {
        dmax = wmax<HW>(dmax, mask);
        smax = wmax<HW>(smax, mask);
      }
      __syncwarp(mask);
      if (it == 0) continue;
      used = it;
      // error left after this correction ~ |ds| times the contraction factor,
      // estimated by the relative size of the correction (first refinement
      // step) or by the ratio of successive corrections (later ones)
      const float rho = (it == 1) ? dmax / fmaxf(smax, 1e-37f) : dmax / fmaxf(prev, 1e-37f);
      const float est = dmax * fminf(1.0f, rho);
      conv = est <= tolf * smax;
      prev = dmax;
      if (conv) break;
    }
    if (!conv) {
      if (lane == 0) {
        const int slot = atomicAdd(j.fb_count, 1);
        j.fb_items[slot] = (int32_t)to;
        j.status[to] = ill ? GMLS_T_ILL_CONDITIONED : GMLS_T_REFINE_NOT_CONVERGED;
      }
      continue;
    }

    }
    // ---- 5. store w = sqrt(W) s (FP64) in [row][neighbour][component]
    for (int f = 0; f < j.nout; ++f) {
      const int R = j.out_rows[f], C = j.out_ncomp[f], src = j.out_src[f];
      double* wo = j.out_w[f] + o0 * (int64_t)R * C;
      const int per_row = k * C;
      const bool div_scalar = (j.out_fn[f] == GMLS_F_DIV) && (KIND == GMLS_BASIS_SCALAR);
      const float sgn = (float)j.out_sign[f];
      for (int rr = 0; rr < R; ++rr) {
        double others = 0.0;  // staggered: sum of the row's weights but the target's own
        for (int e = lane; e < per_row; e += HW) {
          double val = 0.0;
          if (src >= 0) {
            if (div_scalar) {
              const int q = e / C, c = e % C;
              const ff s = Ss[(src + c) * LD + q] * SWs[q];  // scalar basis: one row per neighbour
              val = to_double(s);
            } else {
              const ff s = Ss[(src + rr) * LD + e] * SWs[e / NC];
              val = to_double(ff(sgn * s.h, sgn * s.l));
            }
          }
          if constexpr (KIND == GMLS_BASIS_STAGGERED) {
            if (e == self) continue;  // written below
            others += val;
          }
          __stcs(wo + (int64_t)rr * per_row + e, val);  // written once: evict first
        }
        if constexpr (KIND == GMLS_BASIS_STAGGERED) {
#pragma unroll
          for (int o = HW / 2; o > 0; o >>= 1) others += __shfl_xor_sync(mask, others, o, HW);
          if (lane == 0) wo[(int64_t)rr * per_row + self] = src >= 0 ? -others : 0.0;
        }
      }
    }
    if (j.beta) {
      if constexpr (NEU) {
        // coefficient of h: beta = (lambda~_piv - s^T p~) / rho, p~ the
        // reflected pivot column (the tile's column NB - 1)
        const ff rinv = recip(LAMT[L * NB]);
#pragma unroll
        for (int l = 0; l < L; ++l) {
          Dot2 acc;
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const int r = lane + HW * i;
            acc.add_prod(Ss[l * LD + r], Bs[(NB - 1) * LD + r]);
          }
          ff part = acc.value();
#pragma unroll
          for (int o = HW / 2; o > 0; o >>= 1)
            part = part + ff(__shfl_xor_sync(mask, part.h, o, HW), __shfl_xor_sync(mask, part.l, o, HW));
          if (lane == 0) j.beta[to * L + l] = to_double((LAMT[l * NB + NB - 1] - part) * rinv);
        }
      } else {
        for (int l = lane; l < L; l += HW) j.beta[to * L + l] = 0.0;
      }
    }
    if (lane == 0) {
      j.status[to] = st;
      if (j.iters) j.iters[to] = (uint8_t)used;
    }
    __syncwarp(mask);
  }
}

// ----------------------------------------------------------------- dispatch
struct FastEntry {
  int kind, dim, deg, mr, L, hw;
  const void* fn;
  size_t (*bytes)(int L);  // shared memory per group (target)
  bool neu;                // the Neumann instantiation
};

#define GMLS_FAST(KIND, D, DEG, MR, L, HW)                                                                            \
  FastEntry {                                                                                                          \
    KIND, D, DEG, MR, L, HW, (const void*)stencil_fast_kernel<KIND, D, DEG, MR, L, HW>,                                \
        &FastLay<HW, MR, gmls_gen::basis_size(KIND, D, DEG), (KIND == 1 ? D : 1)>::bytes, false                        \
  }
#define GMLS_FAST_T(KIND, D, DEG, MR, L, HW, MAXT)                                                                    \
  FastEntry {                                                                                                          \
    KIND, D, DEG, MR, L, HW, (const void*)stencil_fast_kernel<KIND, D, DEG, MR, L, HW, false, MAXT>,                   \
        &FastLay<HW, MR, gmls_gen::basis_size(KIND, D, DEG), (KIND == 1 ? D : 1)>::bytes, false                        \
  }
#define GMLS_FAST_NEU(D, DEG, MR, L, HW)                                                                              \
  FastEntry {                                                                                                          \
    0, D, DEG, MR, L, HW, (const void*)stencil_fast_kernel<0, D, DEG, MR, L, HW, true>,                                \
        &FastLay<HW, MR, gmls_gen::basis_size(0, D, DEG), 1, true>::bytes, true                                        \
  }
#define GMLS_FAST_NEU_T(D, DEG, MR, L, HW, MAXT)                                                                      \
  FastEntry {                                                                                                          \
    0, D, DEG, MR, L, HW, (const void*)stencil_fast_kernel<0, D, DEG, MR, L, HW, true, MAXT>,                          \
        &FastLay<HW, MR, gmls_gen::basis_size(0, D, DEG), 1, true>::bytes, true                                        \
  }

}  // namespace gmls
